// Fluxes of one split sweep with the learned normal (FP32 path; the
// estimator has no counterpart in the paper, the fluxes are Section 2.2's).
//
// k_face_normals_net: a CTA of 128 threads takes 128 consecutive listed
// faces at a time: each thread gathers the 3x3x3 stencil of its face's
// upwind donor and writes the canonical input row, the CTA runs the network
// on the tensor cores, and each thread maps its output back to the grid
// frame and stores it at the face's cell.
//
// k_face_flux_judged: the same tiles at full occupancy.  Every thread judges
// its network normal (27-cell residual against the tolerance); the faces
// that need MYC's normal and its residual are compacted to the first
// threads of the CTA so that the fallback runs on full warps; then every
// thread takes its plane constant (the few near c = 0 or 1 refined in FP64,
// again compacted) and flux.
//
// Measured and dropped: one kernel doing both (the stencil gathered once,
// the network and the judge per tile) fits three CTAs per SM beside the
// network's shared image and ran 26% slower than the pair -- the judge
// needs the occupancy; the network's residual taken in the network kernel
// (its stencil kept in registers) moved 0.16 ms per sweep out of the judge
// and added 0.22 ms to the network; stopping MYC's residual once it
// reaches the network's saved nothing (the warp runs to its slowest lane)
// and cost 4%; splitting the tiles in two, the second half's normals and
// fluxes on a second stream beside the first half's fluxes (the judge's
// grid cut to leave a network CTA room on every SM), ran 18-29% slower
// than the pair in turn (the two kernels did not overlap usefully, and the
// judge lost the occupancy it needs); letting every thread of a tile whose
// faces all need MYC take its own face's MYC normal and residual (no
// compaction, two barriers fewer) ran 4% slower.
#include "boxes.cuh"
#include "mlp.cuh"
#include "mlp_tile.cuh"

namespace vof {

static_assert(kFaceTile == 128, "one face per thread of a 128-thread CTA");

template <int NB>
__global__ void __launch_bounds__(128, 4) k_face_normals_net(const __grid_constant__ BoxSet<float, NB> S, int d,
                                                             int sweep, const unsigned long long* __restrict__ list,
                                                             long long cap, const int* __restrict__ off,
                                                             int nseg, const int* __restrict__ tile_seg,
                                                             const MlpBlob* __restrict__ w,
                                                             int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    MlpSmem& s = *reinterpret_cast<MlpSmem*>(smem_raw);
    mlp_cta_begin(s, w);
    const uint32_t taddr = s.tbase;
    uint32_t phase = 0;
    const int t = threadIdx.x;
    const int n = off[nseg];
    // the loop bound is the same for every thread of the CTA
    for (int base = blockIdx.x * 128; base < n; base += gridDim.x * 128) {
        const int e = base + t;
        const bool valid = e < n;
        float st[27];
        float4* dst = nullptr;
        if (valid) {
            const int sgi = segment_from(off, tile_seg[base / kFaceTile], e);
            float uv;
            const BoxFace fc = decode_box_face(S, list[(size_t)sgi * cap + (e - off[sgi])], d, uv);
            const BoxDev<float>& B = S.b[fc.box];
            dst = B.net + fc.t;
            gather_stencil_ijk(sweep_in(B, sweep) + (size_t)fc.f * B.g.N, fc.di, fc.dj, fc.dk, B.g, st);
        } else {
#pragma unroll
            for (int q = 0; q < 27; ++q) st[q] = 0.5f;
        }
        CanonFrame fr;
        canon_frame(st, fr);
        // the stencil through this thread's scratch column, so that the
        // frame's offsets index shared memory rather than registers
        float* col = stencil_scratch(s) + t;
#pragma unroll
        for (int q = 0; q < 27; ++q) col[q * 128] = st[q];
        float x[27];
        canon_input_col(col, 128, fr, x);
        store_input_row(s, t, x);
        float oc[3];
        if (!mlp_tile_forward(s, taddr, phase, oc)) break;
        if (valid) {
            float nn[3];
            canon_output(oc, fr, nn);
            *dst = make_float4(nn[0], nn[1], nn[2], 0.f);
        }
    }
    mlp_cta_end(s, status);
}

// Faces per CTA of the judged flux (a thread each).  Tiles of 256 faces
// halve the barriers per face of the tile's compactions but ran 2% slower
// (longer barrier waits, four CTAs per SM instead of eight).
constexpr int kJudgeTile = 128, kJudgeWarps = kJudgeTile / 32;

template <int NB>
__global__ void __launch_bounds__(kJudgeTile) k_face_flux_judged(const __grid_constant__ BoxSet<float, NB> S, int d,
                                                          int sweep, float band,
                                                          const unsigned long long* __restrict__ list,
                                                          long long cap, const int* __restrict__ off, int nseg,
                                                          const int* __restrict__ tile_seg, float tol,
                                                          unsigned long long* __restrict__ counters) {
    __shared__ float s_st[27][kJudgeTile];  // stencil of thread t's donor in column t
    __shared__ float s_m[4][kJudgeTile];    // MYC's normal and plane constant where it replaces the network's
    __shared__ float s_enet[kJudgeTile];
    __shared__ int s_list[kJudgeTile];
    __shared__ unsigned char s_myc[kJudgeTile];
    __shared__ int s_wq[kJudgeWarps];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int n = off[nseg];
    unsigned n_net = 0, n_myc = 0, n_queued = 0;
    for (int base = blockIdx.x * kJudgeTile; base < n; base += gridDim.x * kJudgeTile) {
        const int e = base + t;
        const bool valid = e < n;
        float sv = 0.f, mn[3] = {1.f, 0.f, 0.f};
        bool net_ok = false;
        float* dst = nullptr;
        if (valid) {
            const int sgi = segment_from(off, tile_seg[base / kFaceTile], e);
            float uv;
            const BoxFace fc = decode_box_face(S, list[(size_t)sgi * cap + (e - off[sgi])], d, uv);
            const BoxDev<float>& B = S.b[fc.box];
            sv = uv * B.sfac;
            dst = B.flux + fc.t;
            float st[27];
            gather_stencil_ijk(sweep_in(B, sweep) + (size_t)fc.f * B.g.N, fc.di, fc.dj, fc.dk, B.g, st);
#pragma unroll
            for (int q = 0; q < 27; ++q) s_st[q][t] = st[q];
            const float4 nv = B.net[fc.t];
            const float nn[3] = {nv.x, nv.y, nv.z};
            net_ok = l1_normalise(nn, mn);
        }
        s_myc[t] = 0;
        __syncthreads();
        // network residual of every face; the ones above the tolerance queue,
        // in face order (a thread then reads the stencil column of its own
        // face or of one close after it: no bank conflicts when most queue)
        float al = 0.f;
        bool queue = false;
        if (valid) {
            float e_net = INFINITY;
            if (net_ok) {
                const Residual r = normal_residual_m<kJudgeTile>(&s_st[0][t], mn[0], mn[1], mn[2]);
                e_net = r.e;
                al = r.alpha;
            }
            queue = !(e_net <= tol);
            s_enet[t] = e_net;
        }
        const unsigned qb = __ballot_sync(0xffffffffu, queue);
        if (lane == 0) s_wq[warp] = __popc(qb);
        __syncthreads();
        int q_off = 0;
#pragma unroll
        int nq = 0;
#pragma unroll
        for (int w = 0; w < kJudgeWarps; ++w) {
            q_off += w < warp ? s_wq[w] : 0;
            nq += s_wq[w];
        }
        if (queue) s_list[q_off + __popc(qb & ((1u << lane) - 1u))] = t;
        __syncthreads();
        if (t == 0) n_queued += nq;
        // MYC's normal and residual for the queued faces, on the first threads
        if (t < nq) {
            const int u = s_list[t];
            float stl[27], m[3], am;
#pragma unroll
            for (int q = 0; q < 27; ++q) stl[q] = s_st[q][u];
            myc_normal(stl, m);
            const Residual rm = normal_residual_m<kJudgeTile>(&s_st[0][u], m[0], m[1], m[2]);
            am = rm.alpha;
            if (!(s_enet[u] <= rm.e)) {
                s_m[0][u] = m[0];
                s_m[1][u] = m[1];
                s_m[2][u] = m[2];
                s_m[3][u] = am;
                s_myc[u] = 1;
            }
        }
        __syncthreads();
        float m[3] = {mn[0], mn[1], mn[2]};
        if (valid) {
            if (s_myc[t]) {
                m[0] = s_m[0][t];
                m[1] = s_m[1][t];
                m[2] = s_m[2][t];
                al = s_m[3][t];
                ++n_myc;
            } else {
                ++n_net;
            }
        }
        // the residual's FP32 plane constant, refined in FP64 near c = 0 or 1:
        // those faces are compacted to the first threads (in face order), so
        // that few warps issue the FP64 steps
        const float cv = s_st[13][t];
        const bool in_band = valid && (cv < band || cv > 1.f - band);
        const unsigned bb = __ballot_sync(0xffffffffu, in_band);
        __syncthreads();  // s_m, s_list and s_wq are free again
        if (lane == 0) s_wq[warp] = __popc(bb);
        if (in_band) {
            s_m[0][t] = m[0];
            s_m[1][t] = m[1];
            s_m[2][t] = m[2];
        }
        __syncthreads();
        int b_off = 0;
#pragma unroll
        int nb = 0;
#pragma unroll
        for (int w = 0; w < kJudgeWarps; ++w) {
            b_off += w < warp ? s_wq[w] : 0;
            nb += s_wq[w];
        }
        if (in_band) s_list[b_off + __popc(bb & ((1u << lane) - 1u))] = t;
        __syncthreads();
        if (t < nb) {
            const int u = s_list[t];
            s_m[3][u] = plic_alpha_banded(s_m[0][u], s_m[1][u], s_m[2][u], s_st[13][u], band);
        }
        __syncthreads();
        if (in_band) al = s_m[3][t];
        if (valid) *dst = face_flux(m, al, d, sv);
        __syncthreads();  // the tile's shared arrays are reused by the next tile
    }
    n_net = __reduce_add_sync(0xffffffffu, n_net);
    n_myc = __reduce_add_sync(0xffffffffu, n_myc);
    if ((t & 31) == 0 && counters) {
        if (n_net) atomicAdd(&counters[0], (unsigned long long)n_net);
        if (n_myc) atomicAdd(&counters[1], (unsigned long long)n_myc);
    }
    if (t == 0 && counters && n_queued) atomicAdd(&counters[2], (unsigned long long)n_queued);
}

template <int NB>
void face_normals_net_set(const BoxSet<float, NB>& S, int d, int sweep, const unsigned long long* list, long long cap,
                          const int* off, int nseg, const int* tile_seg, const MlpBlob* w, int* status,
                          cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_face_normals_net<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(MlpSmem));
        attr = true;
    }
    k_face_normals_net<NB><<<sm_count() * 4, 128, sizeof(MlpSmem), st>>>(S, d, sweep, list, cap, off, nseg, tile_seg, w,
                                                                  status);
}

template <int NB>
void face_flux_judged_set(const BoxSet<float, NB>& S, int d, int sweep, float band, const unsigned long long* list,
                          long long cap, const int* off, int nseg, const int* tile_seg, float tol,
                          unsigned long long* counters, cudaStream_t st) {
    k_face_flux_judged<NB><<<sm_count() * (16 * 128 / kJudgeTile), kJudgeTile, 0, st>>>(S, d, sweep, band, list, cap, off, nseg, tile_seg, tol, counters);
}

#define VOF_LEARNED_SET(NB)                                                                                       \
    template void face_normals_net_set<NB>(const BoxSet<float, NB>&, int, int, const unsigned long long*,         \
                                           long long, const int*, int, const int*, const MlpBlob*, int*,          \
                                           cudaStream_t);                                                         \
    template void face_flux_judged_set<NB>(const BoxSet<float, NB>&, int, int, float, const unsigned long long*,  \
                                           long long, const int*, int, const int*, float, unsigned long long*,    \
                                           cudaStream_t);
VOF_LEARNED_SET(1)
VOF_LEARNED_SET(kMaxBoxes)
#undef VOF_LEARNED_SET

}  // namespace vof
