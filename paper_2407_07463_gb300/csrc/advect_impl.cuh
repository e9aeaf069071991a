// Directionally split geometric advection of the active colour fields
// (Section 2.2 transport of every C_i; Section 2.3: one transport equation
// per tracer), two launches per sweep:
//
//   face_flux  one thread per listed face whose upwind donor is interfacial
//              (0 < c < 1): MYC normal and plane constant of the donor, PLIC
//              volume of the swept sub-cell.  Listing keeps the costly
//              reconstruction on full warps.  With a learned normal the FP32
//              path runs face_flux_learned instead (tiles of 128 listed
//              faces through the network on the tensor cores).
//   update     one warp per 32-cell row segment, looping over the fields so
//              the velocity is read once: c <- c - (F_hi - F_lo) +
//              c_c (s_hi - s_lo) with c_c = [c > 1/2] at the step's start
//              (Weymouth & Yue 2010); empty/full donors give F = 0 / s.  The
//              same pass lists the faces of the NEXT sweep whose donor is
//              interfacial, records c_c as bits in the first sweep, and in
//              the last sweep clips to [0,1] and writes the occupancy bits
//              used by the near-contact test.
//
// The step therefore reads and writes c once per sweep; derived quantities
// (normals, plane constants, fluxes) never leave the chip.
#pragma once

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "plic.cuh"
#include "update_vec.cuh"

namespace vof {

struct AdvectArgs {
    Dims g;
    int K;                       // fields advected (the active ones)
    int Kcap;                    // fields stored (sizes the face lists)
    void* c;                     // [K][N] state, updated in place
    const void* u;               // [3][N]
    void* buf1;                  // [K][N] scratch
    void* buf2;                  // [K][N] scratch
    void* flux;                  // [K][N] scratch (listed faces only)
    unsigned long long* list;    // [2][K*N] face lists (current, next), segmented by block
    int* counts;                 // [2][kSweepBlocks] segment lengths
    int* offsets;                // [kSweepBlocks + 1] scan of the current counts
    uint32_t* ccbits;            // [K][rows][W] c > 1/2 at the step start
    uint32_t* occbits;           // [K][rows][W] occupancy after the step
    double* clipped;             // [K] accumulated clip volume
    double dt, h;
    long long step;
    double band;
    double tau;                  // occupancy threshold in the element type's terms
    bool list_valid;             // list[cur] holds the first sweep's faces
    int list_cur;                // which of the two lists is current
    cudaStream_t stream;
    long long* launches;
    Prof* prof;
    // learned normal (FP32 path only; null = MYC everywhere)
    const MlpBlob* mlp;
    float4* net;                         // [K][N] network normal of each listed face's cell
    int* tile_seg;                       // first segment of each tile of kFaceTile listed faces
    int tile_cap;
    float mlp_tol;                       // residual below which the network is kept outright
    int* mlp_status;                     // set on a timed-out tensor-core wait
    unsigned long long* mlp_counters;    // [0] faces on the network's normal, [1] on MYC's
};

template <typename T>
__device__ __forceinline__ void gather_stencil(const T* __restrict__ cf, int x, const Dims& g, T st[27]) {
    int i, j, k;
    decode(x, g, i, j, k);
    int im = i == 0 ? g.nx - 1 : i - 1, ip = i == g.nx - 1 ? 0 : i + 1;
    int jm = j == 0 ? g.ny - 1 : j - 1, jp = j == g.ny - 1 ? 0 : j + 1;
    int km = k == 0 ? g.nz - 1 : k - 1, kp = k == g.nz - 1 ? 0 : k + 1;
    const int is[3] = {im, i, ip}, js[3] = {jm, j, jp}, ks[3] = {km, k, kp};
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) st[c * 9 + b * 3 + a] = cf[cell(is[a], js[b], ks[c], g)];
}

// Face lists are segmented by block: block b of the listing kernels owns
// list[b * cap .. b * cap + count[b]), filled through a shared-memory counter,
// so no global atomic is contended.

// Contiguous range of row-segment words of one block, walked without
// divisions: (wi, j, k) advance like an odometer.
struct WordWalk {
    int gw, end, wi, j, k, rowbase;
    __device__ __forceinline__ WordWalk(const Dims& g, int nblocks) {
        const int words = g.rows * g.W;
        const int per = (words + nblocks - 1) / nblocks;
        gw = blockIdx.x * per;
        end = min(gw + per, words);
        const int row = gw / g.W;
        wi = gw - row * g.W;
        j = row % g.ny;
        k = row / g.ny;
        rowbase = row * g.nx;
    }
    __device__ __forceinline__ void next(const Dims& g) {
        ++gw;
        if (++wi == g.W) {
            wi = 0;
            rowbase += g.nx;
            if (++j == g.ny) {
                j = 0;
                ++k;
            }
        }
    }
};


// Warp-aggregated append to a block's shared counter; every lane calls it.
__device__ __forceinline__ int block_append(bool flag, int* s_count) {
    const unsigned mask = __ballot_sync(0xffffffffu, flag);
    if (mask == 0) return -1;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(s_count, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    return flag ? base + __popc(mask & ((1u << lane) - 1u)) : -1;
}

// Initial listing (start of vof_step): faces of sweep d with an interfacial
// donor.  Block = one 32-cell row segment for every field (warp y = field).
template <typename T>
__global__ void __launch_bounds__(512) k_list_faces(const T* __restrict__ cin, const T* __restrict__ ud, Dims g,
                                                    int d, unsigned long long* __restrict__ list, long long cap,
                                                    int* __restrict__ counts) {
    __shared__ int s_count;
    if (threadIdx.x == 0 && threadIdx.y == 0) s_count = 0;
    __syncthreads();
    const int lane = threadIdx.x;
    const int f = threadIdx.y;
    unsigned long long* seg = list + (size_t)blockIdx.x * cap;
    for (WordWalk ww(g, gridDim.x); ww.gw < ww.end; ww.next(g)) {
        const int i = ww.wi * 32 + lane, j = ww.j, k = ww.k;
        const bool in = i < g.nx;
        const int x = ww.rowbase + (in ? i : 0);
        const int sg = in ? vsign(ud[x]) : 0;
        const int donor = sg > 0 ? step_cell(x, i, j, k, d, -1, g) : x;
        const bool flag = sg != 0 && vclass(cin[(size_t)f * g.N + donor]) == 1;
        const int slot = block_append(flag, &s_count);
        if (slot >= 0) seg[slot] = face_key(f, i, j, k);
    }
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) counts[blockIdx.x] = s_count;
}

// Flat index space over the segments: off[b] = first entry of segment b
// (exclusive scan of the counts), off[nseg] = total.
__device__ __forceinline__ int segment_of(const int* __restrict__ off, int nseg, int e) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Segment of entry e >= base given the segment sb of base: a short forward
// walk (a tile of consecutive entries spans few segments).
__device__ __forceinline__ int segment_from(const int* __restrict__ off, int sb, int e) {
    while (off[sb + 1] <= e) ++sb;
    return sb;
}

// Decoded listed face: field f, cell x of the face's high side, the cell
// index t = f * N + x of its flux, the upwind donor cell.
struct ListedFace {
    int f, x, donor;
    size_t t;
};

// uv receives the face velocity ud[x]; the donor is upwind of the face.
template <typename T>
__device__ __forceinline__ ListedFace decode_face(unsigned long long key, const Dims& g, int d,
                                                  const T* __restrict__ ud, T& uv) {
    ListedFace r;
    r.f = (int)(key >> 54);
    const int k = (int)((key >> 36) & 0x3ffffu);
    const int j = (int)((key >> 18) & 0x3ffffu);
    const int i = (int)(key & 0x3ffffu);
    r.x = cell(i, j, k, g);
    r.t = (size_t)r.f * g.N + r.x;
    uv = ud[r.x];
    r.donor = vsign(uv) > 0 ? step_cell(r.x, i, j, k, d, -1, g) : r.x;
    return r;
}

// One thread per listed face, CTA-contiguous tiles of kFaceTile faces
// (tile_seg gives each tile's first segment): MYC normal, plane constant
// and PLIC flux of the donor.
template <typename T>
__global__ void __launch_bounds__(kFaceTile) k_face_flux(const T* __restrict__ cin, const T* __restrict__ ud,
                                                         Dims g, int d, T sfac, T band,
                                                         const unsigned long long* __restrict__ list,
                                                         long long cap, const int* __restrict__ off, int nseg,
                                                         const int* __restrict__ tile_seg, T* __restrict__ flux) {
    const int n = off[nseg];
    for (int base = blockIdx.x * kFaceTile; base < n; base += gridDim.x * kFaceTile) {
        const int e = base + threadIdx.x;
        if (e >= n) continue;
        const int sgi = segment_from(off, tile_seg[base / kFaceTile], e);
        T uv;
        const ListedFace fc = decode_face(list[(size_t)sgi * cap + (e - off[sgi])], g, d, ud, uv);
        const T s = uv * sfac;
        T st[27];
        gather_stencil(cin + (size_t)fc.f * g.N, fc.donor, g, st);
        T m[3];
        myc_normal(st, m);
        const T alpha = plic_alpha_banded(m[0], m[1], m[2], st[13], band);
        flux[fc.t] = face_flux(m, alpha, d, s);
    }
}

template <typename T>
__device__ __forceinline__ T face_value(int kind, T s, const T* __restrict__ flux, size_t t) {
    return kind == 0 ? T(0) : (kind == 2 ? s : flux[t]);
}

// sweep: 0 first (records c_c bits from cin = c at the step start), 1
// middle, 2 last (clip + occupancy bits).  dn = next sweep's direction.  A
// block walks a contiguous range of 32-cell row segments for every field
// (warp y = field); each warp issues the loads of UW segments before using
// any of them, so that enough bytes are in flight to cover DRAM latency.
constexpr int UW = 2;

template <typename T>
__global__ void __launch_bounds__(512, 2) k_update(const T* __restrict__ cin, T* __restrict__ cout,
                                                const T* __restrict__ ud, const T* __restrict__ udn, Dims g,
                                                int d, int dn, int sweep, T sfac, T tau,
                                                const T* __restrict__ flux, uint32_t* __restrict__ ccbits,
                                                uint32_t* __restrict__ occbits,
                                                unsigned long long* __restrict__ nlist, long long cap,
                                                int* __restrict__ ncounts, double* __restrict__ clipped) {
    __shared__ int s_count;
    if (threadIdx.x == 0 && threadIdx.y == 0) s_count = 0;
    __syncthreads();
    const int lane = threadIdx.x;
    const int f = threadIdx.y;
    unsigned long long* seg = nlist + (size_t)blockIdx.x * cap;
    const size_t wstride = (size_t)g.rows * g.W;  // words per field
    const size_t base = (size_t)f * g.N;
    const T* cf = cin + base;
    T* co = cout + base;
    uint32_t* ccb = ccbits + (size_t)f * wstride;
    uint32_t* occ = occbits + (size_t)f * wstride;
    double removed = 0.0;  // volume removed by the clip (last sweep), per thread
    WordWalk ww(g, gridDim.x);
    while (ww.gw < ww.end) {
        int gwv[UW], iv[UW], jv[UW], kv[UW], xv[UW], xlv[UW], xhv[UW];
        bool inv[UW], ok[UW];
        T ulo[UW], uhi[UW], cxv[UW], clv[UW], chv[UW], unl[UW], unh[UW];
        uint32_t ccw[UW];
#pragma unroll
        for (int q = 0; q < UW; ++q) {
            ok[q] = ww.gw < ww.end;
            gwv[q] = ww.gw;
            const int ii = ww.wi * 32 + lane;
            jv[q] = ww.j;
            kv[q] = ww.k;
            inv[q] = ok[q] && ii < g.nx;
            // lanes past the end of a ragged row work on the row's first
            // cell (all their neighbour indices stay inside the grid) and
            // write nothing
            iv[q] = inv[q] ? ii : 0;
            xv[q] = ww.rowbase + iv[q];
            if (ok[q]) ww.next(g);
        }
#pragma unroll
        for (int q = 0; q < UW; ++q) {
            if (!ok[q]) continue;
            const int x = xv[q];
            xlv[q] = step_cell(x, iv[q], jv[q], kv[q], d, -1, g);
            xhv[q] = step_cell(x, iv[q], jv[q], kv[q], d, +1, g);
            ulo[q] = inv[q] ? ud[x] : T(0);
            uhi[q] = inv[q] ? ud[xhv[q]] : T(0);
            cxv[q] = inv[q] ? cf[x] : T(0);
            clv[q] = cf[xlv[q]];
            chv[q] = cf[xhv[q]];
            unl[q] = inv[q] ? udn[x] : T(0);
            unh[q] = inv[q] ? udn[step_cell(x, iv[q], jv[q], kv[q], dn, +1, g)] : T(0);
            ccw[q] = sweep == 0 ? 0u : ccb[gwv[q]];
        }
#pragma unroll
        for (int q = 0; q < UW; ++q) {
            if (!ok[q]) continue;
            const bool in = inv[q];
            const int x = xv[q], xh = xhv[q], i = iv[q], j = jv[q], k = kv[q];
            const int sl = vsign(ulo[q]), sh = vsign(uhi[q]);
            const T cx = cxv[q];
            const int kl = sl == 0 ? 0 : vclass(sl > 0 ? clv[q] : cx);
            const int kh = sh == 0 ? 0 : vclass(sh < 0 ? chv[q] : cx);
            bool cc;
            if (sweep == 0) {
                cc = above_half(cx);
                const unsigned m = __ballot_sync(0xffffffffu, in && cc);
                if (lane == 0) ccb[gwv[q]] = m;
            } else {
                cc = (ccw[q] >> lane) & 1u;
            }
            T v;
            if (kl == 0 && kh == 0 && !cc && is_exact_zero(cx)) {
                v = cx;
            } else {
                const T s_lo = ulo[q] * sfac, s_hi = uhi[q] * sfac;
                const T F_lo = face_value(kl, s_lo, flux, base + x);
                const T F_hi = face_value(kh, s_hi, flux, base + xh);
                const T ccv = cc ? T(1) : T(0);
                v = cx - (F_hi - F_lo) + ccv * (s_hi - s_lo);
                if (sweep == 2 && (v < T(0) || v > T(1))) {
                    const T cl = v < T(0) ? T(0) : T(1);
                    removed += (double)v - (double)cl;
                    v = cl;
                }
            }
            if (in) co[x] = v;
            if (sweep == 2) {
                const unsigned m = __ballot_sync(0xffffffffu, in && v > tau);
                if (lane == 0) occ[gwv[q]] = m;
            }
            // faces of the next sweep whose donor is this cell
            const bool interf = in && vclass(v) == 1;
            const int snl = vsign(unl[q]), snh = vsign(unh[q]);
            int ih = i, jh = j, kh2 = k;
            if (dn == 0) ih = i + 1 == g.nx ? 0 : i + 1;
            else if (dn == 1) jh = j + 1 == g.ny ? 0 : j + 1;
            else kh2 = k + 1 == g.nz ? 0 : k + 1;
            const int s1 = block_append(interf && snl < 0, &s_count);
            if (s1 >= 0) seg[s1] = face_key(f, i, j, k);
            const int s2 = block_append(interf && snh > 0, &s_count);
            if (s2 >= 0) seg[s2] = face_key(f, ih, jh, kh2);
        }
    }
    if (sweep == 2) {
        // warp y is field f: one atomic per warp
        for (int o = 16; o > 0; o >>= 1) removed += __shfl_down_sync(0xffffffffu, removed, o);
        if (lane == 0 && removed != 0.0) atomicAdd(clipped + f, removed);
    }
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) ncounts[blockIdx.x] = s_count;
}

template <typename T>
cudaError_t advect_steps_t(AdvectArgs& a, int nsteps) {
    const Dims& g = a.g;
    if (a.K == 0 || nsteps <= 0) return cudaSuccess;
    const T sfac = (T)(a.dt / a.h);
    const T band = (T)a.band;
    const T tau = (T)a.tau;
    const T* u = (const T*)a.u;
    T* c = (T*)a.c;
    T* b1 = (T*)a.buf1;
    T* b2 = (T*)a.buf2;
    T* fl = (T*)a.flux;
    const long long words = (long long)g.rows * g.W;
    // persistent-size grid: as many (32 x K)-thread blocks as fit on the
    // SMs at 64 registers per thread, each walking a long range of words
    const int per_sm = std::max(1, std::min(32, 32 / a.K));
    // rows of whole 32-cell words take the vectorised update (16-byte lanes)
    const bool vec = g.nx % 32 == 0;
    int gb = (int)std::min<long long>(words, std::min<long long>(kSweepBlocks, 152LL * per_sm));
    if (vec) {
        // one resident wave of (32 x K)-thread blocks
        int resident = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_update_vec<T>, 32 * a.K, 0) != cudaSuccess ||
            resident < 1)
            resident = per_sm;
        gb = std::min(152 * resident, 2048);
    }
    // list segment per block: at most 2 faces per cell and field of the
    // block's cells (words per block = ceil(words / gb); chunks of 32 * VW
    // cells for the vectorised pass); gb * cap stays within the reserved span
    long long cap = 2LL * 32 * a.K * ((words + gb - 1) / gb);
    if (vec) {
        const long long CH = 32LL * VecOf<T>::W, nch = ((long long)g.N + CH - 1) / CH;
        cap = std::max(cap, 2LL * a.K * CH * ((nch + gb - 1) / gb));
    }
    // second list after the first list's reserved span (see the workspace layout)
    unsigned long long* lists[2] = {a.list, a.list + (size_t)2 * 32 * a.Kcap * ((size_t)words + kSweepBlocks)};
    int* counts[2] = {a.counts, a.counts + kSweepBlocks};
    for (int s = 0; s < nsteps; ++s) {
        const long long step = a.step + s;
        const int rot = (int)(step % 3);
        const T* ins[3] = {c, b1, b2};
        T* outs[3] = {b1, b2, c};
        if (!a.list_valid) {
            if (a.prof) a.prof->begin(P_FIND_FACES);
            k_list_faces<T><<<gb, dim3(32, a.K), 0, a.stream>>>(c, u + (size_t)rot * g.N, g, rot, lists[a.list_cur],
                                                                 cap, counts[a.list_cur]);
            if (a.prof) a.prof->end();
            if (a.launches) *a.launches += 1;
        }
        for (int sw = 0; sw < 3; ++sw) {
            const int d = (rot + sw) % 3;
            // next sweep: within the step, or the first sweep of the next step
            const int dn = sw < 2 ? (rot + sw + 1) % 3 : (int)((step + 1) % 3);
            const T* ud = u + (size_t)d * g.N;
            const T* udn = u + (size_t)dn * g.N;
            const int cur = a.list_cur, nxt = 1 - a.list_cur;
            if (a.prof) a.prof->begin(P_FACE_FLUX);
            scan_face_counts(counts[cur], a.offsets, gb, a.tile_seg, a.tile_cap, a.stream);
            bool learned = false;
            if constexpr (std::is_same<T, float>::value) {
                if (a.mlp) {
                    // network normals of the listed faces (tensor cores), then the judged fluxes
                    learned = true;
                    if (a.prof) { a.prof->end(); a.prof->begin(P_NET_NORMALS); }
                    face_normals_net(ins[sw], ud, g, d, lists[cur], cap, a.offsets, gb, a.tile_seg, a.net,
                                     a.mlp, a.mlp_status, a.stream);
                    if (a.prof) { a.prof->end(); a.prof->begin(P_FACE_FLUX); }
                    face_flux_judged(ins[sw], ud, g, d, sfac, band, lists[cur], cap, a.offsets, gb, a.tile_seg,
                                     fl, a.net, a.mlp_tol, a.mlp_counters, a.stream);
                    if (a.launches) *a.launches += 1;
                }
            }
            if (!learned)
                k_face_flux<T><<<152 * 16, kFaceTile, 0, a.stream>>>(ins[sw], ud, g, d, sfac, band, lists[cur],
                                                                      cap, a.offsets, gb, a.tile_seg, fl);
            if (a.prof) { a.prof->end(); a.prof->begin(P_UPDATE); }
            if (vec)
                k_update_vec<T><<<gb, dim3(32, a.K), 0, a.stream>>>(ins[sw], outs[sw], ud, udn, g, d, dn, sw, sfac,
                                                                     tau, fl, a.ccbits, a.occbits, lists[nxt], cap,
                                                                     counts[nxt], a.clipped);
            else
                k_update<T><<<gb, dim3(32, a.K), 0, a.stream>>>(ins[sw], outs[sw], ud, udn, g, d, dn, sw, sfac, tau,
                                                                 fl, a.ccbits, a.occbits, lists[nxt], cap, counts[nxt],
                                                                 a.clipped);
            if (a.prof) a.prof->end();
            a.list_cur = nxt;
            if (a.launches) *a.launches += 3;  // scan, flux, update
        }
        a.list_valid = true;
    }
    return cudaGetLastError();
}

}  // namespace vof
