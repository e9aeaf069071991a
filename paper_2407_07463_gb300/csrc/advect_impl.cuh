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
#include "boxes.cuh"
#include "faces.cuh"
#include "plic.cuh"
#include "update_vec.cuh"

namespace vof {

// Buffers and settings shared by the boxes of one advance (internal).
struct SweepArgs {
    unsigned long long* list;    // two face lists of list_entries entries each, segmented by block
    long long list_entries;      // reserved entries per list
    int* counts;                 // [2][kSweepBlocks] segment lengths
    int* offsets;                // [kSweepBlocks + 1] scan of the current counts
    int* tile_seg;               // first segment of each tile of kFaceTile listed faces
    int tile_cap;
    long long step;              // index of the first step
    double band;                 // FP64 plane-constant band (FP32 path)
    double tau;                  // occupancy threshold
    bool list_valid;             // list[list_cur] holds the first sweep's faces
    int list_cur;
    cudaStream_t stream;
    long long* launches;
    Prof* prof;
    // learned normal (FP32 path only; null = MYC everywhere)
    const MlpBlob* mlp;
    float mlp_tol;                     // residual at or below which the network is kept outright
    int* mlp_status;                   // set on a timed-out tensor-core wait
    unsigned long long* mlp_counters;  // [0] faces on the network's normal, [1] on MYC's
    // launch shape of the update pass (0 = default)
    int update_warps;                  // warps per block
    int update_blocks_per_sm;
};


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

// Rows of whole 16-byte lanes take the box kernels; others (a context only)
// the scalar update and listing.
template <typename T>
__host__ __device__ inline bool rows_vectorisable(const Dims& g) {
    return g.nx % VecOf<T>::W == 0;
}

// Grid and per-block list capacity of one advance; every producer of a list
// in it uses the same grid so that the consumers' segment walk is uniform.
struct SweepGrid {
    int gb, wpb;
    long long cap;
};

template <typename T, int NB>
SweepGrid sweep_grid(const BoxSet<T, NB>& S, bool vec, const SweepArgs& a) {
    SweepGrid r;
    if (vec) {
        constexpr int CH = 32 * VecOf<T>::W;
        r.wpb = a.update_warps > 0 ? a.update_warps : 8;
        int per_sm = a.update_blocks_per_sm;
        if (per_sm <= 0) per_sm = std::max(1, update_blocks_per_sm<T, NB>(r.wpb));
        r.gb = std::max(1, std::min(sm_count() * per_sm, kListBlocks / std::max(1, r.wpb / 8)));
        r.gb = std::min(r.gb, (S.items + r.wpb - 1) / r.wpb);
        r.gb = std::max(r.gb, 1);
        // a warp of the listing pass takes items (one field of a row chunk),
        // one of the update pass row chunks with every field
        const long long warps = (long long)r.gb * r.wpb;
        int kmax = 1;
        for (int b = 0; b < S.n; ++b) kmax = std::max(kmax, S.b[b].K);
        const long long per_warp = std::max(((long long)S.items + warps - 1) / warps,
                                            kmax * (((long long)S.chunks + warps - 1) / warps));
        r.cap = 2LL * CH * r.wpb * per_warp;
    } else {
        const Dims& g = S.b[0].g;
        const long long words = (long long)g.rows * g.W;
        const int K = S.b[0].K;
        const int per_sm = std::max(1, std::min(32, 32 / K));
        r.wpb = K;
        r.gb = (int)std::min<long long>(words, std::min<long long>(kSweepBlocks, (long long)sm_count() * per_sm));
        r.cap = 2LL * 32 * K * ((words + r.gb - 1) / r.gb);
    }
    return r;
}

template <typename T, int NB>
void face_fluxes(const BoxSet<T, NB>& S, int d, int sweep, const unsigned long long* list, long long cap, int gb,
                 SweepArgs& a) {
    if constexpr (std::is_same<T, float>::value) {
        if (a.mlp) {
            if (a.prof) a.prof->begin(P_NET_NORMALS);
            face_normals_net_set<NB>(S, d, sweep, list, cap, a.offsets, gb, a.tile_seg, a.mlp, a.mlp_status,
                                     a.stream);
            if (a.prof) { a.prof->end(); a.prof->begin(P_FACE_FLUX); }
            face_flux_judged_set<NB>(S, d, sweep, (float)a.band, list, cap, a.offsets, gb, a.tile_seg, a.mlp_tol,
                                     a.mlp_counters, a.stream);
            if (a.prof) a.prof->end();
            if (a.launches) *a.launches += 2;
            return;
        }
    }
    if (a.prof) a.prof->begin(P_FACE_FLUX);
    k_face_flux_bx<T, NB><<<sm_count() * 16, kFaceTile, 0, a.stream>>>(S, d, sweep, (T)a.band, list, cap, a.offsets, gb,
                                                                 a.tile_seg);
    if (a.prof) a.prof->end();
    if (a.launches) *a.launches += 1;
}

// nsteps steps of every box of S (Section 2.2 split advection with the
// Weymouth & Yue term; c_c bits, clip and occupancy bits as in k_update).
template <typename T, int NB>
cudaError_t advect_set(const BoxSet<T, NB>& S, SweepArgs& a, int nsteps) {
    if (S.n == 0 || nsteps <= 0) return cudaSuccess;
    const bool vec = NB > 1 || rows_vectorisable<T>(S.b[0].g);
    const SweepGrid G = sweep_grid(S, vec, a);
    if ((long long)G.gb * G.cap > a.list_entries || G.gb > kSweepBlocks) return cudaErrorInvalidValue;
    unsigned long long* lists[2] = {a.list, a.list + a.list_entries};
    int* counts[2] = {a.counts, a.counts + kSweepBlocks};
    const T tau = (T)a.tau;
    const BoxDev<T>& B0 = S.b[0];
    const Dims& g0 = B0.g;
    for (int s = 0; s < nsteps; ++s) {
        const long long step = a.step + s;
        const int rot = (int)(step % 3);
        if (!a.list_valid) {
            if (a.prof) a.prof->begin(P_FIND_FACES);
            if (vec)
                k_list_bx<T, NB><<<G.gb, 32 * G.wpb, 0, a.stream>>>(S, rot, lists[a.list_cur], G.cap,
                                                                    counts[a.list_cur]);
            else
                k_list_faces<T><<<G.gb, dim3(32, B0.K), 0, a.stream>>>(B0.c, B0.u + (size_t)rot * g0.N, g0, rot,
                                                                        lists[a.list_cur], G.cap,
                                                                        counts[a.list_cur]);
            if (a.prof) a.prof->end();
            if (a.launches) *a.launches += 1;
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        for (int sw = 0; sw < 3; ++sw) {
            const int d = (rot + sw) % 3;
            // next sweep: within the step, or the first sweep of the next step
            const int dn = sw < 2 ? (rot + sw + 1) % 3 : (int)((step + 1) % 3);
            const int cur = a.list_cur, nxt = 1 - a.list_cur;
            // every launch's error is taken where it happens (a later launch's
            // query would clear it)
            if (a.prof) a.prof->begin(P_SCAN);
            cudaError_t e = scan_face_counts(counts[cur], a.offsets, G.gb, a.tile_seg, a.tile_cap, a.stream);
            if (a.launches) *a.launches += 1;
            if (a.prof) a.prof->end();
            if (e != cudaSuccess) return e;
            face_fluxes(S, d, sw, lists[cur], G.cap, G.gb, a);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if (a.prof) a.prof->begin(P_UPDATE);
            if (vec) {
                e = launch_update_bx(S, d, dn, sw, tau, lists[nxt], G.cap, counts[nxt], G.gb, 32 * G.wpb,
                                     a.stream);
                if (e != cudaSuccess) {
                    if (a.prof) a.prof->end();
                    return e;
                }
            } else {
                const T* ins[3] = {B0.c, B0.b1, B0.b2};
                T* outs[3] = {B0.b1, B0.b2, B0.c};
                k_update<T><<<G.gb, dim3(32, B0.K), 0, a.stream>>>(
                    ins[sw], outs[sw], B0.u + (size_t)d * g0.N, B0.u + (size_t)dn * g0.N, g0, d, dn, sw, B0.sfac,
                    tau, B0.flux, B0.ccbits, B0.occbits, lists[nxt], G.cap, counts[nxt], B0.clipped);
            }
            if (a.prof) a.prof->end();
            if (a.launches) *a.launches += 1;
            a.list_cur = nxt;
        }
        a.list_valid = true;
    }
    return cudaGetLastError();
}

// The current face list after Step 4 moved drops of a single box: faces
// whose donor moved change field (k_list_patch); d is the direction of the
// sweep the list serves.  The list geometry is the one advect_set used.
template <typename T>
cudaError_t patch_list_set(const BoxSet<T, 1>& S, SweepArgs& a, int d, const uint32_t* bits, const int* labels,
                           const MoveTables& mt, const int* target) {
    if (!a.list_valid) return cudaSuccess;
    const bool vec = rows_vectorisable<T>(S.b[0].g);
    const SweepGrid G = sweep_grid(S, vec, a);
    unsigned long long* list = a.list + (a.list_cur ? a.list_entries : 0);
    const int* counts = a.counts + (a.list_cur ? kSweepBlocks : 0);
    k_list_patch<T><<<std::min(G.gb, sm_count() * 8), 256, 0, a.stream>>>(S, d, list, G.cap, counts, G.gb, bits,
                                                                         labels, mt, target);
    if (a.launches) *a.launches += 1;
    return cudaGetLastError();
}

// Listing from c and the first sweep of step a.step only (c -> first
// scratch buffer; c itself is not modified): a representative, repeatable
// unit of work for timing launch shapes.
template <typename T, int NB>
cudaError_t advect_first_sweep(const BoxSet<T, NB>& S, SweepArgs& a) {
    if (S.n == 0) return cudaSuccess;
    const bool vec = NB > 1 || rows_vectorisable<T>(S.b[0].g);
    if (!vec) return cudaErrorInvalidValue;
    const SweepGrid G = sweep_grid(S, vec, a);
    if ((long long)G.gb * G.cap > a.list_entries || G.gb > kSweepBlocks) return cudaErrorInvalidValue;
    unsigned long long* lists[2] = {a.list, a.list + a.list_entries};
    int* counts[2] = {a.counts, a.counts + kSweepBlocks};
    const int rot = (int)(a.step % 3), dn = (rot + 1) % 3;
    k_list_bx<T, NB><<<G.gb, 32 * G.wpb, 0, a.stream>>>(S, rot, lists[0], G.cap, counts[0]);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = scan_face_counts(counts[0], a.offsets, G.gb, a.tile_seg, a.tile_cap, a.stream);
    if (e != cudaSuccess) return e;
    face_fluxes(S, rot, 0, lists[0], G.cap, G.gb, a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_update_bx(S, rot, dn, 0, (T)a.tau, lists[1], G.cap, counts[1], G.gb, 32 * G.wpb, a.stream);
}

}  // namespace vof
