// Split advection over a set of independent boxes (one box for a context,
// up to kMaxBoxes for a batch): every pass of a sweep is one launch that
// covers every field of every box.
//
// The set travels by value as a __grid_constant__ kernel parameter (about
// 8 KB for 64 boxes; read in place from the parameter space), so a
// captured CUDA graph holds it and no table has to be copied to the
// device.  The update and listing passes give a warp one row chunk (32 * VW
// cells of one row of one box, VW cells per lane, 16-byte accesses) and
// walk every field of it, so that the chunk's geometry and velocities are
// taken once; chunks are numbered box by box, row by row, and the grid
// walks them in bands of consecutive chunks, so that neighbouring rows and
// planes are read close together in time (L2 reuse of c and u).  Items (one
// field of a chunk) number the same work field by field within a chunk.
// The face list of the next sweep holds 64-bit keys box | field | k | j | i.
#pragma once

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "plic.cuh"
#include "faces.cuh"
#include "tc.cuh"
#include "update_vec.cuh"

namespace vof {

// Division by a fixed positive divisor d through a multiply-high (the
// round-up method of Granlund & Montgomery 1994), exact for n < 2^31: with
// 2^(l-1) < d < 2^l, mul = ceil(2^(31+l) / d) < 2^32 and
// q = umulhi(n, mul) >> (l - 1); a power of two is a shift.
struct FastDiv {
    uint32_t mul, sh;  // mul == 0: q = n >> sh
};
__host__ inline FastDiv fastdiv_make(uint32_t d) {
    FastDiv f;
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    if ((1ull << l) == d) {
        f.mul = 0;
        f.sh = l;
    } else {
        f.mul = (uint32_t)(((1ull << (31 + l)) + d - 1) / d);
        f.sh = l - 1;
    }
    return f;
}
__device__ __forceinline__ uint32_t fastdiv(uint32_t n, const FastDiv& f) {
    return f.mul == 0 ? (n >> f.sh) : (__umulhi(n, f.mul) >> f.sh);
}

template <typename T>
struct BoxDev {
    Dims g;
    int K;      // fields advected
    int item0;  // first work item of the box
    int chunk0; // first row chunk of the box (the update pass's unit: every field of it)
    int cpr;    // row chunks per row, ceil(nx / (32 VW))
    FastDiv divK, divcpr, divny;  // by K, cpr and ny
    T sfac;     // dt / h
    T* c;       // [K][N] state (updated in place over a step)
    T* b1;      // [K][N] state after the first sweep
    T* b2;      // [K][N] state after the second sweep
    T* flux;    // [K][N] flux of listed faces, at the face's high-side cell
    const T* u; // [3][N] face velocities (low faces)
    float4* net;        // [K][N] network normal at listed faces (learned path)
    uint32_t* ccbits;   // [K][rows][W] c > 1/2 at the step start
    uint32_t* occbits;  // [K][rows][W] c > tau after the step
    double* clipped;    // [K] volume removed by the clip
};

// NB = capacity: 1 for a context, kMaxBoxes for a batch.
template <typename T, int NB>
struct BoxSet {
    int n;
    int items;   // row chunk x field, over every box
    int chunks;  // row chunks, over every box
    BoxDev<T> b[NB];
};

// Face-list key: box (6 bits) | field (4) | k | j | i (18 bits each).
__device__ __forceinline__ unsigned long long box_face_key(int box, int f, int i, int j, int k) {
    return ((unsigned long long)box << 58) | face_key(f, i, j, k);
}

template <typename T, int NB>
__device__ __forceinline__ int box_of_item(const BoxSet<T, NB>& S, int it) {
    if (NB == 1) return 0;
    int lo = 0, hi = S.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (S.b[mid].item0 <= it) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename T, int NB>
__device__ __forceinline__ int box_of_chunk(const BoxSet<T, NB>& S, int ch) {
    if (NB == 1) return 0;
    int lo = 0, hi = S.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (S.b[mid].chunk0 <= ch) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename T>
__device__ __forceinline__ const T* sweep_in(const BoxDev<T>& B, int sweep) {
    return sweep == 0 ? B.c : (sweep == 1 ? B.b1 : B.b2);
}
template <typename T>
__device__ __forceinline__ T* sweep_out(const BoxDev<T>& B, int sweep) {
    return sweep == 0 ? B.b1 : (sweep == 1 ? B.b2 : B.c);
}

// Geometry of one item for lane `lane`.
struct ItemCells {
    int f, row, j, k, i0, x0;
    bool valid;  // the lane's VW cells lie in the row
    int lo_y, hi_y, lo_z, hi_z;
};

// Geometry of row chunk `chunk` of a box for lane `lane` (f = 0).
template <typename T>
__device__ __forceinline__ ItemCells chunk_cells(const BoxDev<T>& B, int chunk, int lane) {
    constexpr int VW = VecOf<T>::W;
    const Dims& g = B.g;
    ItemCells r;
    r.f = 0;
    r.row = (int)fastdiv((uint32_t)chunk, B.divcpr);
    const int seg = chunk - r.row * B.cpr;
    const int i0 = seg * 32 * VW + lane * VW;
    r.valid = i0 < g.nx;
    // lanes past the row's end work on the row's first cells (every index
    // stays in the grid) and write nothing
    r.i0 = r.valid ? i0 : 0;
    r.x0 = r.row * g.nx + r.i0;
    r.k = (int)fastdiv((uint32_t)r.row, B.divny);
    r.j = r.row - r.k * g.ny;
    const int plane = g.nx * g.ny;
    r.lo_y = r.j == 0 ? (g.ny - 1) * g.nx : -g.nx;
    r.hi_y = r.j == g.ny - 1 ? -(g.ny - 1) * g.nx : g.nx;
    r.lo_z = r.k == 0 ? (g.nz - 1) * plane : -plane;
    r.hi_z = r.k == g.nz - 1 ? -(g.nz - 1) * plane : plane;
    return r;
}

// Geometry of item `local` (row chunk x field) of a box for lane `lane`.
template <typename T>
__device__ __forceinline__ ItemCells item_cells(const BoxDev<T>& B, int local, int lane) {
    const int chunk = (int)fastdiv((uint32_t)local, B.divK);
    ItemCells r = chunk_cells(B, chunk, lane);
    r.f = local - chunk * B.K;
    return r;
}

// Warp-aggregated append of nflag entries per lane to the block's segment;
// returns the lane's first slot.
__device__ __forceinline__ int warp_reserve(int nflag, int lane, int* s_count) {
    int incl = nflag;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    int wbase = 0;
    if (lane == 31 && incl > 0) wbase = atomicAdd(s_count, incl);
    wbase = __shfl_sync(0xffffffffu, wbase, 31);
    return wbase + incl - nflag;
}

// Faces of sweep d whose upwind donor is interfacial (start of a call, or
// after a recolouring moved drops), from the state c of every box.  A warp
// takes one row chunk and walks its fields (the velocity read once), with
// the next field's loads issued before the current one is tested.
template <typename T, int NB>
__global__ void __launch_bounds__(256) k_list_bx(const __grid_constant__ BoxSet<T, NB> S, int d,
                                                 unsigned long long* __restrict__ list, long long cap,
                                                 int* __restrict__ counts) {
    constexpr int VW = VecOf<T>::W;
    __shared__ int s_count;
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    unsigned long long* seg = list + (size_t)blockIdx.x * cap;
    for (int chk = blockIdx.x * wpb + (threadIdx.x >> 5); chk < S.chunks; chk += gridDim.x * wpb) {
        const int bx = box_of_chunk(S, chk);
        const BoxDev<T>& B = S.b[bx];
        const Dims& g = B.g;
        const ItemCells ic = chunk_cells(B, chk - B.chunk0, lane);
        const int x0 = ic.x0, i0 = ic.i0;
        const int lo_d = d == 1 ? ic.lo_y : ic.lo_z;
        const bool need_prev = lane == 0 || i0 == 0;
        const int xp = i0 == 0 ? x0 + g.nx - 1 : x0 - 1;
        // faces with a nonzero velocity, and those whose donor is the low cell
        T ul[VW];
        ld16(B.u + (size_t)d * g.N + x0, ul);
        uint32_t nz = 0, pos = 0;
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            const int sg = vsign(ul[e]);
            nz |= (ic.valid && sg != 0 ? 1u : 0u) << e;
            pos |= (sg > 0 ? 1u : 0u) << e;
        }
        T cx[VW], cl[VW], nx_[VW], nl[VW], pv = T(0), npv = T(0);
        auto load = [&](int f, T (&x)[VW], T (&l)[VW], T& p) {
            const T* cf = B.c + (size_t)f * g.N;
            ld16(cf + x0, x);
            if (d == 0) p = need_prev ? cf[xp] : T(0);
            else ld16(cf + x0 + lo_d, l);
        };
        load(0, cx, cl, pv);
        for (int f = 0; f < B.K; ++f) {
            if (f + 1 < B.K) load(f + 1, nx_, nl, npv);
            if (d == 0) {
                T cprev = __shfl_up_sync(0xffffffffu, cx[VW - 1], 1);
                if (need_prev) cprev = pv;
#pragma unroll
                for (int e = 0; e < VW; ++e) cl[e] = e == 0 ? cprev : cx[e - 1];
            }
            uint32_t fl = 0;
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                const T dn = (pos >> e) & 1u ? cl[e] : cx[e];
                fl |= (((nz >> e) & 1u) && above_zero(dn) && !at_least_one(dn) ? 1u : 0u) << e;
            }
            if (__any_sync(0xffffffffu, fl != 0)) {
                int p = warp_reserve(__popc(fl), lane, &s_count);
#pragma unroll
                for (int e = 0; e < VW; ++e)
                    if ((fl >> e) & 1u) seg[p++] = box_face_key(bx, f, i0 + e, ic.j, ic.k);
            }
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                cx[e] = nx_[e];
                cl[e] = nl[e];
            }
            pv = npv;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) counts[blockIdx.x] = s_count;
}

// Stages of the update pass's copy ring: every lane keeps kUpdStages
// (row chunk, field) items in flight through shared memory with
// asynchronous 16-byte copies (one commit group per item), so that the
// bytes in flight do not depend on registers.  A stage holds the item's
// 32 * VW values of c (512 bytes per warp) and, for a y or z sweep, the same
// chunk of its low and high neighbour rows along d; every lane reads back
// only the 16 bytes it copied itself.
constexpr int kUpdStages = 4;
constexpr int kUpdRowBytes = 512;  // 32 lanes x 16 bytes

__host__ __device__ constexpr int upd_rows(bool dx) { return dx ? 1 : 3; }
__host__ __device__ constexpr size_t upd_smem_bytes(int warps, bool dx) {
    return (size_t)warps * kUpdStages * upd_rows(dx) * kUpdRowBytes;
}

__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The scalars of one field of a row chunk that do not come through the copy
// ring: the two values beyond the chunk's ends along x that the lanes at the
// warp's or the row's ends read (x sweep) and the c_c bit word (sweeps 1, 2).
template <typename T>
struct FieldScalars {
    T pv, nv;
    uint32_t ccw;
};

template <typename T, int PH, bool DX>
__device__ __forceinline__ void load_field_scalars(FieldScalars<T>& r, const T* __restrict__ cf, bool need_prev,
                                                   int xp, bool need_next, int xn,
                                                   const uint32_t* __restrict__ ccw) {
    if (DX) {
        r.pv = need_prev ? cf[xp] : T(0);
        r.nv = need_next ? cf[xn] : T(0);
    }
    r.ccw = PH == 0 ? 0u : *ccw;
}

// The producer side of a lane's copy ring: the next (row chunk, field) item
// to fetch, with the chunk's source addresses computed once per chunk.
// Lanes past a row's end copy from the row's start (in the grid; their
// values are never used).  Every item commits one group, an empty one once
// the warp's items are exhausted, so that waiting for all but the newest
// kUpdStages - 1 groups always means the oldest item has landed.
template <typename T, int NB, int PH, bool DX>
struct UpdProducer {
    int chk, f, K, stride, chunks;
    const T* src;        // the lane's 16 bytes of field 0 of the chunk (sweep input)
    size_t field_stride; // cells per field
    int lo_d, hi_d;      // offsets of the neighbour rows along d

    __device__ __forceinline__ void locate(const BoxSet<T, NB>& S, int d, int lane) {
        if (chk >= chunks) return;
        const BoxDev<T>& B = S.b[box_of_chunk(S, chk)];
        const ItemCells ic = chunk_cells(B, chk - B.chunk0, lane);
        src = sweep_in(B, PH) + ic.x0;
        field_stride = (size_t)B.g.N;
        K = B.K;
        lo_d = d == 1 ? ic.lo_y : ic.lo_z;
        hi_d = d == 1 ? ic.hi_y : ic.hi_z;
    }
    // Copy the next item into stage `buf` and commit its group.
    __device__ __forceinline__ void issue(const BoxSet<T, NB>& S, int d, unsigned char* buf, int lane) {
        if (chk < chunks) {
            const T* row = src + (size_t)f * field_stride;
            cp_async16(buf + lane * 16, row);
            if (!DX) {
                cp_async16(buf + kUpdRowBytes + lane * 16, row + lo_d);
                cp_async16(buf + 2 * kUpdRowBytes + lane * 16, row + hi_d);
            }
            if (++f == K) {
                f = 0;
                chk += stride;
                locate(S, d, lane);
            }
        }
        cp_async_commit();
    }
};

// Update pass of sweep PH (0, 1, 2) along d (DX: d == 0) for every box (see k_update for
// the arithmetic): c_out = c_in - (F_hi - F_lo) + c_c (s_hi - s_lo), c_c
// bits written in sweep 0 and read after, the clip and the occupancy bits
// in sweep 2, and the faces of the next sweep (direction dn) whose donor is
// interfacial appended to the block's list segment.
//
// A warp takes one 32 * VW-cell row chunk at a time and walks every field
// of it: the geometry, the velocities and their signs are taken once per
// chunk.  The rows of c come through the copy ring: every lane keeps
// kUpdStages (chunk, field) items in flight with asynchronous copies,
// across the fields of a chunk and into the warp's next chunk.
template <typename T, int NB, int PH, bool DX>
__global__ void __launch_bounds__(256, 3) k_update_bx(const __grid_constant__ BoxSet<T, NB> S, int d, int dn,
                                                      T tau, unsigned long long* __restrict__ nlist,
                                                      long long cap, int* __restrict__ ncounts) {
    constexpr int VW = VecOf<T>::W;
    constexpr int ROWS = upd_rows(DX);
    extern __shared__ __align__(128) unsigned char upd_smem[];
    __shared__ int s_count;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    unsigned char* ring = upd_smem + (size_t)warp * kUpdStages * ROWS * kUpdRowBytes;
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    const int sh_bits = (lane * VW) & 31;
    unsigned long long* seg = nlist + (size_t)blockIdx.x * cap;
    const int cstride = gridDim.x * wpb;
    // producer position (lane 0 issues; every lane tracks it) and the
    // number of items in flight
    UpdProducer<T, NB, PH, DX> prod;
    prod.chk = blockIdx.x * wpb + warp;
    prod.f = 0;
    prod.stride = cstride;
    prod.chunks = S.chunks;
    prod.locate(S, d, lane);
    auto issue_next = [&](int slot) { prod.issue(S, d, ring + (size_t)slot * ROWS * kUpdRowBytes, lane); };
    for (int q = 0; q < kUpdStages; ++q) issue_next(q);
    int c_slot = 0;
    for (int chk = blockIdx.x * wpb + warp; chk < S.chunks; chk += cstride) {
        const int bx = box_of_chunk(S, chk);
        const BoxDev<T>& B = S.b[bx];
        const Dims& g = B.g;
        const ItemCells ic = chunk_cells(B, chk - B.chunk0, lane);
        const int x0 = ic.x0, i0 = ic.i0;
        const int hi_d = d == 1 ? ic.hi_y : ic.hi_z;
        const bool row_start = i0 == 0, row_end = i0 + VW == g.nx;
        const bool need_prev = lane == 0 || row_start, need_next = lane == 31 || row_end;
        const int xp = row_start ? x0 + g.nx - 1 : x0 - 1;
        const int xn = row_end ? x0 + VW - g.nx : x0 + VW;
        // offset from the lane's first cell to the high neighbour along d of
        // cell e (periodic)
        auto hi_off = [&](int e) { return DX ? (e < VW - 1 ? e + 1 : xn - x0) : e + hi_d; };
        // velocities of the chunk: signs, s = u dt / h, and the faces of the
        // next sweep that an interfacial cell lists
        T s_lo[VW], s_hi[VW];
        uint32_t lo_nz = 0, lo_pos = 0, hi_nz = 0, hi_neg = 0, nf_lo = 0, nf_hi = 0;
        {
            const T* __restrict__ ud = B.u + (size_t)d * g.N;
            const T* __restrict__ udn = B.u + (size_t)dn * g.N;
            T ulo[VW], uhi[VW], unl[VW], unh[VW];
            ld16(ud + x0, ulo);
            ld16(udn + x0, unl);
            if (DX) {
                const T unext = next_along_x<T, VW>(ulo, ud, x0, i0, g.nx, lane);
#pragma unroll
                for (int e = 0; e < VW; ++e) uhi[e] = e == VW - 1 ? unext : ulo[e + 1];
            } else {
                ld16(ud + x0 + hi_d, uhi);
            }
            if (dn == 0) {
                const T nnext = next_along_x<T, VW>(unl, udn, x0, i0, g.nx, lane);
#pragma unroll
                for (int e = 0; e < VW; ++e) unh[e] = e == VW - 1 ? nnext : unl[e + 1];
            } else {
                const int hi_dn = dn == 1 ? ic.hi_y : ic.hi_z;
                ld16(udn + x0 + hi_dn, unh);
            }
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                const int sl = vsign(ulo[e]), sh = vsign(uhi[e]);
                s_lo[e] = mul_rn(ulo[e], B.sfac);
                s_hi[e] = mul_rn(uhi[e], B.sfac);
                lo_nz |= (sl != 0 ? 1u : 0u) << e;
                lo_pos |= (sl > 0 ? 1u : 0u) << e;
                hi_nz |= (sh != 0 ? 1u : 0u) << e;
                hi_neg |= (sh < 0 ? 1u : 0u) << e;
                nf_lo |= (ic.valid && vsign(unl[e]) < 0 ? 1u : 0u) << e;
                nf_hi |= (ic.valid && vsign(unh[e]) > 0 ? 1u : 0u) << e;
            }
        }
        const size_t wpf = (size_t)g.rows * g.W;
        const size_t word0 = (size_t)ic.row * g.W + (i0 >> 5);
        const bool leader = ic.valid && (lane & (32 / VW - 1)) == 0;
        const T* __restrict__ cin = sweep_in(B, PH);
        T* __restrict__ cout = sweep_out(B, PH);
        FieldScalars<T> cur, nxt;
        load_field_scalars<T, PH, DX>(cur, cin, need_prev, xp, need_next, xn, B.ccbits + word0);
        for (int f = 0; f < B.K; ++f) {
            if (f + 1 < B.K)
                load_field_scalars<T, PH, DX>(nxt, cin + (size_t)(f + 1) * g.N, need_prev, xp, need_next, xn,
                                              B.ccbits + (size_t)(f + 1) * wpf + word0);
            // this item's rows from the ring (the stage goes back to the
            // producer once the item is done, every read of it consumed)
            cp_async_wait<kUpdStages - 1>();
            T cx[VW], cl[VW], ch[VW];
            {
                const unsigned char* sb = ring + (size_t)c_slot * ROWS * kUpdRowBytes + lane * 16;
                ld16_shared(reinterpret_cast<const T*>(sb), cx);
                if (!DX) {
                    ld16_shared(reinterpret_cast<const T*>(sb + kUpdRowBytes), cl);
                    ld16_shared(reinterpret_cast<const T*>(sb + 2 * kUpdRowBytes), ch);
                }
            }
            const size_t base = (size_t)f * g.N;
            const size_t word = (size_t)f * wpf + word0;
            if (DX) {
                T cprev = __shfl_up_sync(0xffffffffu, cx[VW - 1], 1);
                T cnext = __shfl_down_sync(0xffffffffu, cx[0], 1);
                if (need_prev) cprev = cur.pv;
                if (need_next) cnext = cur.nv;
#pragma unroll
                for (int e = 0; e < VW; ++e) {
                    cl[e] = e == 0 ? cprev : cx[e - 1];
                    ch[e] = e == VW - 1 ? cnext : cx[e + 1];
                }
            }
            uint32_t ccm = 0;
            if (PH == 0) {
                if (ic.valid) {
#pragma unroll
                    for (int e = 0; e < VW; ++e) ccm |= (above_half(cx[e]) ? 1u : 0u) << e;
                }
                const uint32_t w = gather_word<VW>(ccm, lane);
                if (leader) B.ccbits[word] = w;
            } else {
                ccm = (cur.ccw >> sh_bits) & ((1u << VW) - 1u);
            }
            // A warp whose cells and both neighbours along d are all empty
            // (class 0) and carry no c_c bit has no flux through any face:
            // every cell keeps its value and none is interfacial.
            bool any_pos = false;
#pragma unroll
            for (int e = 0; e < VW; ++e) any_pos |= above_zero(cl[e]) || above_zero(cx[e]) || above_zero(ch[e]);
            const bool quiet = !ic.valid || (ccm == 0 && !any_pos);
            T v[VW];
            uint32_t flo = 0, fhi = 0;
            int nflag = 0;
#pragma unroll
            for (int e = 0; e < VW; ++e) v[e] = cx[e];
            if (!__all_sync(0xffffffffu, quiet)) {
                const T* __restrict__ flux = B.flux + base;
#pragma unroll
                for (int e = 0; e < VW; ++e) {
                    // upwind donors through the low and high faces: empty (no
                    // flux), full (flux s) or interfacial (the listed flux)
                    const T dl = (lo_pos >> e) & 1u ? cl[e] : cx[e];
                    const T dh = (hi_neg >> e) & 1u ? ch[e] : cx[e];
                    const bool ml = ((lo_nz >> e) & 1u) && above_zero(dl);
                    const bool mh = ((hi_nz >> e) & 1u) && above_zero(dh);
                    const bool fl = at_least_one(dl), fh = at_least_one(dh);
                    const bool cc = (ccm >> e) & 1u;
                    T F_lo = ml && fl ? s_lo[e] : T(0), F_hi = mh && fh ? s_hi[e] : T(0);
                    if (ml && !fl) F_lo = flux[x0 + e];
                    if (mh && !fh) F_hi = flux[x0 + hi_off(e)];
                    // a cell that nothing enters or leaves keeps its bits (signed zero)
                    if (ml || mh || cc) v[e] = cx[e] - (F_hi - F_lo) + (cc ? T(1) : T(0)) * (s_hi[e] - s_lo[e]);
                    if (PH == 2 && (v[e] < T(0) || v[e] > T(1))) continue;  // clipped below: not interfacial
                    if (above_zero(v[e]) && !at_least_one(v[e])) {
                        flo |= nf_lo & (1u << e);
                        fhi |= nf_hi & (1u << e);
                    }
                }
                nflag = __popc(flo) + __popc(fhi);
            }
            T rem[VW];
            uint32_t occm = 0;
            bool clipped = false;
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                rem[e] = T(0);
                if (PH == 2) {
                    const bool clip = v[e] < T(0) || v[e] > T(1);
                    const T cl0 = v[e] < T(0) ? T(0) : T(1);
                    // v - cl0 is exact (Sterbenz), so the FP64 sum below sees
                    // the same terms as a sum of FP64 differences
                    rem[e] = clip && ic.valid ? v[e] - cl0 : T(0);
                    clipped |= clip && ic.valid;
                    v[e] = clip ? cl0 : v[e];
                    if (ic.valid && v[e] > tau) occm |= 1u << e;
                }
            }
            if (ic.valid) st16(cout + base + x0, v);
            if (PH == 2) {
                const uint32_t w = gather_word<VW>(occm, lane);
                if (leader) B.occbits[word] = w;
                if (__any_sync(0xffffffffu, clipped)) {
                    double removed = 0.0;
#pragma unroll
                    for (int e = 0; e < VW; ++e) removed += (double)rem[e];
                    for (int o = 16; o > 0; o >>= 1) removed += __shfl_down_sync(0xffffffffu, removed, o);
                    if (lane == 0 && removed != 0.0) atomicAdd(B.clipped + f, removed);
                }
            }
            if (__any_sync(0xffffffffu, nflag != 0)) {
                int pos = warp_reserve(nflag, lane, &s_count);
#pragma unroll
                for (int e = 0; e < VW; ++e) {
                    const int i = i0 + e;
                    if ((flo >> e) & 1u) seg[pos++] = box_face_key(bx, f, i, ic.j, ic.k);
                    if ((fhi >> e) & 1u) {
                        int ih = i, jh = ic.j, kh2 = ic.k;
                        if (dn == 0) ih = i + 1 == g.nx ? 0 : i + 1;
                        else if (dn == 1) jh = ic.j + 1 == g.ny ? 0 : ic.j + 1;
                        else kh2 = ic.k + 1 == g.nz ? 0 : ic.k + 1;
                        seg[pos++] = box_face_key(bx, f, ih, jh, kh2);
                    }
                }
            }
            cur = nxt;
            // the item's values have been used: its stage takes the item
            // kUpdStages ahead
            issue_next(c_slot);
            c_slot = c_slot + 1 == kUpdStages ? 0 : c_slot + 1;
        }
    }
    cp_async_wait<0>();  // nothing of this thread's is still in flight when it leaves
    __syncthreads();
    if (threadIdx.x == 0) ncounts[blockIdx.x] = s_count;
}

// Launch of the update pass of sweep `sweep` (0, 1, 2) along d.
// Dynamic shared memory of the copy rings; the y/z instances need more than
// the default 48 KB per block.  Every translation unit holds its own copy of
// a kernel (no relocatable device code), so the attribute is set on the copy
// this unit launches: internal linkage keeps one flag per unit and instance.
template <typename T, int NB, int PH, bool DX>
static cudaError_t update_smem_attr() {
    static bool done = false;
    if (done) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(k_update_bx<T, NB, PH, DX>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)upd_smem_bytes(8, DX));
    if (e == cudaSuccess) done = true;
    return e;
}

template <typename T, int NB, int PH>
static cudaError_t launch_update_ph(const BoxSet<T, NB>& S, int d, int dn, T tau, unsigned long long* nlist,
                                    long long cap, int* ncounts, int gb, int threads, cudaStream_t st) {
    const int warps = threads / 32;
    cudaError_t e;
    if (d == 0) {
        if ((e = update_smem_attr<T, NB, PH, true>()) != cudaSuccess) return e;
        k_update_bx<T, NB, PH, true><<<gb, threads, upd_smem_bytes(warps, true), st>>>(S, d, dn, tau, nlist, cap,
                                                                                      ncounts);
    } else {
        if ((e = update_smem_attr<T, NB, PH, false>()) != cudaSuccess) return e;
        k_update_bx<T, NB, PH, false><<<gb, threads, upd_smem_bytes(warps, false), st>>>(S, d, dn, tau, nlist, cap,
                                                                                        ncounts);
    }
    return cudaGetLastError();
}
template <typename T, int NB>
static cudaError_t launch_update_bx(const BoxSet<T, NB>& S, int d, int dn, int sweep, T tau,
                                    unsigned long long* nlist, long long cap, int* ncounts, int gb, int threads,
                                    cudaStream_t st) {
    if (sweep == 0) return launch_update_ph<T, NB, 0>(S, d, dn, tau, nlist, cap, ncounts, gb, threads, st);
    if (sweep == 1) return launch_update_ph<T, NB, 1>(S, d, dn, tau, nlist, cap, ncounts, gb, threads, st);
    return launch_update_ph<T, NB, 2>(S, d, dn, tau, nlist, cap, ncounts, gb, threads, st);
}

// Resident blocks per SM of the y/z update pass with `warps` warps per
// block, queried on the kernel copy of the unit that launches it.
template <typename T, int NB>
static int update_blocks_per_sm(int warps) {
    int per_sm = 0;
    if (update_smem_attr<T, NB, 1, false>() != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_update_bx<T, NB, 1, false>, 32 * warps,
                                                      upd_smem_bytes(warps, false)) != cudaSuccess)
        per_sm = 0;
    (void)cudaGetLastError();
    return per_sm;
}

// A listed face of a box set: box, field, the cell x of the face's high
// side, the flux index t = f N + x, the upwind donor.
struct BoxFace {
    int box, f, x, donor;
    int di, dj, dk;  // the donor's cell coordinates
    size_t t;
};

template <typename T, int NB>
__device__ __forceinline__ BoxFace decode_box_face(const BoxSet<T, NB>& S, unsigned long long key, int d, T& uv) {
    BoxFace r;
    r.box = (int)(key >> 58);
    r.f = (int)((key >> 54) & 15u);
    const int k = (int)((key >> 36) & 0x3ffffu);
    const int j = (int)((key >> 18) & 0x3ffffu);
    const int i = (int)(key & 0x3ffffu);
    const Dims& g = S.b[r.box].g;
    r.x = cell(i, j, k, g);
    r.t = (size_t)r.f * g.N + r.x;
    uv = S.b[r.box].u[(size_t)d * g.N + r.x];
    // upwind donor: the face's cell, or its low neighbour along d (periodic)
    r.di = i;
    r.dj = j;
    r.dk = k;
    if (vsign(uv) > 0) {
        if (d == 0) r.di = i == 0 ? g.nx - 1 : i - 1;
        else if (d == 1) r.dj = j == 0 ? g.ny - 1 : j - 1;
        else r.dk = k == 0 ? g.nz - 1 : k - 1;
    }
    r.donor = cell(r.di, r.dj, r.dk, g);
    return r;
}

// After Step 4 moved drops (one box): every face of the current list (the
// next sweep's faces, direction d, whose upwind donor is interfacial) whose
// donor is a cell of a moving drop now belongs to the drop's target field.
// A moved cell keeps its value and only changes field, and the target
// field held nothing occupied within reach of the drop, so the rest of the
// list stands (a target cell that held a residue below the occupancy
// threshold may end up listed twice, which writes the same flux twice).  A
// donor's tag is read only where the Step 1 snapshot marks it occupied.
template <typename T>
__global__ void __launch_bounds__(256) k_list_patch(const __grid_constant__ BoxSet<T, 1> S, int d,
                                                    unsigned long long* __restrict__ list, long long cap,
                                                    const int* __restrict__ counts, int nseg,
                                                    const uint32_t* __restrict__ bits,
                                                    const int* __restrict__ labels, MoveTables mt,
                                                    const int* __restrict__ target) {
    const Dims& g = S.b[0].g;
    const size_t wpf = (size_t)g.rows * g.W;
    for (int sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
        const int n = counts[sg];
        unsigned long long* seg = list + (size_t)sg * cap;
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            const unsigned long long key = seg[e];
            const int f = (int)((key >> 54) & 15u);
            if (mt.mv_count[f] == 0) continue;
            T uv;
            const BoxFace fc = decode_box_face(S, key, d, uv);
            const size_t row = (size_t)fc.dk * g.ny + fc.dj;
            if (!((bits[(size_t)f * wpf + row * g.W + (fc.di >> 5)] >> (fc.di & 31)) & 1u)) continue;
            const int l = labels[(size_t)f * g.N + fc.donor];
            if (!is_moving(mt, f, l)) continue;
            const int m = moving_index(mt, f, l);
            const int tg = m >= 0 ? target[m] : -1;
            if (tg >= 0) seg[e] = (key & ~(15ull << 54)) | ((unsigned long long)tg << 54);
        }
    }
}

// MYC fluxes of the listed faces of every box (one thread per face, tiles of
// kFaceTile consecutive entries whose first segment tile_seg gives).
template <typename T, int NB>
__global__ void __launch_bounds__(kFaceTile) k_face_flux_bx(const __grid_constant__ BoxSet<T, NB> S, int d,
                                                            int sweep, T band,
                                                            const unsigned long long* __restrict__ list,
                                                            long long cap, const int* __restrict__ off, int nseg,
                                                            const int* __restrict__ tile_seg) {
    const int n = off[nseg];
    for (int base = blockIdx.x * kFaceTile; base < n; base += gridDim.x * kFaceTile) {
        const int e = base + threadIdx.x;
        if (e >= n) continue;
        const int sgi = segment_from(off, tile_seg[base / kFaceTile], e);
        T uv;
        const BoxFace fc = decode_box_face(S, list[(size_t)sgi * cap + (e - off[sgi])], d, uv);
        const BoxDev<T>& B = S.b[fc.box];
        T st[27];
        gather_stencil_ijk(sweep_in(B, sweep) + (size_t)fc.f * B.g.N, fc.di, fc.dj, fc.dk, B.g, st);
        T m[3];
        myc_normal(st, m);
        const T alpha = plic_alpha_banded(m[0], m[1], m[2], st[13], band);
        B.flux[fc.t] = face_flux(m, alpha, d, uv * B.sfac);
    }
}

}  // namespace vof
