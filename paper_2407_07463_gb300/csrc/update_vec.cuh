// Vectorised update pass of a split sweep (Section 2.2 transport with the
// Weymouth & Yue 2010 divergence term), for grids whose rows are a multiple
// of 32 cells.  Same arithmetic as k_update; only the data movement differs:
// a lane owns VW consecutive cells of a row (16 bytes of c: 4 floats or 2
// doubles), a warp 32 * VW consecutive cells, so every load and store of c
// and u is one 16-byte access and the per-cell index work is shared by VW
// cells.  Neighbours along x come from the adjacent lane by a shuffle (or
// from the row's other end at a periodic boundary); neighbours along y and
// z are the same lane's vector in the adjacent row or plane.  The c_c and
// occupancy bit words (32 cells) are assembled from 32 / VW lanes with
// shuffles, and the next sweep's face list is appended with one shared
// atomic per warp.
#pragma once

#include "common.cuh"

namespace vof {

template <typename T>
struct VecOf;
template <>
struct VecOf<float> {
    static constexpr int W = 4;
};
template <>
struct VecOf<double> {
    static constexpr int W = 2;
};

template <typename T>
__device__ __forceinline__ void ld16(const T* __restrict__ p, T v[16 / sizeof(T)]) {
    if constexpr (sizeof(T) == 4) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(p));
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
    } else {
        const double2 q = __ldg(reinterpret_cast<const double2*>(p));
        v[0] = q.x;
        v[1] = q.y;
    }
}

template <typename T>
__device__ __forceinline__ void st16(T* p, const T v[16 / sizeof(T)]) {
    if constexpr (sizeof(T) == 4)
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
}

// Value of the cell after the lane's last one along x (periodic in the row).
template <typename T, int VW>
__device__ __forceinline__ T next_along_x(const T v[VW], const T* __restrict__ arr, int x0, int i0, int nx,
                                          int lane) {
    T n = __shfl_down_sync(0xffffffffu, v[0], 1);
    const bool row_end = i0 + VW == nx;
    if (lane == 31 || row_end) n = arr[row_end ? x0 + VW - nx : x0 + VW];
    return n;
}

// Value of the cell before the lane's first one along x (periodic in the row).
template <typename T, int VW>
__device__ __forceinline__ T prev_along_x(const T v[VW], const T* __restrict__ arr, int x0, int i0, int nx,
                                          int lane) {
    T p = __shfl_up_sync(0xffffffffu, v[VW - 1], 1);
    if (lane == 0 || i0 == 0) p = arr[i0 == 0 ? x0 + nx - 1 : x0 - 1];
    return p;
}

// OR of the lanes' VW-bit masks into 32-bit words: lane 0 of each group of
// 32 / VW lanes returns the word of its group.
template <int VW>
__device__ __forceinline__ uint32_t gather_word(uint32_t bits, int lane) {
    uint32_t w = bits << ((lane * VW) & 31);
#pragma unroll
    for (int o = 1; o < 32 / VW; o <<= 1) w |= __shfl_xor_sync(0xffffffffu, w, o);
    return w;
}

template <typename T>
__global__ void __launch_bounds__(512, 2)
    k_update_vec(const T* __restrict__ cin, T* __restrict__ cout, const T* __restrict__ ud,
                 const T* __restrict__ udn, Dims g, int d, int dn, int sweep, T sfac, T tau,
                 const T* __restrict__ flux, uint32_t* __restrict__ ccbits, uint32_t* __restrict__ occbits,
                 unsigned long long* __restrict__ nlist, long long cap, int* __restrict__ ncounts,
                 double* __restrict__ clipped) {
    constexpr int VW = VecOf<T>::W;
    constexpr int CH = 32 * VW;  // cells per warp chunk
    __shared__ int s_count;
    if (threadIdx.x == 0 && threadIdx.y == 0) s_count = 0;
    __syncthreads();
    const int lane = threadIdx.x;
    const int f = threadIdx.y;
    unsigned long long* seg = nlist + (size_t)blockIdx.x * cap;
    const size_t base = (size_t)f * g.N;
    const T* __restrict__ cf = cin + base;
    T* __restrict__ co = cout + base;
    const size_t wpf = (size_t)g.N / 32;  // bit words per field (rows are whole words)
    uint32_t* ccb = ccbits + (size_t)f * wpf;
    uint32_t* occ = occbits + (size_t)f * wpf;
    const int plane = g.nx * g.ny;
    double removed = 0.0;
    const int nchunks = (g.N + CH - 1) / CH;
    // grid-stride over the chunks: at any time the blocks work on one band
    // of consecutive chunks, so the neighbouring rows and planes a chunk
    // reads were read from DRAM by the band just before (L2 reuse)
    for (int chk = blockIdx.x; chk < nchunks; chk += gridDim.x) {
        const int xv = chk * CH + lane * VW;
        const bool valid = xv < g.N;
        // lanes past the end of the grid work on cell 0 (every index stays in
        // the grid) and write nothing
        const int x0 = valid ? xv : 0;
        const int i0 = x0 % g.nx;
        const int row = x0 / g.nx;
        const int j = row % g.ny, k = row / g.ny;
        const int ylo = j == 0 ? (g.ny - 1) * g.nx : -g.nx, yhi = j == g.ny - 1 ? -(g.ny - 1) * g.nx : g.nx;
        const int zlo = k == 0 ? (g.nz - 1) * plane : -plane, zhi = k == g.nz - 1 ? -(g.nz - 1) * plane : plane;
        const int lo_d = d == 1 ? ylo : zlo, hi_d = d == 1 ? yhi : zhi;
        const int hi_dn = dn == 1 ? yhi : zhi;

        T cx[VW], ulo[VW], uhi[VW], cl[VW], ch[VW], unl[VW], unh[VW];
        ld16(cf + x0, cx);
        ld16(ud + x0, ulo);
        ld16(udn + x0, unl);
        if (d == 0) {
            const T cprev = prev_along_x<T, VW>(cx, cf, x0, i0, g.nx, lane);
            const T cnext = next_along_x<T, VW>(cx, cf, x0, i0, g.nx, lane);
            const T unext = next_along_x<T, VW>(ulo, ud, x0, i0, g.nx, lane);
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                cl[e] = e == 0 ? cprev : cx[e - 1];
                ch[e] = e == VW - 1 ? cnext : cx[e + 1];
                uhi[e] = e == VW - 1 ? unext : ulo[e + 1];
            }
        } else {
            ld16(cf + x0 + lo_d, cl);
            ld16(cf + x0 + hi_d, ch);
            ld16(ud + x0 + hi_d, uhi);
        }
        if (dn == 0) {
            const T nnext = next_along_x<T, VW>(unl, udn, x0, i0, g.nx, lane);
#pragma unroll
            for (int e = 0; e < VW; ++e) unh[e] = e == VW - 1 ? nnext : unl[e + 1];
        } else {
            ld16(udn + x0 + hi_dn, unh);
        }
        const int sh_bits = (lane * VW) & 31;
        uint32_t ccm = 0;
        if (sweep == 0) {
#pragma unroll
            for (int e = 0; e < VW; ++e) ccm |= (above_half(cx[e]) ? 1u : 0u) << e;
            const uint32_t w = gather_word<VW>(ccm, lane);
            if (valid && (lane & (32 / VW - 1)) == 0) ccb[x0 >> 5] = w;
        } else {
            ccm = (ccb[x0 >> 5] >> sh_bits) & ((1u << VW) - 1u);
        }
        T v[VW];
        uint32_t occm = 0;
        int nflag = 0;
        uint32_t flo = 0, fhi = 0;
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            const int x = x0 + e;
            const int sl = vsign(ulo[e]), sh = vsign(uhi[e]);
            const int kl = sl == 0 ? 0 : vclass(sl > 0 ? cl[e] : cx[e]);
            const int kh = sh == 0 ? 0 : vclass(sh < 0 ? ch[e] : cx[e]);
            const bool cc = (ccm >> e) & 1u;
            T ve;
            if (kl == 0 && kh == 0 && !cc && is_exact_zero(cx[e])) {
                ve = cx[e];
            } else {
                const int xh = d == 0 ? (e < VW - 1 ? x + 1 : (i0 + VW == g.nx ? x0 + VW - g.nx : x0 + VW))
                                      : x + hi_d;
                const T s_lo = ulo[e] * sfac, s_hi = uhi[e] * sfac;
                const T F_lo = kl == 0 ? T(0) : (kl == 2 ? s_lo : flux[base + x]);
                const T F_hi = kh == 0 ? T(0) : (kh == 2 ? s_hi : flux[base + xh]);
                ve = cx[e] - (F_hi - F_lo) + (cc ? T(1) : T(0)) * (s_hi - s_lo);
                if (sweep == 2 && (ve < T(0) || ve > T(1))) {
                    const T cl0 = ve < T(0) ? T(0) : T(1);
                    if (valid) removed += (double)ve - (double)cl0;
                    ve = cl0;
                }
            }
            v[e] = ve;
            if (sweep == 2 && ve > tau) occm |= 1u << e;
            // faces of the next sweep whose donor is this cell
            const bool interf = valid && vclass(ve) == 1;
            if (interf && vsign(unl[e]) < 0) {
                flo |= 1u << e;
                ++nflag;
            }
            if (interf && vsign(unh[e]) > 0) {
                fhi |= 1u << e;
                ++nflag;
            }
        }
        if (valid) st16(co + x0, v);
        if (sweep == 2) {
            const uint32_t w = gather_word<VW>(occm, lane);
            if (valid && (lane & (32 / VW - 1)) == 0) occ[x0 >> 5] = w;
        }
        // warp-aggregated append of the flagged faces
        int incl = nflag;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        int wbase = 0;
        if (lane == 31 && incl > 0) wbase = atomicAdd(&s_count, incl);
        wbase = __shfl_sync(0xffffffffu, wbase, 31);
        int pos = wbase + incl - nflag;
        if (nflag) {
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                const int i = i0 + e;
                if ((flo >> e) & 1u) seg[pos++] = face_key(f, i, j, k);
                if ((fhi >> e) & 1u) {
                    int ih = i, jh = j, kh2 = k;
                    if (dn == 0) ih = i + 1 == g.nx ? 0 : i + 1;
                    else if (dn == 1) jh = j + 1 == g.ny ? 0 : j + 1;
                    else kh2 = k + 1 == g.nz ? 0 : k + 1;
                    seg[pos++] = face_key(f, ih, jh, kh2);
                }
            }
        }
    }
    if (sweep == 2) {
        for (int o = 16; o > 0; o >>= 1) removed += __shfl_down_sync(0xffffffffu, removed, o);
        if (lane == 0 && removed != 0.0) atomicAdd(clipped + f, removed);
    }
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) ncounts[blockIdx.x] = s_count;
}

}  // namespace vof
