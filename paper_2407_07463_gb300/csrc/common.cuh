// Shared device/host helpers of the GB300 VoF library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vof.h"

namespace vof {

// Tri-periodic grid; cell index x = (k*ny + j)*nx + i fits in int32.
struct Dims {
    int nx, ny, nz;
    int N;        // nx*ny*nz
    int W;        // 32-bit words per occupancy row: ceil(nx/32)
    int rows;     // ny*nz
};

__host__ __device__ inline Dims make_dims(int nx, int ny, int nz) {
    Dims d;
    d.nx = nx;
    d.ny = ny;
    d.nz = nz;
    d.N = nx * ny * nz;
    d.W = (nx + 31) / 32;
    d.rows = ny * nz;
    return d;
}

// Product rounded on its own, never fused into a neighbouring add, so that
// every instantiation of a kernel rounds it the same way.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

__device__ __forceinline__ int wrapi(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// i mod n for -n <= i < 2n (an index at most one period outside [0, n)).
__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ void decode(int x, const Dims& g, int& i, int& j, int& k) {
    i = x % g.nx;
    int r = x / g.nx;
    j = r % g.ny;
    k = r / g.ny;
}

__device__ __forceinline__ int cell(int i, int j, int k, const Dims& g) {
    return (k * g.ny + j) * g.nx + i;
}

// Face-list entry: the face is the low face (along a sweep) of cell
// (i, j, k) of field f, packed so that decoding needs no division.
__device__ __forceinline__ unsigned long long face_key(int f, int i, int j, int k) {
    return ((unsigned long long)f << 54) | ((unsigned long long)k << 36) | ((unsigned long long)j << 18) |
           (unsigned long long)i;
}

// Neighbour of x one cell along axis d in direction dir (+1/-1), periodic.
__device__ __forceinline__ int step_cell(int x, int i, int j, int k, int d, int dir, const Dims& g) {
    if (d == 0) {
        int ii = i + dir;
        ii = ii < 0 ? g.nx - 1 : (ii >= g.nx ? 0 : ii);
        return x - i + ii;
    } else if (d == 1) {
        int jj = j + dir;
        jj = jj < 0 ? g.ny - 1 : (jj >= g.ny ? 0 : jj);
        return x + (jj - j) * g.nx;
    } else {
        int kk = k + dir;
        kk = kk < 0 ? g.nz - 1 : (kk >= g.nz ? 0 : kk);
        return x + (kk - k) * g.nx * g.ny;
    }
}

// Classification of a volume fraction: 0 empty (v <= 0), 1 interfacial,
// 2 full (v >= 1).  The double version uses integer compares on the bit
// pattern so that cells far from interfaces cost no FP64 instructions.
__device__ __forceinline__ int vclass(double v) {
    long long b = __double_as_longlong(v);
    if (b <= 0) return 0;  // +0, negative numbers and -0
    if (b >= 0x3FF0000000000000LL) return 2;
    return 1;
}
__device__ __forceinline__ int vclass(float v) {
    return v <= 0.f ? 0 : (v >= 1.f ? 2 : 1);
}
// The two tests vclass is made of: v > 0 and v >= 1 (integer compares of
// the bit pattern for double, as there).
__device__ __forceinline__ bool above_zero(double v) { return __double_as_longlong(v) > 0; }
__device__ __forceinline__ bool above_zero(float v) { return v > 0.f; }
__device__ __forceinline__ bool at_least_one(double v) {
    return __double_as_longlong(v) >= 0x3FF0000000000000LL;
}
__device__ __forceinline__ bool at_least_one(float v) { return v >= 1.f; }
__device__ __forceinline__ bool is_exact_zero(double v) {
    return (__double_as_longlong(v) << 1) == 0;
}
__device__ __forceinline__ bool is_exact_zero(float v) {
    return v == 0.f;
}
// c > 1/2 (the Weymouth-Yue indicator c_c).
__device__ __forceinline__ bool above_half(double v) {
    return __double_as_longlong(v) > 0x3FE0000000000000LL;
}
__device__ __forceinline__ bool above_half(float v) {
    return v > 0.5f;
}
// Sign of a velocity: +1, -1 or 0 (for +-0).
__device__ __forceinline__ int vsign(double v) {
    long long b = __double_as_longlong(v);
    if ((b << 1) == 0) return 0;
    return b > 0 ? 1 : -1;
}
__device__ __forceinline__ int vsign(float v) {
    return v > 0.f ? 1 : (v < 0.f ? -1 : 0);
}

// Warp-aggregated append of `flag` lanes to list[*count ...]; every lane of
// the warp must call it.  Returns the slot (or -1).
__device__ __forceinline__ long long warp_append(bool flag, unsigned long long* count) {
    unsigned mask = __ballot_sync(0xffffffffu, flag);
    if (mask == 0) return -1;
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (!flag) return -1;
    return (long long)(base + __popc(mask & ((1u << lane) - 1u)));
}

// Bits of cells x0 .. x0+31 (periodic in nx) of one occupancy row.
__device__ __forceinline__ uint32_t row_window(const uint32_t* __restrict__ row, int W, int nx, int x0) {
    x0 %= nx;
    if (x0 < 0) x0 += nx;
    if ((nx & 31) == 0) {
        int w = x0 >> 5, sh = x0 & 31;
        uint32_t lo = row[w];
        if (sh == 0) return lo;
        uint32_t hi = row[w + 1 == W ? 0 : w + 1];
        return __funnelshift_r(lo, hi, sh);
    }
    if (x0 + 32 <= nx) {
        int w = x0 >> 5, sh = x0 & 31;
        uint32_t lo = row[w];
        if (sh == 0) return lo;
        return __funnelshift_r(lo, row[w + 1], sh);
    }
    uint32_t r = 0;
    int x = x0;
    for (int b = 0; b < 32; ++b) {
        r |= ((row[x >> 5] >> (x & 31)) & 1u) << b;
        if (++x == nx) x = 0;
    }
    return r;
}

// Bits x0 + dx .. x0 + dx + 31 from the words left, centre and right of x0
// (|dx| < 32).
__device__ __forceinline__ uint32_t shift_window(uint32_t l, uint32_t c, uint32_t r, int dx) {
    if (dx == 0) return c;
    if (dx > 0) return __funnelshift_r(c, r, dx);
    return __funnelshift_l(l, c, -dx);
}

__device__ __forceinline__ bool bit_at(const uint32_t* __restrict__ bits, int W, int row, int i) {
    return (bits[(size_t)row * W + (i >> 5)] >> (i & 31)) & 1u;
}

// Streaming multiprocessors of the current device, queried once per device
// (grids are sized in multiples of it); 152 if the query fails.
inline int sm_count() {
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        (void)cudaGetLastError();
        return 152;
    }
    if (cached[dev] <= 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            (void)cudaGetLastError();
            v = 152;
        }
        cached[dev] = v;
    }
    return cached[dev];
}

inline int grid_for(long long work, int threads, int max_blocks = 0) {
    if (max_blocks <= 0) max_blocks = sm_count() * 32;
    long long b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

}  // namespace vof
