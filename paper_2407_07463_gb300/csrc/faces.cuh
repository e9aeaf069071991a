// Listed-face helpers shared by the sweep kernels (internal).
#pragma once

#include "common.cuh"

namespace vof {

// 3x3x3 stencil of cell (i, j, k) (periodic), st[(k+1)*9 + (j+1)*3 + (i+1)].
template <typename T>
__device__ __forceinline__ void gather_stencil_ijk(const T* __restrict__ cf, int i, int j, int k, const Dims& g,
                                                   T st[27]) {
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

}  // namespace vof
