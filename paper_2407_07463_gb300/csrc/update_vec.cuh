// 16-byte-lane helpers of the vectorised sweep passes: a lane owns VW
// consecutive cells of a row (4 floats or 2 doubles), a warp 32 * VW, so
// every load and store of c and u is one 16-byte access.  Neighbours along
// x come from the adjacent lane by a shuffle (or from the row's other end at
// a periodic boundary); c_c and occupancy bit words (32 cells) are
// assembled from 32 / VW lanes with shuffles.
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

// 16 bytes from shared memory.
template <typename T>
__device__ __forceinline__ void ld16_shared(const T* p, T v[16 / sizeof(T)]) {
    if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
    } else {
        const double2 q = *reinterpret_cast<const double2*>(p);
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

}  // namespace vof
