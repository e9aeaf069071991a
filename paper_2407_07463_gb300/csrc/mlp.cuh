// Shapes and device image of the learned normal estimator (internal).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "mlp_judge.cuh"
#include "plic.cuh"
#include "tc.cuh"

namespace vof {

constexpr int kIn = 32;     // 27 stencil values padded to 32
constexpr int kInHL = 64;   // layer-1 K: BF16 high parts in 0..31, low parts in 32..63
constexpr int kHid = 64;
constexpr int kHidHL = 128; // layer-2/3 K: high parts in 0..63, low parts in 64..127
constexpr int kOut = 3;
constexpr int kOutP = 16;   // output rows padded to the smallest MMA N

// Weight blob (device memory, row-major, rows = outputs, columns = inputs).
// Padding rows/columns are zero.
struct MlpBlob {
    __nv_bfloat16 W1[kHid * kIn];
    __nv_bfloat16 W2[kHid * kHid];
    __nv_bfloat16 W3[kOutP * kHid];
    float b1[kHid];
    float b2[kHid];
    float b3[kOutP];
};

struct CanonFrame {
    int sign[3];  // reflection of original axis a
    int perm[3];  // canonical axis q is original axis perm[q]
};

// ---------------------------------------------------------------------------
// canonical frame (reflect so every Youngs component is >= 0, order the axes
// by increasing |Youngs component|, ties to the lower axis)

// Element i of a 3-array by selects (no local-memory indexing).
template <typename T>
__device__ __forceinline__ T pick3(const T v[3], int i) {
    return i == 0 ? v[0] : (i == 1 ? v[1] : v[2]);
}

__device__ __forceinline__ void canon_frame(const float st[27], CanonFrame& fr) {
    float y[3];
    youngs_raw(st, y);
#pragma unroll
    for (int a = 0; a < 3; ++a) fr.sign[a] = y[a] < 0.f ? -1 : 1;
    // the three compares and swaps of a sort of |y| (ties keep the lower axis)
    float v0 = fabsf(y[0]), v1 = fabsf(y[1]), v2 = fabsf(y[2]), tv;
    int p0 = 0, p1 = 1, p2 = 2, t;
    if (v1 < v0) { t = p0; p0 = p1; p1 = t; tv = v0; v0 = v1; v1 = tv; }
    if (v2 < v1) { t = p1; p1 = p2; p2 = t; tv = v1; v1 = v2; v2 = tv; }
    if (v1 < v0) { t = p0; p0 = p1; p1 = t; }
    fr.perm[0] = p0;
    fr.perm[1] = p1;
    fr.perm[2] = p2;
}

// x[q] = canonical stencil value - 1/2, canonical order (k'+1)*9+(j'+1)*3+(i'+1)
__device__ __forceinline__ void canon_input(const float st[27], const CanonFrame& fr, float x[27]) {
    const int step[3] = {1, 3, 9};
    int s[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) s[q] = pick3(fr.sign, fr.perm[q]) * pick3(step, fr.perm[q]);
#pragma unroll
    for (int kc = -1; kc <= 1; ++kc)
#pragma unroll
        for (int jc = -1; jc <= 1; ++jc)
#pragma unroll
            for (int ic = -1; ic <= 1; ++ic) {
                x[(kc + 1) * 9 + (jc + 1) * 3 + (ic + 1)] = st[13 + ic * s[0] + jc * s[1] + kc * s[2]] - 0.5f;
            }
}

__device__ __forceinline__ void canon_output(const float nc[3], const CanonFrame& fr, float n[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float v = 0.f;
#pragma unroll
        for (int q = 0; q < 3; ++q) v = fr.perm[q] == a ? (float)fr.sign[a] * nc[q] : v;
        n[a] = v;
    }
}

// BF16 split of a layer input: x ~ hi + lo with both parts representable
// (about 16 significant bits; each weight multiplies both parts).
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Store v as the pair (hi at column k, lo at column k + half) of row r of a
// K-major tile with kext columns.
__device__ __forceinline__ void store_pair(unsigned char* tile, int r, int k, int half, int kext, float v) {
    __nv_bfloat16 hi, lo;
    split_bf16(v, hi, lo);
    *reinterpret_cast<__nv_bfloat16*>(tile + tc::kmajor_offset(r, k, kext)) = hi;
    *reinterpret_cast<__nv_bfloat16*>(tile + tc::kmajor_offset(r, k + half, kext)) = lo;
}

// Eight consecutive layer inputs v[0..7] of row r (columns k0..k0+7, k0 a
// multiple of 8) as pairs: one 16-byte store of the high parts at column k0
// and one of the low parts at column k0 + half (a core-matrix row holds 8
// consecutive K elements).
__device__ __forceinline__ void store_pairs8(unsigned char* tile, int r, int k0, int half, int kext, const float v[8]) {
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        // split_bf16 on two values at once: one packed conversion per part
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(v[2 * q] - hf.x, v[2 * q + 1] - hf.y);
        hi[q] = *reinterpret_cast<const uint32_t*>(&h);
        lo[q] = *reinterpret_cast<const uint32_t*>(&l);
    }
    *reinterpret_cast<uint4*>(tile + tc::kmajor_offset(r, k0, kext)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<uint4*>(tile + tc::kmajor_offset(r, k0 + half, kext)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
}

// x[q] = canonical stencil value - 1/2 from a stencil held as a column of a
// shared-memory tile (value of cell q at col[q * stride]): the frame's
// reflections and permutation become one offset per canonical axis.
__device__ __forceinline__ void canon_input_col(const float* col, int stride, const CanonFrame& fr, float x[27]) {
    const int step[3] = {1, 3, 9};
    int s[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) s[q] = pick3(fr.sign, fr.perm[q]) * pick3(step, fr.perm[q]);
#pragma unroll
    for (int kc = -1; kc <= 1; ++kc)
#pragma unroll
        for (int jc = -1; jc <= 1; ++jc)
#pragma unroll
            for (int ic = -1; ic <= 1; ++ic)
                x[(kc + 1) * 9 + (jc + 1) * 3 + (ic + 1)] = col[(13 + ic * s[0] + jc * s[1] + kc * s[2]) * stride] - 0.5f;
}

// Weight matrix w[rows][cols] (global, BF16) into a K-major tile holding it
// twice along K: columns c and cols + c.
__device__ __forceinline__ void load_weight_pair(unsigned char* tile, const __nv_bfloat16* __restrict__ w, int rows,
                                                 int cols, int tid, int nthreads) {
    for (int idx = tid; idx < rows * cols; idx += nthreads) {
        const int o = idx / cols, i = idx % cols;
        *reinterpret_cast<__nv_bfloat16*>(tile + tc::kmajor_offset(o, i, 2 * cols)) = w[idx];
        *reinterpret_cast<__nv_bfloat16*>(tile + tc::kmajor_offset(o, cols + i, 2 * cols)) = w[idx];
    }
}

}  // namespace vof
