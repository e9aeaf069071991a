// Shapes and device image of the learned normal estimator (internal).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "plic.cuh"

namespace vof {

constexpr int kIn = 32;     // 27 stencil values padded to 32
constexpr int kInHL = 64;   // layer-1 K: BF16 high parts in 0..31, low parts in 32..63
constexpr int kHid = 64;
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

__device__ __forceinline__ void canon_frame(const float st[27], CanonFrame& fr) {
    float y[3];
    youngs_raw(st, y);
    float ay[3];
    for (int a = 0; a < 3; ++a) {
        fr.sign[a] = y[a] < 0.f ? -1 : 1;
        ay[a] = fabsf(y[a]);
    }
    int p0 = 0, p1 = 1, p2 = 2, t;
    if (ay[p1] < ay[p0]) { t = p0; p0 = p1; p1 = t; }
    if (ay[p2] < ay[p1]) { t = p1; p1 = p2; p2 = t; }
    if (ay[p1] < ay[p0]) { t = p0; p0 = p1; p1 = t; }
    fr.perm[0] = p0;
    fr.perm[1] = p1;
    fr.perm[2] = p2;
}

// x[q] = canonical stencil value - 1/2, canonical order (k'+1)*9+(j'+1)*3+(i'+1)
__device__ __forceinline__ void canon_input(const float st[27], const CanonFrame& fr, float x[27]) {
    for (int kc = -1; kc <= 1; ++kc)
        for (int jc = -1; jc <= 1; ++jc)
            for (int ic = -1; ic <= 1; ++ic) {
                int o[3] = {0, 0, 0};
                const int cv[3] = {ic, jc, kc};
                for (int q = 0; q < 3; ++q) o[fr.perm[q]] = fr.sign[fr.perm[q]] * cv[q];
                x[(kc + 1) * 9 + (jc + 1) * 3 + (ic + 1)] = VOF_ST(st, o[0], o[1], o[2]) - 0.5f;
            }
}

__device__ __forceinline__ void canon_output(const float nc[3], const CanonFrame& fr, float n[3]) {
    for (int q = 0; q < 3; ++q) n[fr.perm[q]] = (float)fr.sign[fr.perm[q]] * nc[q];
}

// BF16 split of an input: x ~ hi + lo with both parts representable.
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Residual of a normal n on a stencil: plane through the centre cell with
// the centre's volume fraction, extended into the six face neighbours; the
// largest |predicted - actual| fraction.  (Judge of the learned normal.)
__device__ __forceinline__ float normal_residual(const float st[27], const float n[3]) {
    const float l1 = fabsf(n[0]) + fabsf(n[1]) + fabsf(n[2]);
    if (!(l1 > 0.f) || !isfinite(l1)) return INFINITY;
    const float m0 = n[0] / l1, m1 = n[1] / l1, m2 = n[2] / l1;
    const float al = plic_alpha<float>(m0, m1, m2, st[13]);
    float e = 0.f;
    const int off[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const float a = al - (m0 * off[q][0] + m1 * off[q][1] + m2 * off[q][2]);
        const float v = plic_volume<float>(m0, m1, m2, a);
        e = fmaxf(e, fabsf(v - VOF_ST(st, off[q][0], off[q][1], off[q][2])));
    }
    return e;
}

}  // namespace vof
