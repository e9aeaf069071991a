// Judge of the learned normal (internal; the estimator has no counterpart
// in the paper): the residual of a normal on its 3x3x3 stencil and the
// choice between the network's normal and MYC's.
#pragma once

#include <math.h>
#include <stdint.h>

#include "plic.cuh"

namespace vof {

// L1-normalised copy of a normal; false for a zero or non-finite one.
__device__ __forceinline__ bool l1_normalise(const float n[3], float m[3]) {
    const float l1 = fabsf(n[0]) + fabsf(n[1]) + fabsf(n[2]);
    if (!(l1 > 0.f) || !isfinite(l1)) return false;
    m[0] = n[0] / l1;
    m[1] = n[1] / l1;
    m[2] = n[2] / l1;
    return true;
}

// Residual of an L1-normalised normal m on a stencil: the plane of normal m
// holding the centre cell's volume fraction, extended over the 3x3x3 block;
// the mean over the 27 cells of |predicted - actual| fraction, with that
// plane's constant (FP32).  The reflection and ordering of the normal
// and the constants of its volume are taken once per stencil; every cell
// then takes the piecewise closed form (vol_pw_clamped, which gives 0 or 1
// for a cell the plane leaves whole) in one branch-free pass -- a first pass
// that settled the whole cells by a compare and a loop over the cut ones
// cost 27% more instructions, the loop running to the largest cut count of
// the warp.  The value of cell q is st[q * STRIDE] (STRIDE > 1: a
// column of a shared-memory tile).
struct Residual {
    float e;      // mean |predicted - actual| over the 27 cells
    float alpha;  // the plane constant
};
template <int STRIDE>
static __device__ __noinline__ Residual normal_residual_m(const float* st, float m0, float m1, float m2) {
    // x_i -> 1 - x_i for a negative component moves the constant by |m_i|
    const float off = fmaxf(-m0, 0.f) + fmaxf(-m1, 0.f) + fmaxf(-m2, 0.f);
    float a = fabsf(m0), b = fabsf(m1), c = fabsf(m2);
    sort3(a, b, c);
    const VolPW p = vol_pw_make(a, b, c);
    // the plane constant in the reflected frame, and in the grid's
    const float A = alpha_pw(p, st[13 * STRIDE]);
    float e = 0.f;
    // one rolled loop over the three planes along z keeps the code small
    // enough for the instruction cache; each plane's 9 cells are unrolled
#pragma unroll 1
    for (int k = -1; k <= 1; ++k) {
        const float* sk = st + (k + 1) * 9 * STRIDE;
        const float mk = m2 * (float)k;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const int i = q % 3 - 1, j = q / 3 - 1;
            e += fabsf(vol_pw_clamped(p, A - (m0 * i + m1 * j + mk)) - sk[q * STRIDE]);
        }
    }
    return {e * (1.f / 27.f), A - off};
}

// Residual of any normal n (+inf for a zero or non-finite one).
__device__ __forceinline__ float normal_residual(const float st[27], const float n[3]) {
    float m[3];
    if (!l1_normalise(n, m)) return INFINITY;
    return normal_residual_m<1>(st, m[0], m[1], m[2]).e;
}

// The learned normal as the step uses it: the network's normal nn (original
// frame, L1-normalised by division) is kept when the residual of its plane
// is at most tol, or no larger than that of MYC's normal; otherwise MYC's.
// m gets the choice; returns true when the network's was kept.
__device__ __forceinline__ bool judged_normal(const float st[27], const float nn[3], float tol, float m[3]) {
    float mn[3];
    const float e_net = l1_normalise(nn, mn) ? normal_residual_m<1>(st, mn[0], mn[1], mn[2]).e : INFINITY;
    bool keep = e_net <= tol;
    if (!keep) {
        myc_normal(st, m);
        keep = e_net <= normal_residual_m<1>(st, m[0], m[1], m[2]).e;
    }
    if (keep) {
        m[0] = mn[0];
        m[1] = mn[1];
        m[2] = mn[2];
    }
    return keep;
}

}  // namespace vof
