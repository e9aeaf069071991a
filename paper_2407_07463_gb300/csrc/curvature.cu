// Curvature of each colour field by height functions and the surface-tension
// source f = sum_i gamma kappa_i grad C_i (Section 2.3: with N(t) tracers
// the capillary force is the sum of every tracer's contribution, each with
// its own curvature computed as for a single tracer).
//
// Curvature of an interfacial cell (0 < c < 1): the axis a of the largest
// |component| of the cell's Mixed-Youngs-Centred normal (ties to the lower
// axis); the 3x3 columns of 7 cells along a (offsets -3..3) centred on the
// cell and its neighbours across a hold the heights H = sum of c.  Every
// column must contain the interface -- its end on the c = 1 side (opposite
// the normal) above 1/2, the other end below 1/2 -- else the cell has no
// curvature (NaN).  With f_x, f_y, f_xx, f_yy, f_xy the centred
// differences of H (cell units),
//   kappa = -[f_xx (1 + f_y^2) + f_yy (1 + f_x^2) - 2 f_xy f_x f_y]
//           / (1 + f_x^2 + f_y^2)^(3/2) / h,
// the divergence of the normal pointing out of the c = 1 phase (2/R for a
// drop of radius R).  One thread per cell; the cells that are not
// interfacial only write NaN.
#include "common.cuh"
#include "internal.h"
#include "plic.cuh"

namespace vof {

template <typename T>
__device__ __forceinline__ T nan_of();
template <>
__device__ __forceinline__ double nan_of<double>() { return __longlong_as_double(0x7ff8000000000000LL); }
template <>
__device__ __forceinline__ float nan_of<float>() { return __int_as_float(0x7fc00000); }

template <typename T>
__device__ T cell_curvature(const T* __restrict__ cf, const Dims& g, int i, int j, int k, T h) {
    T st[27];
    {
        const int im = i == 0 ? g.nx - 1 : i - 1, ip = i == g.nx - 1 ? 0 : i + 1;
        const int jm = j == 0 ? g.ny - 1 : j - 1, jp = j == g.ny - 1 ? 0 : j + 1;
        const int km = k == 0 ? g.nz - 1 : k - 1, kp = k == g.nz - 1 ? 0 : k + 1;
        const int is[3] = {im, i, ip}, js[3] = {jm, j, jp}, ks[3] = {km, k, kp};
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int a = 0; a < 3; ++a) st[c * 9 + b * 3 + a] = cf[cell(is[a], js[b], ks[c], g)];
    }
    T m[3];
    myc_normal(st, m);
    int a = 0;
    if (fabs(m[1]) > fabs(m[a])) a = 1;
    if (fabs(m[2]) > fabs(m[a])) a = 2;
    const int s = m[a] < T(0) ? -1 : 1;
    const int b = a == 0 ? 1 : 0, e = a == 2 ? 1 : 2;
    const int n[3] = {g.nx, g.ny, g.nz};
    const int p0[3] = {i, j, k};
    T H[3][3];
#pragma unroll
    for (int p = -1; p <= 1; ++p)
#pragma unroll
        for (int q = -1; q <= 1; ++q) {
            T sum = T(0), lo = T(0), hi = T(0);
#pragma unroll
            for (int t = -3; t <= 3; ++t) {
                int o[3];
                o[a] = t;
                o[b] = p;
                o[e] = q;
                const int x = wrapi(p0[0] + o[0], n[0]), y = wrapi(p0[1] + o[1], n[1]), z = wrapi(p0[2] + o[2], n[2]);
                const T v = cf[cell(x, y, z, g)];
                sum += v;
                if (t == -3 * s) lo = v;
                if (t == 3 * s) hi = v;
            }
            if (!(lo > T(0.5) && hi < T(0.5))) return nan_of<T>();
            H[p + 1][q + 1] = sum;
        }
    const T fx = T(0.5) * (H[2][1] - H[0][1]), fy = T(0.5) * (H[1][2] - H[1][0]);
    const T fxx = H[2][1] - T(2) * H[1][1] + H[0][1], fyy = H[1][2] - T(2) * H[1][1] + H[1][0];
    const T fxy = T(0.25) * (H[2][2] - H[2][0] - H[0][2] + H[0][0]);
    const T g2 = T(1) + fx * fx + fy * fy;
    return -(fxx * (T(1) + fy * fy) + fyy * (T(1) + fx * fx) - T(2) * fxy * fx * fy) / (g2 * sqrt_t(g2)) / h;
}

template <typename T>
__global__ void __launch_bounds__(256) k_curvature(const T* __restrict__ cf, Dims g, T h, T* __restrict__ kappa) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < g.N; x += gridDim.x * blockDim.x) {
        const T v = cf[x];
        T out = nan_of<T>();
        if (v > T(0) && v < T(1)) {
            int i, j, k;
            decode(x, g, i, j, k);
            out = cell_curvature(cf, g, i, j, k, h);
        }
        kappa[x] = out;
    }
}

// f[d][x] on the low d-face of cell x: sum over the K fields of
// gamma kappa_f (c(x) - c(x - e_d)) / h, kappa_f the mean of the two cells'
// curvatures where both have one, else the one that does, else 0.
template <typename T>
__global__ void __launch_bounds__(256) k_surface_tension(const T* __restrict__ c, const T* __restrict__ kappa, int K,
                                                         Dims g, T h, T gamma, T* __restrict__ f) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < g.N; x += gridDim.x * blockDim.x) {
        int i, j, k;
        decode(x, g, i, j, k);
        const int xl[3] = {step_cell(x, i, j, k, 0, -1, g), step_cell(x, i, j, k, 1, -1, g),
                           step_cell(x, i, j, k, 2, -1, g)};
        T acc[3] = {T(0), T(0), T(0)};
        for (int q = 0; q < K; ++q) {
            const size_t base = (size_t)q * g.N;
            const T cr = c[base + x], kr = kappa[base + x];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const T cl = c[base + xl[d]], kl = kappa[base + xl[d]];
                const bool fl = isfinite(kl), fr = isfinite(kr);
                const T kf = fl && fr ? T(0.5) * (kl + kr) : (fl ? kl : (fr ? kr : T(0)));
                acc[d] += gamma * kf * (cr - cl) / h;
            }
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) f[(size_t)d * g.N + x] = acc[d];
    }
}

cudaError_t curvature_field(bool fp64, const void* cf, const Dims& g, double h, void* kappa, cudaStream_t st) {
    const int grid = grid_for(g.N, 256);
    if (fp64)
        k_curvature<double><<<grid, 256, 0, st>>>((const double*)cf, g, h, (double*)kappa);
    else
        k_curvature<float><<<grid, 256, 0, st>>>((const float*)cf, g, (float)h, (float*)kappa);
    return cudaGetLastError();
}

cudaError_t surface_tension(bool fp64, const void* c, const void* kappa, int K, const Dims& g, double h,
                            double gamma, void* f, cudaStream_t st) {
    const int grid = grid_for(g.N, 256);
    if (fp64)
        k_surface_tension<double><<<grid, 256, 0, st>>>((const double*)c, (const double*)kappa, K, g, h, gamma,
                                                        (double*)f);
    else
        k_surface_tension<float><<<grid, 256, 0, st>>>((const float*)c, (const float*)kappa, K, g, (float)h,
                                                       (float)gamma, (float*)f);
    return cudaGetLastError();
}

}  // namespace vof
