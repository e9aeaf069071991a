// Step 4 (recolouring) kernels, drop table and nearest-particle statistics
// (Section 2.3 Step 4; Section 3), plus the stateless PLIC primitives.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "plic.cuh"

namespace vof {

// --------------------------------------------------------------------------
// Step 4

// Occupancy bits of the cells of moving drops, one bit plane per field of
// mv_fields (same row layout as the occupancy bits).  A lane takes a word:
// only its occupied cells (the field's occupancy bits, from which its tags
// were made) read their tag.
__global__ void __launch_bounds__(256) k_moving_bits(const int* __restrict__ labels,
                                                     const uint32_t* __restrict__ bits, Dims g, MoveTables mt,
                                                     const int* __restrict__ mv_fields, int n_mv_fields,
                                                     uint32_t* __restrict__ mvbits) {
    const long long per_field = (long long)g.rows * g.W;
    const long long words = (long long)n_mv_fields * per_field;
    for (long long wd = (long long)blockIdx.x * blockDim.x + threadIdx.x; wd < words;
         wd += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(wd / per_field);
        const int rem = (int)(wd - (long long)q * per_field);
        const int f = mv_fields[q];
        uint32_t occ = bits[(size_t)f * per_field + rem], mv = 0u;
        if (occ) {
            const int row = rem / g.W, wi = rem - row * g.W;
            const int* lab = labels + (size_t)f * g.N + (size_t)row * g.nx + wi * 32;
            while (occ) {
                const int b = __ffs(occ) - 1;
                occ &= occ - 1u;
                const int l = lab[b];
                if (is_moving(mt, f, l)) mv |= 1u << b;
            }
        }
        mvbits[wd] = mv;
    }
}

// 64 consecutive occupancy bits of a row starting at cell x0 (periodic).
__device__ __forceinline__ unsigned long long row_window64(const uint32_t* __restrict__ row, int W, int nx, int x0) {
    return (unsigned long long)row_window(row, W, nx, x0) |
           ((unsigned long long)row_window(row, W, nx, x0 + 32) << 32);
}

// For every moving drop m: the fields (other than its own) with an occupied
// cell within Chebyshev distance `reach` of a cell of m (touch[m], a field
// mask), and the other moving drops within that distance (conflict[m], a
// bit per moving drop).  dil_bits holds the occupancy of every active field
// dilated by `reach`, dil_mv the moving-drop bits dilated the same way.  One
// warp takes one 32-cell word of a moving-drop bit plane at a time and
// groups its set bits by drop.  A group touches field n where n's dilated
// occupancy meets it (lane n tests field n).  Conflicts are searched cell by
// cell only in the moving fields whose dilated bits meet the group (its own
// field always, for the field's other moving drops): the lanes share the
// (2 reach + 1)^2 rows of the window and read each row as a 64-bit window
// (reach <= 16) against the group dilated along x.
__global__ void __launch_bounds__(256) k_touch_words(const int* __restrict__ labels,
                                                     const uint32_t* __restrict__ mvbits,
                                                     const uint32_t* __restrict__ dil_bits,
                                                     const uint32_t* __restrict__ dil_mv, Dims g, int n_active,
                                                     int reach, MoveTables mt, const int* __restrict__ mv_fields,
                                                     int n_mv_fields, unsigned* __restrict__ touch,
                                                     unsigned* __restrict__ conflict, int Mw) {
    const int lane = threadIdx.x & 31;
    const long long per_field = (long long)g.rows * g.W;
    const long long words = (long long)n_mv_fields * per_field;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int span = 2 * reach + 1, nrows = span * span;
    for (long long base = warp * 32; base < words; base += nwarps * 32) {
        // 32 words per round, one per lane; then every non-empty one in turn
        const long long my = base + lane;
        const uint32_t mine = my < words ? mvbits[my] : 0u;
        unsigned todo = __ballot_sync(0xffffffffu, mine != 0u);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1u;
            const long long wd = base + src;
            const uint32_t word = __shfl_sync(0xffffffffu, mine, src);
            const int q = (int)(wd / per_field);
            const long long rem = wd - (long long)q * per_field;
            const int row = (int)(rem / g.W);
            const int wi = (int)(rem - (long long)row * g.W);
            const int j = row % g.ny, k = row / g.ny;
            const int f = mv_fields[q];
            const int* lab = labels + (size_t)f * g.N + (size_t)row * g.nx;
            // the moving drop of each set bit
            const bool set = (word >> lane) & 1u;
            const int m_lane = set ? moving_index(mt, f, lab[wi * 32 + lane]) : -1;
            // this word of every dilated plane, one plane per lane
            const uint32_t db = lane < n_active ? dil_bits[(size_t)lane * per_field + rem] : 0u;
            const uint32_t dm = lane < n_mv_fields ? dil_mv[(size_t)lane * per_field + rem] : 0u;
            unsigned rest = __ballot_sync(0xffffffffu, set);
            while (rest) {
                const int lead = __ffs(rest) - 1;
                const int m = __shfl_sync(0xffffffffu, m_lane, lead);
                const unsigned grp = __ballot_sync(0xffffffffu, set && m_lane == m);
                rest &= ~grp;
                if (m < 0) continue;
                const unsigned tmask = __ballot_sync(0xffffffffu, lane != f && (db & grp) != 0u);
                if (lane == 0 && tmask) atomicOr(touch + m, tmask);
                const unsigned cand = __ballot_sync(0xffffffffu, lane == q || (dm & grp) != 0u);
                // frame bit c <-> cell 32 wi - reach + c; cells within reach
                // along x of the group's cells
                unsigned long long dil = 0;
                for (int s2 = 0; s2 <= 2 * reach; ++s2) dil |= (unsigned long long)grp << s2;
                const int x0 = wi * 32 - reach;
                for (int r2 = lane; r2 < nrows; r2 += 32) {
                    const int dz = r2 / span - reach, dy = r2 % span - reach;
                    const int kk = wrapi(k + dz, g.nz), jj = wrapi(j + dy, g.ny);
                    const size_t roff = (size_t)(kk * g.ny + jj) * g.W;
                    unsigned cm = cand;
                    while (cm) {
                        const int q2 = __ffs(cm) - 1;
                        cm &= cm - 1u;
                        unsigned long long wv = row_window64(mvbits + (size_t)q2 * per_field + roff, g.W, g.nx, x0) & dil;
                        const int f2 = mv_fields[q2];
                        while (wv) {
                            const int b = __ffsll((long long)wv) - 1;
                            wv &= wv - 1ull;
                            const int y = cell(wrapi(x0 + b, g.nx), jj, kk, g);
                            const int l2 = labels[(size_t)f2 * g.N + y];
                            if (f2 == f && l2 == mt.mv_label[m]) continue;  // the drop's own cell
                            const int m2 = moving_index(mt, f2, l2);
                            if (m2 < 0 || m2 == m) continue;
                            const unsigned bitm = 1u << (m2 & 31);
                            unsigned* wd2 = conflict + (size_t)m * Mw + (m2 >> 5);
                            if (!(*wd2 & bitm)) atomicOr(wd2, bitm);
                        }
                    }
                }
            }
        }
    }
}

// dil: workspace of (n_active + 2 * n_mv_fields) bit planes.
cudaError_t recolour_touch(const int* labels, const uint32_t* bits, uint32_t* mvbits, uint32_t* dil, const Dims& g,
                           int n_active, int reach, MoveTables mt, const int* mv_fields, int n_mv_fields,
                           unsigned* touch, unsigned* conflict, int Mw, cudaStream_t st, long long* launches) {
    if (reach > 16) return cudaErrorInvalidValue;  // the 64-cell frame holds 32 + 2 reach cells
    if (n_active > 32 || n_mv_fields > 32) return cudaErrorInvalidValue;  // one lane per plane
    const long long pf = (long long)g.rows * g.W;
    const long long words = (long long)n_mv_fields * pf;
    uint32_t* dil_bits = dil;
    uint32_t* dil_mv = dil + (size_t)n_active * pf;
    uint32_t* tmp = dil_mv + (size_t)n_mv_fields * pf;
    k_moving_bits<<<grid_for(words, 256), 256, 0, st>>>(labels, bits, g, mt, mv_fields, n_mv_fields, mvbits);
    cudaError_t e = dilate_planes(bits, dil_bits, tmp, n_active, g, reach, st);
    if (e == cudaSuccess) e = dilate_planes(mvbits, dil_mv, tmp, n_mv_fields, g, reach, st);
    if (e != cudaSuccess) return e;
    k_touch_words<<<grid_for(words, 256), 256, 0, st>>>(labels, mvbits, dil_bits, dil_mv, g, n_active, reach, mt,
                                                         mv_fields, n_mv_fields, touch, conflict, Mw);
    if (launches) *launches += 8;
    return cudaGetLastError();
}

// Step 4's move: every cell of a moving drop hands its c to the drop's
// target field.  A lane takes a word of the moving-drop bits; only its set
// cells are touched.
template <typename T>
__global__ void __launch_bounds__(256) k_move(T* c, const int* __restrict__ labels,
                                              const uint32_t* __restrict__ mvbits, Dims g, MoveTables mt,
                                              const int* __restrict__ mv_fields, int n_mv_fields,
                                              const int* __restrict__ target) {
    const long long per_field = (long long)g.rows * g.W;
    const long long words = (long long)n_mv_fields * per_field;
    for (long long wd = (long long)blockIdx.x * blockDim.x + threadIdx.x; wd < words;
         wd += (long long)gridDim.x * blockDim.x) {
        uint32_t mv = mvbits[wd];
        if (!mv) continue;
        const int q = (int)(wd / per_field);
        const long long rem = wd - (long long)q * per_field;
        const int row = (int)(rem / g.W), wi = (int)(rem - (long long)row * g.W);
        const int f = mv_fields[q];
        const size_t x0 = (size_t)row * g.nx + wi * 32;
        while (mv) {
            const int b = __ffs(mv) - 1;
            mv &= mv - 1u;
            const size_t x = x0 + b;
            const int m = moving_index(mt, f, labels[(size_t)f * g.N + x]);
            const int tg = m >= 0 ? target[m] : -1;
            if (tg < 0) continue;
            const T v = c[(size_t)f * g.N + x];
            c[(size_t)tg * g.N + x] += v;
            c[(size_t)f * g.N + x] = T(0);
        }
    }
}

// One block per listed field sets the bits of its moving tags.
__global__ void k_move_map(MoveTables mt, uint32_t* __restrict__ map, const int* __restrict__ mv_fields) {
    const int f = mv_fields[blockIdx.x];
    const int lo = mt.mv_start[f], n = mt.mv_count[f];
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int l = mt.mv_label[lo + k];
        if (l > 0 && l < kMoveMapTags) atomicOr(map + (size_t)f * kMoveMapWords + (l >> 5), 1u << (l & 31));
    }
}

cudaError_t move_map(MoveTables mt, uint32_t* map, const int* mv_fields, int n_fields, cudaStream_t st) {
    if (n_fields <= 0) return cudaSuccess;
    k_move_map<<<n_fields, 128, 0, st>>>(mt, map, mv_fields);
    return cudaGetLastError();
}

cudaError_t recolour_move(void* c, bool fp64, const int* labels, const uint32_t* mvbits, const Dims& g,
                          MoveTables mt, const int* mv_fields, int n_mv_fields, const int* target, cudaStream_t st) {
    const long long words = (long long)n_mv_fields * g.rows * g.W;
    if (fp64)
        k_move<double><<<grid_for(words, 256), 256, 0, st>>>((double*)c, labels, mvbits, g, mt, mv_fields,
                                                            n_mv_fields, target);
    else
        k_move<float><<<grid_for(words, 256), 256, 0, st>>>((float*)c, labels, mvbits, g, mt, mv_fields,
                                                           n_mv_fields, target);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Drop table: volume and centroid by integrating c over the cells of each
// tag, offsets taken under the minimum image about the tag's root (its
// smallest linear index).

template <typename T>
__global__ void k_drop_sums(const T* __restrict__ cf, const int* __restrict__ label_f,
                            const int* __restrict__ root_of, Dims g, double* __restrict__ S, int n_max) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < g.N; x += gridDim.x * blockDim.x) {
        int l = label_f[x];
        if (l <= 0 || l > n_max) continue;
        int r = root_of[l - 1];
        int i, j, k, ri, rj, rk;
        decode(x, g, i, j, k);
        decode(r, g, ri, rj, rk);
        int d0 = i - ri, d1 = j - rj, d2 = k - rk;
        if (2 * d0 >= g.nx) d0 -= g.nx;
        if (2 * d0 < -g.nx) d0 += g.nx;
        if (2 * d1 >= g.ny) d1 -= g.ny;
        if (2 * d1 < -g.ny) d1 += g.ny;
        if (2 * d2 >= g.nz) d2 -= g.nz;
        if (2 * d2 < -g.nz) d2 += g.nz;
        double v = (double)cf[x];
        double* s = S + 4 * (size_t)(l - 1);
        atomicAdd(s + 0, v);
        if (d0) atomicAdd(s + 1, v * (double)d0);
        if (d1) atomicAdd(s + 2, v * (double)d1);
        if (d2) atomicAdd(s + 3, v * (double)d2);
    }
}

cudaError_t drop_sums(const void* cf, bool fp64, const int* label_f, const int* root_of, const Dims& g,
                      double* S, int n_max, cudaStream_t st) {
    if (fp64)
        k_drop_sums<double><<<grid_for(g.N, 256), 256, 0, st>>>((const double*)cf, label_f, root_of, g, S, n_max);
    else
        k_drop_sums<float><<<grid_for(g.N, 256), 256, 0, st>>>((const float*)cf, label_f, root_of, g, S, n_max);
    return cudaGetLastError();
}

__global__ void k_drop_finalize(const double* __restrict__ S, const int* __restrict__ root_of, Dims g,
                                double h, int n, double* __restrict__ vol, double* __restrict__ cen) {
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
        const double* s = S + 4 * (size_t)l;
        int r = root_of[l];
        int rc[3];
        decode(r, g, rc[0], rc[1], rc[2]);
        int L[3] = {g.nx, g.ny, g.nz};
        vol[l] = s[0] * h * h * h;
        for (int a = 0; a < 3; ++a) {
            double p = ((double)rc[a] + 0.5 + s[1 + a] / s[0]) * h;
            double Lh = (double)L[a] * h;
            p = fmod(p, Lh);
            if (p < 0.0) p += Lh;
            if (p >= Lh) p = 0.0;
            cen[3 * (size_t)l + a] = p;
        }
    }
}

cudaError_t drop_finalize(const double* S, const int* root_of, const Dims& g, double h, int n,
                          double* vol, double* cen, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_drop_finalize<<<grid_for(n, 128), 128, 0, st>>>(S, root_of, g, h, n, vol, cen);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Drop shape (Appendix A): inertia tensor of each drop about its centre of
// mass, I = integral over the drop of [(r.r) delta - r r], of the drop's
// colour density (each cell of the tag holding c uniformly: the cell-centre
// term plus the cube's own moment c h^5 / 6 on the diagonal), r under the
// minimum image; and the aspect ratio chi = sqrt(I_max / I_min).

template <typename T>
__global__ void k_drop_inertia(const T* __restrict__ cf, const int* __restrict__ label_f, Dims g, double h,
                               const double* __restrict__ cen, int n_max, double* __restrict__ I) {
    const double L[3] = {g.nx * h, g.ny * h, g.nz * h};
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < g.N; x += gridDim.x * blockDim.x) {
        const int l = label_f[x];
        if (l <= 0 || l > n_max) continue;
        int ijk[3];
        decode(x, g, ijk[0], ijk[1], ijk[2]);
        double r[3];
        for (int a = 0; a < 3; ++a) {
            double t = ((double)ijk[a] + 0.5) * h - cen[3 * (size_t)(l - 1) + a];
            if (t > 0.5 * L[a]) t -= L[a];
            if (t < -0.5 * L[a]) t += L[a];
            r[a] = t;
        }
        const double w = (double)cf[x] * h * h * h;
        const double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2], own = h * h / 6.0;
        double* s = I + 6 * (size_t)(l - 1);
        atomicAdd(s + 0, w * (rr - r[0] * r[0] + own));
        atomicAdd(s + 1, w * (rr - r[1] * r[1] + own));
        atomicAdd(s + 2, w * (rr - r[2] * r[2] + own));
        atomicAdd(s + 3, -w * r[0] * r[1]);
        atomicAdd(s + 4, -w * r[0] * r[2]);
        atomicAdd(s + 5, -w * r[1] * r[2]);
    }
}

cudaError_t drop_inertia(const void* cf, bool fp64, const int* label_f, const Dims& g, double h, const double* cen,
                         int n, double* I, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(I, 0, (size_t)n * 6 * 8, st);
    if (e != cudaSuccess) return e;
    if (fp64)
        k_drop_inertia<double><<<grid_for(g.N, 256), 256, 0, st>>>((const double*)cf, label_f, g, h, cen, n, I);
    else
        k_drop_inertia<float><<<grid_for(g.N, 256), 256, 0, st>>>((const float*)cf, label_f, g, h, cen, n, I);
    return cudaGetLastError();
}

// Extreme eigenvalues of the symmetric matrix [[a, d, e], [d, b, f], [e, f, c]]:
// with q = tr/3 and B = (A - q 1)/p, p^2 = tr((A - q 1)^2)/6, the eigenvalues
// are q + 2 p cos(phi + 2 pi m / 3), m = 0, 1, 2, where cos(3 phi) = det(B)/2
// (the characteristic polynomial of B is the triple-angle identity).
__device__ __forceinline__ void sym3_extremes(double a, double b, double c, double d, double e, double f,
                                              double& lmax, double& lmin) {
    const double off = d * d + e * e + f * f;
    const double q = (a + b + c) / 3.0;
    const double p2 = ((a - q) * (a - q) + (b - q) * (b - q) + (c - q) * (c - q) + 2.0 * off) / 6.0;
    if (!(p2 > 0.0)) {
        lmax = lmin = q;
        return;
    }
    const double p = sqrt(p2);
    const double B00 = (a - q) / p, B11 = (b - q) / p, B22 = (c - q) / p;
    const double B01 = d / p, B02 = e / p, B12 = f / p;
    const double det = B00 * (B11 * B22 - B12 * B12) - B01 * (B01 * B22 - B12 * B02) + B02 * (B01 * B12 - B11 * B02);
    const double r = fmin(1.0, fmax(-1.0, 0.5 * det));
    const double phi = acos(r) / 3.0;
    lmax = q + 2.0 * p * cos(phi);
    lmin = q + 2.0 * p * cos(phi + 2.0 * M_PI / 3.0);
}

// chi of every drop; acc[0] += sum of chi, acc[1] += drops, acc[2] = max chi.
__global__ void __launch_bounds__(128) k_drop_chi(const double* __restrict__ I, int n, double* __restrict__ chi,
                                                  double* __restrict__ acc) {
    double sum = 0.0, cnt = 0.0, mx = 0.0;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
        const double* s = I + 6 * (size_t)l;
        double lmax, lmin;
        sym3_extremes(s[0], s[1], s[2], s[3], s[4], s[5], lmax, lmin);
        const double x = lmin > 0.0 ? sqrt(lmax / lmin) : INFINITY;
        if (chi) chi[l] = x;
        if (isfinite(x)) {
            sum += x;
            cnt += 1.0;
            mx = fmax(mx, x);
        }
    }
    if (!acc) return;
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_down_sync(0xffffffffu, sum, o);
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0 && cnt > 0.0) {
        atomicAdd(acc + 0, sum);
        atomicAdd(acc + 1, cnt);
        // positive doubles order like their bit patterns
        atomicMax(reinterpret_cast<unsigned long long*>(acc + 2), (unsigned long long)__double_as_longlong(mx));
    }
}

cudaError_t drop_chi(const double* I, int n, double* chi, double* acc, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_drop_chi<<<grid_for(n, 128, 1024), 128, 0, st>>>(I, n, chi, acc);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Nearest-particle statistics (Section 3, eq. P_nstij with h_ij = 1/N_i for
// the N_i equidistant nearest neighbours; histograms of eqs. vec_cond and
// Ptheta_r; moments M and R of Section 4).

__device__ __forceinline__ double min_image(double t, double L) {
    if (t > 0.5 * L) t -= L;
    if (t < -0.5 * L) t += L;
    return t;
}

__global__ void __launch_bounds__(128) k_pair_stats(const double* __restrict__ cen, long long n, double bx,
                                                    double by, double bz, int vaxis, int n_rbins, double dr,
                                                    int n_tbins, double dtheta, double tie_tol,
                                                    double* __restrict__ hist_r, double* __restrict__ hist_rt,
                                                    double* __restrict__ moments) {
    double loc[13];
    for (int q = 0; q < 13; ++q) loc[q] = 0.0;
    double box[3] = {bx, by, bz};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (n < 2) break;
        double ci[3] = {cen[3 * i], cen[3 * i + 1], cen[3 * i + 2]};
        double dmin = INFINITY;
        for (long long j = 0; j < n; ++j) {
            if (j == i) continue;
            double r0 = min_image(cen[3 * j] - ci[0], box[0]);
            double r1 = min_image(cen[3 * j + 1] - ci[1], box[1]);
            double r2 = min_image(cen[3 * j + 2] - ci[2], box[2]);
            double dd = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
            if (dd < dmin) dmin = dd;
        }
        int ni = 0;
        for (long long j = 0; j < n; ++j) {
            if (j == i) continue;
            double r0 = min_image(cen[3 * j] - ci[0], box[0]);
            double r1 = min_image(cen[3 * j + 1] - ci[1], box[1]);
            double r2 = min_image(cen[3 * j + 2] - ci[2], box[2]);
            double dd = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
            if (dd - dmin <= tie_tol) ++ni;
        }
        double wgt = 1.0 / (double)ni;
        for (long long j = 0; j < n; ++j) {
            if (j == i) continue;
            double r[3];
            r[0] = min_image(cen[3 * j] - ci[0], box[0]);
            r[1] = min_image(cen[3 * j + 1] - ci[1], box[1]);
            r[2] = min_image(cen[3 * j + 2] - ci[2], box[2]);
            double dd = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            if (!(dd - dmin <= tie_tol)) continue;
            int kr = (int)floor(dd / dr);
            if (kr > n_rbins || kr < 0) kr = n_rbins;
            double ct = dd > 0.0 ? r[vaxis] / dd : 1.0;
            if (ct > 1.0) ct = 1.0;
            if (ct < -1.0) ct = -1.0;
            int kt = (int)floor(acos(ct) / dtheta);
            if (kt >= n_tbins) kt = n_tbins - 1;
            if (kt < 0) kt = 0;
            atomicAdd(hist_r + kr, wgt);
            atomicAdd(hist_rt + (size_t)kr * n_tbins + kt, wgt);
            for (int a = 0; a < 3; ++a) {
                loc[a] += wgt * r[a];
                for (int b = 0; b < 3; ++b) loc[3 + 3 * a + b] += wgt * r[a] * r[b];
            }
        }
        loc[12] += 1.0;
    }
    // block reduction of the 13 sums
    __shared__ double red[13][4];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = 0; q < 13; ++q) {
        double v = loc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[q][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 13) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
        if (v != 0.0) atomicAdd(moments + threadIdx.x, v);
    }
}

cudaError_t pair_stats(const double* cen, long long n, double bx, double by, double bz, int vaxis,
                       int n_rbins, double dr, int n_tbins, double dtheta, double tie_tol, double* hist_r,
                       double* hist_rt, double* moments, cudaStream_t st) {
    if (n < 2) return cudaSuccess;
    k_pair_stats<<<grid_for(n, 128), 128, 0, st>>>(cen, n, bx, by, bz, vaxis, n_rbins, dr, n_tbins, dtheta,
                                                    tie_tol, hist_r, hist_rt, moments);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// PLIC primitives, normals, velocity scan

template <typename T>
__global__ void k_plic_volume(const T* __restrict__ m, const T* __restrict__ alpha, T* __restrict__ v,
                              long long n) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        v[t] = plic_volume<T>(m[3 * t], m[3 * t + 1], m[3 * t + 2], alpha[t]);
}

template <typename T>
__global__ void k_plic_alpha(const T* __restrict__ m, const T* __restrict__ c, T* __restrict__ alpha,
                             long long n, T band) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        alpha[t] = plic_alpha_banded(m[3 * t], m[3 * t + 1], m[3 * t + 2], c[t], band);
}

cudaError_t plic_volume_batch(bool fp64, const void* m, const void* alpha, void* v, long long n,
                              cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (fp64)
        k_plic_volume<double><<<grid_for(n, 128), 128, 0, st>>>((const double*)m, (const double*)alpha,
                                                               (double*)v, n);
    else
        k_plic_volume<float><<<grid_for(n, 128), 128, 0, st>>>((const float*)m, (const float*)alpha,
                                                              (float*)v, n);
    return cudaGetLastError();
}

cudaError_t plic_alpha_batch(bool fp64, const void* m, const void* c, void* alpha, long long n,
                             double band, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (fp64)
        k_plic_alpha<double><<<grid_for(n, 128), 128, 0, st>>>((const double*)m, (const double*)c,
                                                              (double*)alpha, n, band);
    else
        k_plic_alpha<float><<<grid_for(n, 128), 128, 0, st>>>((const float*)m, (const float*)c,
                                                             (float*)alpha, n, (float)band);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_normals(const T* __restrict__ cf, Dims g, T* __restrict__ m) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < g.N; x += gridDim.x * blockDim.x) {
        T r[3] = {T(0), T(0), T(0)};
        if (vclass(cf[x]) == 1) {
            int i, j, k;
            decode(x, g, i, j, k);
            T st[27];
            int is[3] = {wrapi(i - 1, g.nx), i, wrapi(i + 1, g.nx)};
            int js[3] = {wrapi(j - 1, g.ny), j, wrapi(j + 1, g.ny)};
            int ks[3] = {wrapi(k - 1, g.nz), k, wrapi(k + 1, g.nz)};
            for (int c = 0; c < 3; ++c)
                for (int b = 0; b < 3; ++b)
                    for (int a = 0; a < 3; ++a) st[c * 9 + b * 3 + a] = cf[cell(is[a], js[b], ks[c], g)];
            myc_normal(st, r);
        }
        m[3 * (size_t)x] = r[0];
        m[3 * (size_t)x + 1] = r[1];
        m[3 * (size_t)x + 2] = r[2];
    }
}

cudaError_t normals_field(bool fp64, const void* cf, const Dims& g, void* m, cudaStream_t st) {
    if (fp64)
        k_normals<double><<<grid_for(g.N, 128), 128, 0, st>>>((const double*)cf, g, (double*)m);
    else
        k_normals<float><<<grid_for(g.N, 128), 128, 0, st>>>((const float*)cf, g, (float*)m);
    return cudaGetLastError();
}

// out2[0] = max |u|, out2[1] = 1 if any non-finite value (both as double).
template <typename T>
__global__ void k_vscan(const T* __restrict__ u, long long n, unsigned long long* __restrict__ out) {
    double mx = 0.0;
    unsigned bad = 0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        double v = (double)u[t];
        if (!isfinite(v)) bad = 1;
        else mx = fmax(mx, fabs(v));
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
        bad |= __shfl_down_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, (unsigned long long)__double_as_longlong(mx));  // non-negative doubles order as ints
        if (bad) atomicOr(out + 1, 1ull);
    }
}

cudaError_t velocity_scan(bool fp64, const void* u, long long n, double* out2, cudaStream_t st) {
    cudaMemsetAsync(out2, 0, 2 * sizeof(double), st);
    if (fp64)
        k_vscan<double><<<grid_for(n, 256), 256, 0, st>>>((const double*)u, n, (unsigned long long*)out2);
    else
        k_vscan<float><<<grid_for(n, 256), 256, 0, st>>>((const float*)u, n, (unsigned long long*)out2);
    return cudaGetLastError();
}

namespace {
thread_local const char* g_last_cuda_error = "no error";
}

cudaError_t note_cuda_error(cudaError_t e) {
    if (e != cudaSuccess) g_last_cuda_error = cudaGetErrorName(e);
    return e;
}

const char* last_cuda_error_name() { return g_last_cuda_error; }

}  // namespace vof
