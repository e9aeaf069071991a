/*
 * FP64 CPU oracle of the multi-field VoF step (arXiv 2407.07463).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline leg of the benchmark; never by the product path.  Plain, slow and
 * written to be checked by eye against the method:
 *
 *   - PLIC reconstruction (Section 2.2): the volume under a plane is computed
 *     by clipping the cube's faces and applying the divergence theorem; the
 *     plane constant by bisection.
 *   - Mixed-Youngs-Centred normals from the 3x3x3 stencil (Aulisa et al.
 *     2007), under the selection rule stated at oracle_myc().
 *   - Directionally split geometric advection with the Weymouth-Yue
 *     divergence term, sweep order rotated per step, clip after the third
 *     sweep.
 *   - Section 2.3 (no-coalescence) Steps 1-4: near-contact test, tagging
 *     (breadth-first flood fill), near-contact pairs with distinct tags,
 *     recolouring into free fields.
 *   - Section 3: drop centroids from tags and nearest-particle statistics.
 *   - The learned normal (no counterpart in the paper): canonical frame of a
 *     stencil, the 27-64-64-3 network in FP64 (optionally with the BF16
 *     rounding of weights and layer inputs the tensor cores see), FP64
 *     backpropagation, the 27-cell residual that judges a normal, the MYC
 *     fallback, and the split step with that normal.
 *
 * Parity pins: every function is pinned by tests against closed forms,
 * brute force and the paper's worked example, except the MYC selection rule
 * itself (pinned only through the cases where all candidates coincide and
 * the exactness of centred columns on unsaturated planes) -- "parity
 * unpinned" for that rule -- and the fallback rule of the learned normal,
 * which the paper does not have (its parts are pinned: the network by a
 * weight set that reproduces Youngs, the residual by hand-computed axis
 * planes and exact planes, backpropagation by finite differences).
 *
 * Build with -ffp-contract=off so x86-64 and aarch64 round identically.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the OpenMP build (the serial build has one).  The advection
 * step spreads its z-planes over them; every face flux and every cell update
 * is computed exactly as in the serial build, so results are identical. */
int oracle_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* PLIC volume: clipped unit square areas + divergence theorem              */

typedef struct {
    double y, z;
} pt2;

/* Keep the part of a convex polygon with a*y + b*z - beta <= 0. */
static int clip_polygon(const pt2 *in, int n, double a, double b, double beta,
                        pt2 *out)
{
    int m = 0;
    for (int i = 0; i < n; ++i) {
        pt2 p = in[i];
        pt2 q = in[(i + 1) % n];
        double fp = a * p.y + b * p.z - beta;
        double fq = a * q.y + b * q.z - beta;
        if (fp <= 0.0)
            out[m++] = p;
        if ((fp < 0.0 && fq > 0.0) || (fp > 0.0 && fq < 0.0)) {
            double t = fp / (fp - fq);
            pt2 r;
            r.y = p.y + t * (q.y - p.y);
            r.z = p.z + t * (q.z - p.z);
            out[m++] = r;
        }
    }
    return m;
}

/* Area of {(y,z) in [0,1]^2 : a*y + b*z < beta}. */
static double square_area_below(double a, double b, double beta)
{
    if (a == 0.0 && b == 0.0)
        return beta > 0.0 ? 1.0 : 0.0;
    pt2 sq[4] = {{0.0, 0.0}, {1.0, 0.0}, {1.0, 1.0}, {0.0, 1.0}};
    pt2 poly[8];
    int m = clip_polygon(sq, 4, a, b, beta, poly);
    double twice = 0.0;
    for (int i = 0; i < m; ++i) {
        pt2 p = poly[i];
        pt2 q = poly[(i + 1) % m];
        twice += p.y * q.z - q.y * p.z;
    }
    return 0.5 * twice;
}

/*
 * Volume of Omega = {x in [0,1]^3 : m.x < alpha}.  Divergence theorem with
 * the field x:  3 V = sum_faces int x.n dS.  Faces x_i = 0 contribute 0,
 * faces x_i = 1 contribute their clipped area A_i1, the cap (plane m.x =
 * alpha, outward normal m/|m|) contributes alpha/|m| * A_cap, and the closed
 * surface gives A_cap m/|m| = sum_i (A_i0 - A_i1) e_i.
 */
double oracle_plic_volume(const double m[3], double alpha)
{
    double n2 = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
    if (n2 == 0.0)
        return alpha > 0.0 ? 1.0 : 0.0;
    double a1 = 0.0, cap = 0.0;
    for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3, k = (i + 2) % 3;
        double A0 = square_area_below(m[j], m[k], alpha);
        double A1 = square_area_below(m[j], m[k], alpha - m[i]);
        a1 += A1;
        cap += m[i] * (A0 - A1);
    }
    return (a1 + alpha * cap / n2) / 3.0;
}

/* Bisection on [min_x m.x, max_x m.x] until the bracket stops shrinking. */
double oracle_plic_alpha(const double m[3], double c)
{
    double lo = 0.0, hi = 0.0;
    for (int i = 0; i < 3; ++i) {
        if (m[i] < 0.0)
            lo += m[i];
        else
            hi += m[i];
    }
    if (c <= 0.0)
        return lo;
    if (c >= 1.0)
        return hi;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi)
            break;
        if (oracle_plic_volume(m, mid) < c)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------ */
/* Normals                                                                   */

#define ST(st, i, j, k) ((st)[((k) + 1) * 9 + ((j) + 1) * 3 + ((i) + 1)])

static const double YW[3] = {1.0, 2.0, 1.0};

/* Youngs: average of the eight vertex gradients, m = -grad c; the factor
 * common to the three components is dropped (L1 normalisation follows). */
static void youngs_raw(const double st[27], double y[3])
{
    double yx = 0.0, yy = 0.0, yz = 0.0;
    for (int b = -1; b <= 1; ++b)
        for (int a = -1; a <= 1; ++a) {
            double w = YW[a + 1] * YW[b + 1];
            yx += w * (ST(st, -1, a, b) - ST(st, 1, a, b));
            yy += w * (ST(st, a, -1, b) - ST(st, a, 1, b));
            yz += w * (ST(st, a, b, -1) - ST(st, a, b, 1));
        }
    y[0] = yx;
    y[1] = yy;
    y[2] = yz;
}

static double l1(const double v[3])
{
    return fabs(v[0]) + fabs(v[1]) + fabs(v[2]);
}

void oracle_youngs(const double st[27], double m[3])
{
    double y[3];
    youngs_raw(st, y);
    double n = l1(y);
    if (n < 1e-30) {
        m[0] = m[1] = m[2] = 0.0;
        return;
    }
    m[0] = y[0] / n;
    m[1] = y[1] / n;
    m[2] = y[2] / n;
}

/* Stencil value with offset t along `axis`, p and q along the other two
 * axes taken in increasing axis order. */
static double st_axis(const double st[27], int axis, int t, int p, int q)
{
    int o[3];
    int b = (axis + 1) % 3, c = (axis + 2) % 3;
    if (b > c) {
        int tmp = b;
        b = c;
        c = tmp;
    }
    o[axis] = t;
    o[b] = p;
    o[c] = q;
    return ST(st, o[0], o[1], o[2]);
}

/* Centred columns along `axis`: column heights H(p,q) = sum_t c, slopes of
 * the height by central differences, own component +-1 with the sign of the
 * Youngs component along the axis (+1 when it is zero).  Not normalised. */
static void centred_column_raw(const double st[27], int axis, const double y[3],
                               double m[3])
{
    int b = (axis + 1) % 3, c = (axis + 2) % 3;
    if (b > c) {
        int tmp = b;
        b = c;
        c = tmp;
    }
    double H[3][3];
    for (int p = -1; p <= 1; ++p)
        for (int q = -1; q <= 1; ++q)
            H[p + 1][q + 1] = st_axis(st, axis, -1, p, q) + st_axis(st, axis, 0, p, q) +
                              st_axis(st, axis, 1, p, q);
    m[b] = (H[0][1] - H[2][1]) * 0.5;
    m[c] = (H[1][0] - H[1][2]) * 0.5;
    m[axis] = y[axis] < 0.0 ? -1.0 : 1.0;
}

void oracle_centred_column(const double st[27], int axis, double m[3])
{
    double y[3], r[3];
    youngs_raw(st, y);
    centred_column_raw(st, axis, y, r);
    double n = l1(r);
    m[0] = r[0] / n;
    m[1] = r[1] / n;
    m[2] = r[2] / n;
}

/*
 * Mixed-Youngs-Centred selection (reading of Aulisa et al. 2007):
 *   1. among the three centred-column candidates take the one whose own-axis
 *      component |m_a| / |m|_1 is largest (ties to the lowest axis);
 *   2. use the Youngs normal instead when its largest |component| / |m|_1 is
 *      strictly smaller than that value and its L1 norm is at least 1e-30.
 * Columns that saturate make a centred-column normal look more grid-aligned
 * than it is; Youngs then reports a more oblique normal and is taken.  For a
 * plane whose columns do not saturate the centred column is exact.
 */
int oracle_myc_choice(const double st[27])
{
    double y[3];
    youngs_raw(st, y);
    int best = 0;
    double best_own = -1.0;
    for (int a = 0; a < 3; ++a) {
        double r[3];
        centred_column_raw(st, a, y, r);
        double own = fabs(r[a]) / l1(r);
        if (own > best_own) {
            best_own = own;
            best = a;
        }
    }
    double ny = l1(y);
    if (ny >= 1e-30) {
        double ymax = fabs(y[0]);
        if (fabs(y[1]) > ymax)
            ymax = fabs(y[1]);
        if (fabs(y[2]) > ymax)
            ymax = fabs(y[2]);
        if (ymax / ny < best_own)
            return 3;
    }
    return best;
}

void oracle_myc(const double st[27], double m[3])
{
    int ch = oracle_myc_choice(st);
    if (ch == 3)
        oracle_youngs(st, m);
    else
        oracle_centred_column(st, ch, m);
}

/* ------------------------------------------------------------------------ */
/* Split advection                                                           */

/*
 * Flux through a face of the donor cell whose reconstruction is (m, alpha).
 * s > 0: the swept region is x_d in [1-s, 1] of the donor; s < 0: x_d in
 * [0, |s|].  Mapping the sub-cell onto the unit cube scales m_d by |s| and
 * shifts alpha by m_d * x0; the flux is s times the sub-cell fraction.
 */
double oracle_face_flux(const double m[3], double alpha, int d, double s)
{
    if (s == 0.0)
        return 0.0;
    double as = fabs(s);
    double x0 = s > 0.0 ? 1.0 - s : 0.0;
    double mm[3] = {m[0], m[1], m[2]};
    mm[d] = m[d] * as;
    double a2 = alpha - m[d] * x0;
    return s * oracle_plic_volume(mm, a2);
}

static inline int64_t idx3(int i, int j, int k, int nx, int ny)
{
    return ((int64_t)k * ny + j) * nx + i;
}

static inline int wrap(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

static void gather_stencil(const double *c, int nx, int ny, int nz, int i, int j,
                           int k, double st[27])
{
    for (int b = -1; b <= 1; ++b)
        for (int a = -1; a <= 1; ++a)
            for (int e = -1; e <= 1; ++e)
                ST(st, e, a, b) = c[idx3(wrap(i + e, nx), wrap(j + a, ny), wrap(k + b, nz), nx, ny)];
}

/* Learned-normal settings of a step (NULL: MYC everywhere). */
typedef struct {
    const double *params;
    double tol, amb_eps;
    int amb_choice;
    int64_t counts[3]; /* faces on the network, on MYC, decided as ambiguous */
    uint8_t *amb_map;  /* current field's map of cells next to ambiguous faces, or NULL */
} learned_cfg;

static double cell_face_flux(const double *c, int nx, int ny, int nz, int i, int j, int k, int d,
                             double s, learned_cfg *L)
{
    if (s == 0.0)
        return 0.0;
    int di = d == 0, dj = d == 1, dk = d == 2;
    int si = i, sj = j, sk = k; /* donor */
    if (s > 0.0) {
        si = wrap(i - di, nx);
        sj = wrap(j - dj, ny);
        sk = wrap(k - dk, nz);
    }
    double cd = c[idx3(si, sj, sk, nx, ny)];
    if (cd <= 0.0)
        return 0.0;
    if (cd >= 1.0)
        return s;
    double st[27], m[3];
    gather_stencil(c, nx, ny, nz, si, sj, sk, st);
    if (!L) {
        oracle_myc(st, m);
        return oracle_face_flux(m, oracle_plic_alpha(m, cd), d, s);
    }
    int amb = 0;
    int which = oracle_learned_normal(L->params, st, L->tol, L->amb_eps, L->amb_choice, m, &amb);
    L->counts[which] += 1;
    L->counts[2] += amb;
    double F = oracle_face_flux(m, oracle_plic_alpha(m, cd), d, s);
    if (amb && L->amb_map) {
        /* an ambiguous decision matters only where the other branch gives
         * another flux: mark both cells of the face then */
        double m2[3];
        oracle_learned_normal(L->params, st, L->tol, L->amb_eps, 1 - L->amb_choice, m2, NULL);
        double F2 = oracle_face_flux(m2, oracle_plic_alpha(m2, cd), d, s);
        if (fabs(F2 - F) > 1e-7) {
            /* the face's two cells: (i, j, k) and its low neighbour along d */
            uint8_t *a = L->amb_map + idx3(i, j, k, nx, ny);
            uint8_t *b = L->amb_map + idx3(wrap(i - di, nx), wrap(j - dj, ny), wrap(k - dk, nz), nx, ny);
#ifdef _OPENMP
#pragma omp atomic write
#endif
            *a = 1;
#ifdef _OPENMP
#pragma omp atomic write
#endif
            *b = 1;
        }
    }
    return F;
}

double oracle_cell_face_flux(const double *c, int nx, int ny, int nz, int i, int j,
                             int k, int d, double s)
{
    return cell_face_flux(c, nx, ny, nz, i, j, k, d, s, NULL);
}

static int advect_step(double *c, const double *u, int nx, int ny, int nz, int K, double dt,
                       double h, int64_t step_index, double *clipped, learned_cfg *L,
                       uint8_t *L_map)
{
    int64_t N = (int64_t)nx * ny * nz;
    double sfac = dt / h;
    double *cc = (double *)malloc(sizeof(double) * N * (K > 0 ? K : 1));
    double *F = (double *)malloc(sizeof(double) * N);
    double *nw = (double *)malloc(sizeof(double) * N);
    if (!cc || !F || !nw) {
        free(cc);
        free(F);
        free(nw);
        return -1;
    }
    for (int64_t x = 0; x < N * K; ++x)
        cc[x] = c[x] > 0.5 ? 1.0 : 0.0;
    int rot = (int)(step_index % 3);
    int order[3] = {rot % 3, (rot + 1) % 3, (rot + 2) % 3};
    for (int sw = 0; sw < 3; ++sw) {
        int d = order[sw];
        const double *ud = u + (int64_t)d * N;
        for (int f = 0; f < K; ++f) {
            double *cf = c + (int64_t)f * N;
            const double *ccf = cc + (int64_t)f * N;
            if (L)
                L->amb_map = L_map ? L_map + (int64_t)f * N : NULL;
            /* the OpenMP build takes z-planes in parallel; each plane keeps
             * its own face counts, added up afterwards (integer sums) */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
            for (int k = 0; k < nz; ++k) {
                learned_cfg Lk, *Lp = NULL;
                if (L) {
                    Lk = *L;
                    Lk.counts[0] = Lk.counts[1] = Lk.counts[2] = 0;
                    Lp = &Lk;
                }
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i) {
                        int64_t x = idx3(i, j, k, nx, ny);
                        F[x] = cell_face_flux(cf, nx, ny, nz, i, j, k, d, ud[x] * sfac, Lp);
                    }
                if (L)
                    for (int q = 0; q < 3; ++q) {
#ifdef _OPENMP
#pragma omp atomic
#endif
                        L->counts[q] += Lk.counts[q];
                    }
            }
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i) {
                        int64_t x = idx3(i, j, k, nx, ny);
                        int64_t xh = idx3(d == 0 ? wrap(i + 1, nx) : i, d == 1 ? wrap(j + 1, ny) : j,
                                          d == 2 ? wrap(k + 1, nz) : k, nx, ny);
                        double s_lo = ud[x] * sfac;
                        double s_hi = ud[xh] * sfac;
                        nw[x] = cf[x] - (F[xh] - F[x]) + ccf[x] * (s_hi - s_lo);
                    }
            memcpy(cf, nw, sizeof(double) * N);
        }
    }
    for (int f = 0; f < K; ++f) {
        double removed = 0.0;
        double *cf = c + (int64_t)f * N;
        for (int64_t x = 0; x < N; ++x) {
            double v = cf[x];
            double cl = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
            removed += v - cl;
            cf[x] = cl;
        }
        if (clipped)
            clipped[f] = removed;
    }
    free(cc);
    free(F);
    free(nw);
    return 0;
}

int oracle_advect_step(double *c, const double *u, int nx, int ny, int nz, int K,
                       double dt, double h, int64_t step_index, double *clipped)
{
    return advect_step(c, u, nx, ny, nz, K, dt, h, step_index, clipped, NULL, NULL);
}

int oracle_advect_step_learned(double *c, const double *u, int nx, int ny, int nz, int K,
                               double dt, double h, int64_t step_index, const double *params,
                               double tol, double amb_eps, int amb_choice, double *clipped,
                               int64_t counts[3], uint8_t *amb_map)
{
    learned_cfg L = {params, tol, amb_eps, amb_choice, {0, 0, 0}, NULL};
    int r = advect_step(c, u, nx, ny, nz, K, dt, h, step_index, clipped, &L, amb_map);
    if (counts)
        for (int q = 0; q < 3; ++q)
            counts[q] = L.counts[q];
    return r;
}

void oracle_normals(const double *c, int nx, int ny, int nz, double *m_out)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t x = idx3(i, j, k, nx, ny);
                double *m = m_out + 3 * x;
                m[0] = m[1] = m[2] = 0.0;
                if (c[x] > 0.0 && c[x] < 1.0) {
                    double st[27];
                    gather_stencil(c, nx, ny, nz, i, j, k, st);
                    oracle_myc(st, m);
                }
            }
}

/* ------------------------------------------------------------------------ */
/* Curvature by height functions and the surface-tension source             */

/*
 * Curvature of one interfacial cell (Section 2.3: each tracer's curvature
 * kappa_i enters the surface-tension force; computed per tracer as for a
 * single one).  Height functions: along the axis a of the largest |component|
 * of the cell's MYC normal (ties to the lower axis), the 3x3 columns of 7
 * cells (offsets -3..3 along a) centred on the cell and its 8 neighbours
 * across a hold heights H = sum of c (in cells).  Each column must contain
 * the interface: its end on the side the normal points away from (the c = 1
 * phase) holds more than 1/2, the other end less than 1/2; otherwise the
 * cell has no curvature (returns NaN).  With the surface z = f(x, y) of the
 * phase below it, the outward normal (-f_x, -f_y, 1)/sqrt(1 + |grad f|^2)
 * has divergence
 *   kappa = -[f_xx (1 + f_y^2) + f_yy (1 + f_x^2) - 2 f_xy f_x f_y]
 *           / (1 + f_x^2 + f_y^2)^(3/2),
 * positive for a drop (2/R for a sphere); f's derivatives are the centred
 * differences of H over the 3x3 columns (cell units), divided by h for
 * kappa in inverse length.  Reflecting a (the phase above instead) leaves
 * H and this expression unchanged.
 */
static double curvature_along(const double *c, int nx, int ny, int nz, int i, int j, int k, double h, int a,
                              int s)
{
    int b = a == 0 ? 1 : 0, e = a == 2 ? 1 : 2; /* the two other axes, in order */
    double H[3][3];
    for (int p = -1; p <= 1; ++p)
        for (int q = -1; q <= 1; ++q) {
            double sum = 0.0, lo = 0.0, hi = 0.0;
            for (int t = -3; t <= 3; ++t) {
                int o[3];
                o[a] = t;
                o[b] = p;
                o[e] = q;
                double v = c[idx3(wrap(i + o[0], nx), wrap(j + o[1], ny), wrap(k + o[2], nz), nx, ny)];
                sum += v;
                if (t == -3 * s)
                    lo = v; /* the c = 1 end */
                if (t == 3 * s)
                    hi = v; /* the c = 0 end */
            }
            if (!(lo > 0.5 && hi < 0.5))
                return NAN;
            H[p + 1][q + 1] = sum;
        }
    double fx = 0.5 * (H[2][1] - H[0][1]), fy = 0.5 * (H[1][2] - H[1][0]);
    double fxx = H[2][1] - 2.0 * H[1][1] + H[0][1], fyy = H[1][2] - 2.0 * H[1][1] + H[1][0];
    double fxy = 0.25 * (H[2][2] - H[2][0] - H[0][2] + H[0][0]);
    double g2 = 1.0 + fx * fx + fy * fy;
    return -(fxx * (1.0 + fy * fy) + fyy * (1.0 + fx * fx) - 2.0 * fxy * fx * fy) / (g2 * sqrt(g2)) / h;
}

static double cell_curvature(const double *c, int nx, int ny, int nz, int i, int j, int k, double h)
{
    double st[27], m[3];
    gather_stencil(c, nx, ny, nz, i, j, k, st);
    oracle_myc(st, m);
    int a = 0;
    for (int q = 1; q < 3; ++q)
        if (fabs(m[q]) > fabs(m[a]))
            a = q;
    /* the normal points to +s along a */
    return curvature_along(c, nx, ny, nz, i, j, k, h, a, m[a] < 0.0 ? -1 : 1);
}

void oracle_curvature_along(const double *c, int nx, int ny, int nz, double h, int axis, int sign,
                            double *kappa)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t x = idx3(i, j, k, nx, ny);
                kappa[x] = (c[x] > 0.0 && c[x] < 1.0)
                               ? curvature_along(c, nx, ny, nz, i, j, k, h, axis, sign < 0 ? -1 : 1)
                               : NAN;
            }
}

void oracle_curvature(const double *c, int nx, int ny, int nz, double h, double *kappa)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t x = idx3(i, j, k, nx, ny);
                kappa[x] = (c[x] > 0.0 && c[x] < 1.0) ? cell_curvature(c, nx, ny, nz, i, j, k, h) : NAN;
            }
}

/*
 * Surface-tension source f = sum_i gamma kappa_i grad C_i (Section 2.3) on
 * the faces of the grid: f_d at the low d-face of cell x, between x - e_d and
 * x, is sum_i gamma kappa_f,i (C_i(x) - C_i(x - e_d)) / h with kappa_f,i the
 * mean of the curvatures of the two cells that have one (the one of them
 * that does; 0 if neither).  c, kappa: [K][nz][ny][nx]; f: [3][nz][ny][nx].
 */
void oracle_surface_tension(const double *c, const double *kappa, int K, int nx, int ny, int nz,
                            double h, double gamma, double *f)
{
    int64_t N = (int64_t)nx * ny * nz;
    for (int d = 0; d < 3; ++d)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    int64_t x = idx3(i, j, k, nx, ny);
                    int64_t xl = idx3(d == 0 ? wrap(i - 1, nx) : i, d == 1 ? wrap(j - 1, ny) : j,
                                      d == 2 ? wrap(k - 1, nz) : k, nx, ny);
                    double acc = 0.0;
                    for (int q = 0; q < K; ++q) {
                        double kl = kappa[q * N + xl], kr = kappa[q * N + x];
                        double kf = 0.0;
                        if (isfinite(kl) && isfinite(kr))
                            kf = 0.5 * (kl + kr);
                        else if (isfinite(kl))
                            kf = kl;
                        else if (isfinite(kr))
                            kf = kr;
                        acc += gamma * kf * (c[q * N + x] - c[q * N + xl]) / h;
                    }
                    f[d * N + x] = acc;
                }
}

/* ------------------------------------------------------------------------ */
/* Tagging: breadth-first flood fill in linear-index order                   */

int64_t oracle_label(const double *c, int nx, int ny, int nz, double tau,
                     int connectivity, int32_t *label)
{
    int64_t N = (int64_t)nx * ny * nz;
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (N > 0 ? N : 1));
    if (!queue)
        return -1;
    memset(label, 0, sizeof(int32_t) * N);
    int32_t n = 0;
    for (int64_t s = 0; s < N; ++s) {
        if (!(c[s] > tau) || label[s] != 0)
            continue;
        ++n;
        int64_t head = 0, tail = 0;
        queue[tail++] = s;
        label[s] = n;
        while (head < tail) {
            int64_t x = queue[head++];
            int i = (int)(x % nx), j = (int)((x / nx) % ny), k = (int)(x / ((int64_t)nx * ny));
            for (int dk = -1; dk <= 1; ++dk)
                for (int dj = -1; dj <= 1; ++dj)
                    for (int di = -1; di <= 1; ++di) {
                        int nz_off = (di != 0) + (dj != 0) + (dk != 0);
                        if (nz_off == 0)
                            continue;
                        if (connectivity == 6 && nz_off != 1)
                            continue;
                        int64_t y = idx3(wrap(i + di, nx), wrap(j + dj, ny), wrap(k + dk, nz), nx, ny);
                        if (c[y] > tau && label[y] == 0) {
                            label[y] = n;
                            queue[tail++] = y;
                        }
                    }
        }
    }
    free(queue);
    return n;
}

/* ------------------------------------------------------------------------ */
/* Steps 1 and 3: near-contact criterion                                     */

/* Offsets delta of the (2w+1)^3 stencil with delta "positive" (first nonzero
 * component, taken in z, y, x order, is > 0): one per opposite pair. */
static int half_offsets(int w, int (*off)[3])
{
    int n = 0;
    for (int dz = -w; dz <= w; ++dz)
        for (int dy = -w; dy <= w; ++dy)
            for (int dx = -w; dx <= w; ++dx) {
                int pos = dz > 0 || (dz == 0 && (dy > 0 || (dy == 0 && dx > 0)));
                if (!pos)
                    continue;
                off[n][0] = dx;
                off[n][1] = dy;
                off[n][2] = dz;
                ++n;
            }
    return n;
}

void oracle_near_contact_map(const double *c, int nx, int ny, int nz, int w, double tau,
                             uint8_t *out)
{
    int n_off = ((2 * w + 1) * (2 * w + 1) * (2 * w + 1) - 1) / 2;
    int(*off)[3] = (int(*)[3])malloc(sizeof(int) * 3 * (n_off > 0 ? n_off : 1));
    half_offsets(w, off);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t x = idx3(i, j, k, nx, ny);
                out[x] = 0;
                if (c[x] > tau)
                    continue;
                for (int o = 0; o < n_off; ++o) {
                    int64_t a = idx3(wrap(i + off[o][0], nx), wrap(j + off[o][1], ny),
                                     wrap(k + off[o][2], nz), nx, ny);
                    int64_t b = idx3(wrap(i - off[o][0], nx), wrap(j - off[o][1], ny),
                                     wrap(k - off[o][2], nz), nx, ny);
                    if (c[a] > tau && c[b] > tau) {
                        out[x] = 1;
                        break;
                    }
                }
            }
    free(off);
}

int oracle_near_contact(const double *c, int nx, int ny, int nz, int w, double tau)
{
    int64_t N = (int64_t)nx * ny * nz;
    uint8_t *map = (uint8_t *)malloc(N > 0 ? N : 1);
    if (!map)
        return -1;
    oracle_near_contact_map(c, nx, ny, nz, w, tau, map);
    int any = 0;
    for (int64_t x = 0; x < N; ++x)
        any |= map[x];
    free(map);
    return any;
}

static int cmp_pair(const void *pa, const void *pb)
{
    const int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    return (a > b) - (a < b);
}

int64_t oracle_near_pairs(const double *c, const int32_t *label, int nx, int ny, int nz,
                          int w, double tau, int32_t *pa, int32_t *pb, int64_t cap)
{
    int n_off = ((2 * w + 1) * (2 * w + 1) * (2 * w + 1) - 1) / 2;
    int(*off)[3] = (int(*)[3])malloc(sizeof(int) * 3 * (n_off > 0 ? n_off : 1));
    half_offsets(w, off);
    int64_t n = 0, ncap = 1024;
    int64_t *keys = (int64_t *)malloc(sizeof(int64_t) * ncap);
    if (!off || !keys) {
        free(off);
        free(keys);
        return -1;
    }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t x = idx3(i, j, k, nx, ny);
                if (c[x] > tau)
                    continue;
                for (int o = 0; o < n_off; ++o) {
                    int64_t a = idx3(wrap(i + off[o][0], nx), wrap(j + off[o][1], ny),
                                     wrap(k + off[o][2], nz), nx, ny);
                    int64_t b = idx3(wrap(i - off[o][0], nx), wrap(j - off[o][1], ny),
                                     wrap(k - off[o][2], nz), nx, ny);
                    if (!(c[a] > tau && c[b] > tau))
                        continue;
                    int32_t la = label[a], lb = label[b];
                    if (la == lb)
                        continue;
                    int32_t lo = la < lb ? la : lb, hi = la < lb ? lb : la;
                    if (n == ncap) {
                        ncap *= 2;
                        int64_t *nk = (int64_t *)realloc(keys, sizeof(int64_t) * ncap);
                        if (!nk) {
                            free(off);
                            free(keys);
                            return -1;
                        }
                        keys = nk;
                    }
                    keys[n++] = ((int64_t)lo << 32) | (int64_t)(uint32_t)hi;
                }
            }
    qsort(keys, (size_t)n, sizeof(int64_t), cmp_pair);
    int64_t u = 0;
    for (int64_t t = 0; t < n; ++t) {
        if (t > 0 && keys[t] == keys[t - 1])
            continue;
        if (u < cap) {
            pa[u] = (int32_t)(keys[t] >> 32);
            pb[u] = (int32_t)(keys[t] & 0xffffffff);
        }
        ++u;
    }
    free(off);
    free(keys);
    return u;
}

/* ------------------------------------------------------------------------ */
/* Step 4: recolouring                                                       */

/*
 * Reading of Step 4 (the paper leaves the choices open):
 *  - Steps 1-3 are evaluated on every field active at the start of the call,
 *    on the state at the start of the call.
 *  - Per field, distinct pairs (a < b) in increasing order mark b as moving
 *    unless a or b is already moving.
 *  - Moving drops are handled in (field, label) order.  A drop of field i may
 *    go to the smallest active field n != i that has no occupied cell within
 *    Chebyshev distance 2w of any cell of the drop, counting both the
 *    occupancy at the start of the call and the drops already moved into n.
 *    Distance 2w is the reach of the (2w+1)^3 stencil, so a move can never
 *    create a new near contact.  If no field qualifies, field N is activated
 *    (if N < K); otherwise the drop stays and the call reports -4.
 *  - A move adds c_i to c_n on the drop's cells and sets c_i to 0 there.
 */
int oracle_recolour(double *c, int K, int *n_active, int nx, int ny, int nz, int w,
                    double tau, int connectivity, int *n_moved, int32_t *move_log,
                    int log_cap)
{
    int64_t N = (int64_t)nx * ny * nz;
    int na0 = *n_active;
    int status = 0, moved = 0, logged = 0;
    uint8_t *occ0 = (uint8_t *)calloc((size_t)(N * K), 1);
    uint8_t *added = (uint8_t *)calloc((size_t)(N * K), 1);
    int32_t *labels = (int32_t *)calloc((size_t)(N * K), sizeof(int32_t));
    int32_t **mv = (int32_t **)calloc((size_t)K, sizeof(int32_t *));
    int64_t *nmv = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    if (!occ0 || !added || !labels || !mv || !nmv)
        return -1;
    for (int64_t x = 0; x < N * K; ++x)
        occ0[x] = c[x] > tau;
    /* Steps 1-3 on the snapshot */
    for (int i = 0; i < na0; ++i) {
        const double *ci = c + (int64_t)i * N;
        if (oracle_near_contact(ci, nx, ny, nz, w, tau) != 1)
            continue;
        int32_t *lab = labels + (int64_t)i * N;
        int64_t nl = oracle_label(ci, nx, ny, nz, tau, connectivity, lab);
        int64_t np = oracle_near_pairs(ci, lab, nx, ny, nz, w, tau, NULL, NULL, 0);
        if (np <= 0)
            continue;
        int32_t *pa = (int32_t *)malloc(sizeof(int32_t) * np);
        int32_t *pb = (int32_t *)malloc(sizeof(int32_t) * np);
        oracle_near_pairs(ci, lab, nx, ny, nz, w, tau, pa, pb, np);
        uint8_t *moving = (uint8_t *)calloc((size_t)nl + 1, 1);
        for (int64_t p = 0; p < np; ++p)
            if (!moving[pa[p]] && !moving[pb[p]])
                moving[pb[p]] = 1;
        mv[i] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nl + 1));
        for (int64_t l = 1; l <= nl; ++l)
            if (moving[l])
                mv[i][nmv[i]++] = (int32_t)l;
        free(moving);
        free(pa);
        free(pb);
    }
    /* Step 4 */
    for (int i = 0; i < na0; ++i) {
        const int32_t *lab = labels + (int64_t)i * N;
        for (int64_t t = 0; t < nmv[i]; ++t) {
            int32_t b = mv[i][t];
            int target = -1;
            for (int n = 0; n < *n_active && target < 0; ++n) {
                if (n == i)
                    continue;
                const uint8_t *o0 = occ0 + (int64_t)n * N;
                const uint8_t *ad = added + (int64_t)n * N;
                int conflict = 0;
                for (int k = 0; k < nz && !conflict; ++k)
                    for (int j = 0; j < ny && !conflict; ++j)
                        for (int x0 = 0; x0 < nx && !conflict; ++x0) {
                            if (lab[idx3(x0, j, k, nx, ny)] != b)
                                continue;
                            for (int dk = -2 * w; dk <= 2 * w && !conflict; ++dk)
                                for (int dj = -2 * w; dj <= 2 * w && !conflict; ++dj)
                                    for (int di = -2 * w; di <= 2 * w; ++di) {
                                        int64_t y = idx3(wrap(x0 + di, nx), wrap(j + dj, ny),
                                                         wrap(k + dk, nz), nx, ny);
                                        if (o0[y] || ad[y]) {
                                            conflict = 1;
                                            break;
                                        }
                                    }
                        }
                if (!conflict)
                    target = n;
            }
            if (target < 0) {
                if (*n_active < K) {
                    target = *n_active;
                    *n_active += 1;
                } else {
                    status = -4;
                    continue;
                }
            }
            double *ci = c + (int64_t)i * N;
            double *cn = c + (int64_t)target * N;
            uint8_t *ad = added + (int64_t)target * N;
            for (int64_t x = 0; x < N; ++x)
                if (lab[x] == b) {
                    cn[x] += ci[x];
                    ci[x] = 0.0;
                    ad[x] = 1;
                }
            ++moved;
            if (move_log && logged < log_cap) {
                move_log[3 * logged + 0] = i;
                move_log[3 * logged + 1] = b;
                move_log[3 * logged + 2] = target;
                ++logged;
            }
        }
    }
    for (int i = 0; i < K; ++i)
        free(mv[i]);
    free(mv);
    free(nmv);
    free(occ0);
    free(added);
    free(labels);
    *n_moved = moved;
    return status;
}

/* ------------------------------------------------------------------------ */
/* Section 3: drop table and nearest-particle statistics                     */

void oracle_drop_table(const double *c, const int32_t *label, int64_t n_labels, int nx,
                       int ny, int nz, double h, double *vol, double *cen)
{
    int64_t *root = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_labels + 1));
    double *s0 = (double *)calloc((size_t)(n_labels + 1), sizeof(double));
    double *s1 = (double *)calloc((size_t)(3 * (n_labels + 1)), sizeof(double));
    for (int64_t l = 0; l <= n_labels; ++l)
        root[l] = -1;
    int L[3] = {nx, ny, nz};
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t x = idx3(i, j, k, nx, ny);
                int32_t l = label[x];
                if (l <= 0 || l > n_labels)
                    continue;
                if (root[l] < 0)
                    root[l] = x;
                int64_t r = root[l];
                int rc[3] = {(int)(r % nx), (int)((r / nx) % ny), (int)(r / ((int64_t)nx * ny))};
                int pc[3] = {i, j, k};
                s0[l] += c[x];
                for (int a = 0; a < 3; ++a) {
                    int dlt = pc[a] - rc[a];
                    if (2 * dlt >= L[a])
                        dlt -= L[a];
                    if (2 * dlt < -L[a])
                        dlt += L[a];
                    s1[3 * l + a] += c[x] * (double)dlt;
                }
            }
    for (int64_t l = 1; l <= n_labels; ++l) {
        int64_t r = root[l];
        int rc[3] = {(int)(r % nx), (int)((r / nx) % ny), (int)(r / ((int64_t)nx * ny))};
        vol[l - 1] = s0[l] * h * h * h;
        for (int a = 0; a < 3; ++a) {
            double p = ((double)rc[a] + 0.5 + s1[3 * l + a] / s0[l]) * h;
            double Lh = (double)L[a] * h;
            p = fmod(p, Lh);
            if (p < 0.0)
                p += Lh;
            if (p >= Lh) /* -tiny + L rounds to L */
                p = 0.0;
            cen[3 * (l - 1) + a] = p;
        }
    }
    free(root);
    free(s0);
    free(s1);
}

/* Eigenvalues of a symmetric 3x3 matrix by cyclic Jacobi rotations (each
 * rotation zeroes one off-diagonal entry; sweeps until the off-diagonal part
 * is below 1e-15 of the norm).  a is overwritten; w receives the diagonal. */
static void jacobi_eig3(double a[3][3], double w[3])
{
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        double nrm = off + a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (off <= 1e-30 * nrm)
            break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (a[p][q] == 0.0)
                    continue;
                /* angle with tan(2 theta) = 2 a_pq / (a_qq - a_pp) */
                double th = 0.5 * atan2(2.0 * a[p][q], a[q][q] - a[p][p]);
                double cs = cos(th), sn = sin(th);
                for (int k = 0; k < 3; ++k) { /* columns p, q */
                    double akp = a[k][p], akq = a[k][q];
                    a[k][p] = cs * akp - sn * akq;
                    a[k][q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < 3; ++k) { /* rows p, q */
                    double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = cs * apk - sn * aqk;
                    a[q][k] = sn * apk + cs * aqk;
                }
            }
    }
    for (int i = 0; i < 3; ++i)
        w[i] = a[i][i];
}

void oracle_drop_inertia(const double *c, const int32_t *label, int64_t n_labels, int nx, int ny,
                         int nz, double h, const double *cen, double *inertia, double *chi)
{
    int L[3] = {nx, ny, nz};
    memset(inertia, 0, sizeof(double) * 6 * (size_t)n_labels);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t x = idx3(i, j, k, nx, ny);
                int32_t l = label[x];
                if (l <= 0 || l > n_labels)
                    continue;
                int pc[3] = {i, j, k};
                double r[3];
                for (int a = 0; a < 3; ++a) {
                    double Lh = (double)L[a] * h;
                    double t = ((double)pc[a] + 0.5) * h - cen[3 * (l - 1) + a];
                    /* minimum image (the drop is smaller than half the box) */
                    while (t > 0.5 * Lh)
                        t -= Lh;
                    while (t < -0.5 * Lh)
                        t += Lh;
                    r[a] = t;
                }
                double w = c[x] * h * h * h;
                double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                double own = h * h / 6.0; /* the cell's own moment: its fluid fills the cube */
                double *I = inertia + 6 * (size_t)(l - 1);
                I[0] += w * (rr - r[0] * r[0] + own);
                I[1] += w * (rr - r[1] * r[1] + own);
                I[2] += w * (rr - r[2] * r[2] + own);
                I[3] -= w * r[0] * r[1];
                I[4] -= w * r[0] * r[2];
                I[5] -= w * r[1] * r[2];
            }
    for (int64_t l = 0; l < n_labels; ++l) {
        const double *I = inertia + 6 * (size_t)l;
        double a[3][3] = {{I[0], I[3], I[4]}, {I[3], I[1], I[5]}, {I[4], I[5], I[2]}};
        double w[3];
        jacobi_eig3(a, w);
        double mx = fmax(w[0], fmax(w[1], w[2])), mn = fmin(w[0], fmin(w[1], w[2]));
        chi[l] = mn > 0.0 ? sqrt(mx / mn) : INFINITY;
    }
}

void oracle_pair_stats(const double *cen, int64_t n, const double box[3], int vertical_axis,
                       int n_rbins, double dr, int n_tbins, double dtheta, double tie_tol,
                       double *hist_r, double *hist_rt, double *msum, double *rsum,
                       double *events)
{
    if (n < 2)
        return;
    double *dist = (double *)malloc(sizeof(double) * (size_t)n);
    double *rv = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        double dmin = INFINITY;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) {
                dist[j] = INFINITY;
                continue;
            }
            double r[3];
            for (int a = 0; a < 3; ++a) {
                double t = cen[3 * j + a] - cen[3 * i + a];
                if (t > 0.5 * box[a])
                    t -= box[a];
                if (t < -0.5 * box[a])
                    t += box[a];
                r[a] = t;
                rv[3 * j + a] = t;
            }
            dist[j] = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            if (dist[j] < dmin)
                dmin = dist[j];
        }
        int ni = 0;
        for (int64_t j = 0; j < n; ++j)
            if (j != i && dist[j] - dmin <= tie_tol)
                ++ni;
        double wgt = 1.0 / (double)ni;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i || !(dist[j] - dmin <= tie_tol))
                continue;
            double r = dist[j];
            double *v = rv + 3 * j;
            int kr = (int)floor(r / dr);
            if (kr > n_rbins || kr < 0)
                kr = n_rbins;
            double ct = r > 0.0 ? v[vertical_axis] / r : 1.0;
            if (ct > 1.0)
                ct = 1.0;
            if (ct < -1.0)
                ct = -1.0;
            double th = acos(ct);
            int kt = (int)floor(th / dtheta);
            if (kt >= n_tbins)
                kt = n_tbins - 1;
            if (kt < 0)
                kt = 0;
            hist_r[kr] += wgt;
            hist_rt[(int64_t)kr * n_tbins + kt] += wgt;
            for (int a = 0; a < 3; ++a) {
                msum[a] += wgt * v[a];
                for (int b = 0; b < 3; ++b)
                    rsum[3 * a + b] += wgt * v[a] * v[b];
            }
        }
        *events += 1.0;
    }
    free(dist);
    free(rv);
}

/* ------------------------------------------------------------------------ */
/* Learned normal estimator (MLP): canonical frame, forward, backprop       */

#define MLP_IN 32
#define MLP_HID 64
#define MLP_OUTP 16
#define MLP_NPARAM (MLP_HID * MLP_IN + MLP_HID * MLP_HID + MLP_OUTP * MLP_HID + MLP_HID + MLP_HID + MLP_OUTP)

void oracle_canon(const double st[27], double x[27], int sign[3], int perm[3])
{
    double y[3];
    youngs_raw(st, y);
    double ay[3];
    for (int a = 0; a < 3; ++a) {
        sign[a] = y[a] < 0.0 ? -1 : 1;
        ay[a] = fabs(y[a]);
    }
    /* stable order by |y|: an axis precedes another if smaller, ties by index */
    int order[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (ay[order[j]] < ay[order[i]] ||
                (ay[order[j]] == ay[order[i]] && order[j] < order[i])) {
                int tmp = order[i];
                order[i] = order[j];
                order[j] = tmp;
            }
    for (int q = 0; q < 3; ++q)
        perm[q] = order[q];
    for (int kc = -1; kc <= 1; ++kc)
        for (int jc = -1; jc <= 1; ++jc)
            for (int ic = -1; ic <= 1; ++ic) {
                int cv[3] = {ic, jc, kc}, o[3];
                for (int q = 0; q < 3; ++q)
                    o[perm[q]] = sign[perm[q]] * cv[q];
                x[(kc + 1) * 9 + (jc + 1) * 3 + (ic + 1)] = ST(st, o[0], o[1], o[2]) - 0.5;
            }
}

/* round to the nearest BF16 (ties to even) through the FP32 value */
static double bf16r(double v)
{
    float f = (float)v;
    uint32_t b;
    memcpy(&b, &f, 4);
    uint32_t lsb = (b >> 16) & 1u;
    b += 0x7fffu + lsb;
    b &= 0xffff0000u;
    memcpy(&f, &b, 4);
    return (double)f;
}

/* a layer input as the tensor-core path feeds it: the pair hi = bf16(v),
 * lo = bf16(v - hi), which carries about 16 significant bits of v */
static double bf16_pair(double v)
{
    double hi = bf16r(v);
    return hi + bf16r((double)((float)v - (float)hi));
}

typedef struct {
    const double *W1, *W2, *W3, *b1, *b2, *b3;
} mlp_view;

static mlp_view mlp_params(const double *p)
{
    mlp_view v;
    v.W1 = p;
    v.W2 = v.W1 + MLP_HID * MLP_IN;
    v.W3 = v.W2 + MLP_HID * MLP_HID;
    v.b1 = v.W3 + MLP_OUTP * MLP_HID;
    v.b2 = v.b1 + MLP_HID;
    v.b3 = v.b2 + MLP_HID;
    return v;
}

/* forward keeping the pre-activations a1, a2 and the (rounded) layer
 * inputs xin, h1, h2 */
static void mlp_fwd_full(const double *params, const double x[27], int bf16, double xin[MLP_IN],
                         double a1[MLP_HID], double h1[MLP_HID], double a2[MLP_HID], double h2[MLP_HID],
                         double out[3])
{
    mlp_view w = mlp_params(params);
    for (int i = 0; i < MLP_IN; ++i) {
        double v = i < 27 ? x[i] : 0.0;
        xin[i] = bf16 == 1 ? bf16_pair(v) : v;
    }
    for (int o = 0; o < MLP_HID; ++o) {
        double s = 0.0;
        for (int i = 0; i < MLP_IN; ++i) {
            double wv = bf16 ? bf16r(w.W1[o * MLP_IN + i]) : w.W1[o * MLP_IN + i];
            s += wv * xin[i];
        }
        a1[o] = s + w.b1[o];
        double h = a1[o] > 0.0 ? a1[o] : 0.0;
        h1[o] = bf16 == 1 ? bf16_pair(h) : h;
    }
    for (int o = 0; o < MLP_HID; ++o) {
        double s = 0.0;
        for (int i = 0; i < MLP_HID; ++i) {
            double wv = bf16 ? bf16r(w.W2[o * MLP_HID + i]) : w.W2[o * MLP_HID + i];
            s += wv * h1[i];
        }
        a2[o] = s + w.b2[o];
        double h = a2[o] > 0.0 ? a2[o] : 0.0;
        h2[o] = bf16 == 1 ? bf16_pair(h) : h;
    }
    for (int o = 0; o < 3; ++o) {
        double s = 0.0;
        for (int i = 0; i < MLP_HID; ++i) {
            double wv = bf16 ? bf16r(w.W3[o * MLP_HID + i]) : w.W3[o * MLP_HID + i];
            s += wv * h2[i];
        }
        out[o] = s + w.b3[o];
    }
}

void oracle_mlp_forward(const double *params, const double x[27], int bf16, double out[3])
{
    double xin[MLP_IN], a1[MLP_HID], h1[MLP_HID], a2[MLP_HID], h2[MLP_HID];
    mlp_fwd_full(params, x, bf16, xin, a1, h1, a2, h2, out);
}

double oracle_normal_residual(const double st[27], const double n[3])
{
    double l1 = fabs(n[0]) + fabs(n[1]) + fabs(n[2]);
    if (!(l1 > 0.0) || !isfinite(l1))
        return INFINITY;
    double m[3] = {n[0] / l1, n[1] / l1, n[2] / l1};
    double alpha = oracle_plic_alpha(m, ST(st, 0, 0, 0));
    double e = 0.0;
    for (int k = -1; k <= 1; ++k)
        for (int j = -1; j <= 1; ++j)
            for (int i = -1; i <= 1; ++i) {
                /* the plane m.x = alpha of the centre cell [0,1]^3, seen from
                 * the cell at offset (i,j,k): m.(x' + o) = alpha */
                double v = oracle_plic_volume(m, alpha - (m[0] * i + m[1] * j + m[2] * k));
                e += fabs(v - ST(st, i, j, k));
            }
    return e / 27.0;
}

int oracle_learned_normal(const double *params, const double st[27], double tol, double amb_eps,
                          int amb_choice, double m[3], int *ambiguous)
{
    double x[27], oc[3], n[3], mm[3];
    int sign[3], perm[3];
    oracle_canon(st, x, sign, perm);
    oracle_mlp_forward(params, x, 1, oc);
    for (int q = 0; q < 3; ++q)
        n[perm[q]] = sign[perm[q]] * oc[q];
    oracle_myc(st, mm);
    double e_net = oracle_normal_residual(st, n);
    double e_myc = oracle_normal_residual(st, mm);
    double thr = e_myc > tol ? e_myc : tol;
    int use_myc = !(e_net <= thr); /* also for a non-finite network output */
    int amb = isfinite(e_net) && fabs(e_net - thr) <= amb_eps;
    if (amb)
        use_myc = amb_choice;
    if (ambiguous)
        *ambiguous = amb;
    if (use_myc) {
        m[0] = mm[0];
        m[1] = mm[1];
        m[2] = mm[2];
        return 1;
    }
    double l1 = fabs(n[0]) + fabs(n[1]) + fabs(n[2]);
    m[0] = n[0] / l1;
    m[1] = n[1] / l1;
    m[2] = n[2] / l1;
    return 0;
}

double oracle_mlp_loss_grad(const double *params, const double *x, const double *t, int64_t n, int bf16,
                            double *grad)
{
    mlp_view w = mlp_params(params);
    double *gW1 = grad, *gW2 = gW1 + MLP_HID * MLP_IN, *gW3 = gW2 + MLP_HID * MLP_HID;
    double *gb1 = gW3 + MLP_OUTP * MLP_HID, *gb2 = gb1 + MLP_HID, *gb3 = gb2 + MLP_HID;
    memset(grad, 0, sizeof(double) * MLP_NPARAM);
    double loss = 0.0;
    for (int64_t s = 0; s < n; ++s) {
        double xin[MLP_IN], a1[MLP_HID], h1[MLP_HID], a2[MLP_HID], h2[MLP_HID], out[3];
        mlp_fwd_full(params, x + 27 * s, bf16, xin, a1, h1, a2, h2, out);
        const double *ts = t + 3 * s;
        double nrm = sqrt(out[0] * out[0] + out[1] * out[1] + out[2] * out[2]);
        double nh[3] = {out[0] / nrm, out[1] / nrm, out[2] / nrm};
        double cs = nh[0] * ts[0] + nh[1] * ts[1] + nh[2] * ts[2];
        loss += 1.0 - cs;
        /* d(1 - nh.t)/d out = -(t - (nh.t) nh) / |out|, averaged over n */
        double dy[3];
        for (int o = 0; o < 3; ++o)
            dy[o] = -(ts[o] - cs * nh[o]) / nrm / (double)n;
        double dh2[MLP_HID], da2[MLP_HID], dh1[MLP_HID], da1[MLP_HID];
        for (int o = 0; o < 3; ++o) {
            gb3[o] += dy[o];
            for (int i = 0; i < MLP_HID; ++i)
                gW3[o * MLP_HID + i] += dy[o] * h2[i];
        }
        for (int i = 0; i < MLP_HID; ++i) {
            double sacc = 0.0;
            for (int o = 0; o < 3; ++o)
                sacc += dy[o] * (bf16 ? bf16r(w.W3[o * MLP_HID + i]) : w.W3[o * MLP_HID + i]);
            dh2[i] = sacc;
            da2[i] = a2[i] > 0.0 ? dh2[i] : 0.0;
        }
        for (int o = 0; o < MLP_HID; ++o) {
            gb2[o] += da2[o];
            for (int i = 0; i < MLP_HID; ++i)
                gW2[o * MLP_HID + i] += da2[o] * h1[i];
        }
        for (int i = 0; i < MLP_HID; ++i) {
            double sacc = 0.0;
            for (int o = 0; o < MLP_HID; ++o)
                sacc += da2[o] * (bf16 ? bf16r(w.W2[o * MLP_HID + i]) : w.W2[o * MLP_HID + i]);
            dh1[i] = sacc;
            da1[i] = a1[i] > 0.0 ? dh1[i] : 0.0;
        }
        for (int o = 0; o < MLP_HID; ++o) {
            gb1[o] += da1[o];
            for (int i = 0; i < MLP_IN; ++i)
                gW1[o * MLP_IN + i] += da1[o] * xin[i];
        }
    }
    return loss / (double)n;
}
