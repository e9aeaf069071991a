/*
 * FP64 CPU oracle of the multi-field VoF step (arXiv 2407.07463).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It is a plain, slow,
 * obviously-correct restatement of what the GPU path computes and shares no
 * code, header, table or helper with it.
 *
 * Grid conventions: fields are C-contiguous [nz][ny][nx] (x fastest), cell
 * (i,j,k) occupies [i,i+1]x[j,j+1]x[k,k+1] in cell units, tri-periodic.
 * u[d] holds the velocity on the LOW d-face of each cell.  All reals FP64.
 */
#ifndef VOF_ORACLE_H
#define VOF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Section 2.2 (PLIC): volume of {x in [0,1]^3 : m.x < alpha}. */
double oracle_plic_volume(const double m[3], double alpha);
/* Plane constant alpha with oracle_plic_volume(m, alpha) = c (bisection). */
double oracle_plic_alpha(const double m[3], double c);

/* Normals from a 3x3x3 stencil st[(k+1)*9 + (j+1)*3 + (i+1)], offsets
 * i (x), j (y), k (z) in {-1,0,1}.  Normals point out of the c = 1 phase and
 * are L1-normalised. */
void oracle_youngs(const double st[27], double m[3]);
void oracle_centred_column(const double st[27], int axis, double m[3]);
void oracle_myc(const double st[27], double m[3]);
/* Youngs candidate and which candidate MYC picked: 0,1,2 = centred column
 * along x,y,z; 3 = Youngs. */
int oracle_myc_choice(const double st[27]);

/* Split flux through one face: donor reconstruction (m, alpha), sweep
 * direction d, Courant number s = u dt / h on the face (signed). */
double oracle_face_flux(const double m[3], double alpha, int d, double s);

/* Flux through the low d-face of cell (i,j,k) of field c with Courant number
 * s: donor selection, MYC, alpha and sub-cell volume. */
double oracle_cell_face_flux(const double *c, int nx, int ny, int nz,
                             int i, int j, int k, int d, double s);

/* One time step of every field: three split sweeps in the order rotated by
 * step_index, Weymouth-Yue divergence term with c_c from the start-of-step
 * field, clip to [0,1] after the third sweep.  c is [K][nz][ny][nx] and is
 * updated in place; clipped[k] (may be NULL) receives the volume removed by
 * the clip (negative if added).  Returns 0, or -1 on allocation failure. */
int oracle_advect_step(double *c, const double *u, int nx, int ny, int nz,
                       int K, double dt, double h, int64_t step_index,
                       double *clipped);

/* MYC normal of every cell of one field (3 doubles per cell; zeros for
 * cells with c <= 0 or c >= 1). */
void oracle_normals(const double *c, int nx, int ny, int nz, double *m_out);

/* Curvature of every cell of one field by height functions (Section 2.3,
 * kappa_i of each tracer): NaN where the cell is not interfacial or its 3x3
 * columns of 7 cells along the dominant MYC axis do not all contain the
 * interface; positive for a drop (2/R for a sphere of radius R). */
void oracle_curvature(const double *c, int nx, int ny, int nz, double h, double *kappa);
/* The same with the height axis and the side of the c = 1 phase given
 * (columns along `axis`, the phase at the -sign end) for every cell. */
void oracle_curvature_along(const double *c, int nx, int ny, int nz, double h, int axis, int sign,
                            double *kappa);

/* Surface-tension source f = sum_i gamma kappa_i grad C_i on the low
 * d-faces ([3][nz][ny][nx]) from c and kappa ([K][nz][ny][nx]); the face
 * curvature is the mean of the two cells' where both have one. */
void oracle_surface_tension(const double *c, const double *kappa, int K, int nx, int ny, int nz,
                            double h, double gamma, double *f);

/* Connected-component labels of {c > tau}/* Connected-component labels of {c > tau}, periodic, connectivity 6 or 26,
 * numbered 1..n in the order of each component's smallest linear index.
 * Returns n, or -1 on allocation failure. */
int64_t oracle_label(const double *c, int nx, int ny, int nz, double tau,
                     int connectivity, int32_t *label);

/* Threads of the OpenMP build (n > 0 sets them); 1 for the serial build. */
int oracle_threads(int n);

/* Step 1: 1 if some cell with c <= tau has two opposite cells of its
 * (2w+1)^3 stencil with c > tau. */
int oracle_near_contact(const double *c, int nx, int ny, int nz, int w,
                        double tau);
/* Per-cell Step 1 indicator (uint8 per cell). */
void oracle_near_contact_map(const double *c, int nx, int ny, int nz, int w,
                             double tau, uint8_t *out);

/* Step 3: distinct unordered label pairs (a < b) of opposite stencil cells
 * around an empty centre, sorted; returns the number found (entries beyond
 * cap are counted but not stored), or -1 on allocation failure. */
int64_t oracle_near_pairs(const double *c, const int32_t *label, int nx,
                          int ny, int nz, int w, double tau, int32_t *pa,
                          int32_t *pb, int64_t cap);

/* Steps 1-4 on every field active at the start of the call.  Returns 0,
 * or -4 when some drop found no free field (it stays in place).  Moves are
 * reported through n_moved and the field count through n_active.  If
 * move_log is not NULL, (field, label, target) triples are appended
 * (capacity log_cap triples). */
int oracle_recolour(double *c, int K, int *n_active, int nx, int ny, int nz,
                    int w, double tau, int connectivity, int *n_moved,
                    int32_t *move_log, int log_cap);

/* Drop volume and centroid (minimum-image unwrap about the drop's first
 * cell) for labels 1..n_labels.  cen is [n_labels][3] (x,y,z). */
void oracle_drop_table(const double *c, const int32_t *label,
                       int64_t n_labels, int nx, int ny, int nz, double h,
                       double *vol, double *cen);

/* Appendix A (deformation): inertia tensor of each drop about its centre of
 * mass, I = integral over the drop of [(r.r) delta - r r], r = x - x_cen
 * under the minimum image, with cen[n][3] from oracle_drop_table.  The
 * fluid of cell q (volume c_q h^3) is taken as filling the cube uniformly
 * about the cell centre, which adds c_q h^5 / 6 to each diagonal entry
 * (exact for full cells).  inertia[n][6] = (xx, yy, zz, xy, xz, yz);
 * chi[n] = sqrt(I_1 / I_2), I_1 and I_2 the largest and smallest
 * eigenvalues (Jacobi rotations). */
void oracle_drop_inertia(const double *c, const int32_t *label, int64_t n_labels, int nx, int ny,
                         int nz, double h, const double *cen, double *inertia, double *chi);

/* Nearest-particle statistics (Section 3): for every particle, its nearest
 * neighbours under the minimum image (ties within tie_tol share weight
 * 1/N_i), histograms of r and (r, theta), first and second moment sums.
 * hist_r has n_rbins+1 entries (last = overflow), hist_rt has
 * (n_rbins+1)*n_tbins.  Accumulates into the outputs. */
void oracle_pair_stats(const double *cen, int64_t n, const double box[3],
                       int vertical_axis, int n_rbins, double dr,
                       int n_tbins, double dtheta, double tie_tol,
                       double *hist_r, double *hist_rt, double *msum,
                       double *rsum, double *events);

/* Learned normal (no counterpart in the paper): canonical frame of a
 * stencil (reflect so every Youngs component is >= 0, axes ordered by
 * increasing |Youngs component|, ties to the lower axis); x[27] = canonical
 * stencil - 1/2.  sign[3], perm[3] describe the frame (canonical axis q is
 * original axis perm[q]). */
void oracle_canon(const double st[27], double x[27], int sign[3], int perm[3]);

/* MLP 27 -> 64 -> 64 -> 3, ReLU.  Weights as the GPU blob in FP32:
 * W1[64][32], W2[64][64], W3[16][64], b1[64], b2[64], b3[16] (flat, in that
 * order; 7312 values).  bf16 = 0: everything in FP64.  bf16 = 2: weights
 * rounded to BF16 (round to nearest even), layer inputs and everything else
 * in FP64.  bf16 = 1: as 2, and every layer input v (the 27 stencil values
 * and the two hidden activations) becomes hi + lo with hi = bf16(v),
 * lo = bf16(v - hi), as the tensor-core path feeds it.
 * out[3] = canonical-frame output. */
void oracle_mlp_forward(const double *params, const double x[27], int bf16, double out[3]);

/* Residual of a normal on a stencil (judge of the learned normal): the
 * plane of normal n through the centre cell with the centre's fraction,
 * extended over the 3x3x3 block; mean over the 27 cells of
 * |plane volume - c|.  +inf for a zero or non-finite n. */
double oracle_normal_residual(const double st[27], const double n[3]);

/* Learned normal with MYC fallback: the network's normal (mapped back from
 * the canonical frame, BF16 forward as above) unless it is non-finite or
 * its residual exceeds max(tol, residual of MYC's normal), then MYC's.
 * When the residual lies within amb_eps of that threshold the decision is
 * ambiguous between implementations that compute it in other precisions:
 * *ambiguous = 1 and amb_choice (0 network, 1 MYC) decides.  m receives the
 * L1-normalised normal; returns 0 (network) or 1 (MYC). */
int oracle_learned_normal(const double *params, const double st[27], double tol, double amb_eps,
                          int amb_choice, double m[3], int *ambiguous);

/* oracle_advect_step with oracle_learned_normal in place of MYC for every
 * interfacial donor.  counts[3] (may be NULL) receives the faces on the
 * network, on MYC, and how many of them were ambiguous decisions; amb_map
 * ([K][nz][ny][nx] bytes, may be NULL, not cleared) gets 1 on both cells of
 * every face whose decision was ambiguous and whose flux under the other
 * branch differs by more than 1e-7. */
int oracle_advect_step_learned(double *c, const double *u, int nx, int ny, int nz, int K,
                               double dt, double h, int64_t step_index, const double *params,
                               double tol, double amb_eps, int amb_choice, double *clipped,
                               int64_t counts[3], uint8_t *amb_map);

/* Loss 1 - cos(out, target) averaged over n canonical inputs x[n][27] with
 * canonical unit targets t[n][3]; grad (7312 values, same order as params)
 * receives d loss / d params (FP64 backprop through the same, optionally
 * BF16-rounded, forward).  Returns the loss. */
double oracle_mlp_loss_grad(const double *params, const double *x, const double *t, int64_t n,
                            int bf16, double *grad);

#ifdef __cplusplus
}
#endif
#endif
