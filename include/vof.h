/*
 * vof.h -- C ABI of the GB300 multi-field VoF library (libvof.so).
 *
 * One time step of K colour fields C_i on a tri-periodic uniform grid
 * (Section 2.3 of "Buoyancy driven motion of non-coalescing inertial drops",
 * arXiv 2407.07463): geometric PLIC transport of every field (Section 2.2,
 * Mixed-Youngs-Centred normals, plane-constant inversion, directionally split
 * fluxes), then the no-coalescence Steps 1-4 (near-contact test, tagging,
 * tagged near-contact pairs, recolouring), and the nearest-particle
 * statistics of Section 3 from the tags.
 *
 * Conventions shared by every entry point
 *  - Grids are C-contiguous [nz][ny][nx] (x fastest).  Cell (i,j,k) spans
 *    [i,i+1]x[j,j+1]x[k,k+1] in cells; positions are in units of h.
 *  - c is [K][nz][ny][nx]; u is [3][nz][ny][nx], u[d] being the velocity on
 *    the LOW d-face of the cell.  Element type: double for VOF_FP64, float for
 *    VOF_MIXED and VOF_MIXED_LEARNED.
 *  - "_dev" pointers are device memory of the current CUDA device, "_host"
 *    pointers host memory.  The caller owns every buffer; the library
 *    allocates no device memory after vof_init (all scratch lives in the
 *    caller's workspace) and never frees caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *    Work is enqueued on it; calls that return host values synchronise it.
 *  - Every call validates its arguments before launching anything and
 *    returns a vof_status; no C++ exception crosses the ABI.  VOF_ERR_CUDA
 *    and VOF_ERR_TIMEOUT are sticky: the context must then be destroyed.
 */
#ifndef VOF_H
#define VOF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VOF_OK = 0,
    VOF_ERR_ARG = -1,          /* invalid argument; nothing was launched */
    VOF_ERR_CUDA = -2,         /* a CUDA call failed (sticky) */
    VOF_ERR_WORKSPACE = -3,    /* workspace smaller than vof_workspace_size() */
    VOF_ERR_NO_FREE_FIELD = -4,/* Step 4 found no field for some drop (non-fatal) */
    VOF_ERR_CFL = -5,          /* max |u| dt / h > 1/2 */
    VOF_ERR_TIMEOUT = -6,      /* a bounded device wait gave up (sticky) */
    VOF_ERR_STATE = -7,        /* state blob does not match the context */
    VOF_ERR_NONFINITE = -8,    /* NaN or Inf in the velocity */
    VOF_ERR_CAPACITY = -9      /* a fixed-capacity list overflowed */
} vof_status;

typedef enum {
    VOF_FP64 = 0,          /* everything in double */
    VOF_MIXED = 1,         /* float storage, normals and fluxes; double alpha
                              near c = 0 or 1 and double clipping sums */
    VOF_MIXED_LEARNED = 2  /* VOF_MIXED with the learned normal estimator */
} vof_precision;

typedef struct {
    int32_t nx, ny, nz;      /* cells per axis, each >= 1; nx*ny*nz < 2^31 */
    int32_t k_capacity;      /* number of colour fields stored (K), 1..16 */
    int32_t k_active;        /* fields in use at start, N(0), 1..K */
    int32_t precision;       /* vof_precision */
    double h;                /* cell size > 0 */
    int32_t stencil_w;       /* near-contact half width w, 1..7 (2 = 5-cell stencil) */
    int32_t connectivity;    /* tagging connectivity: 6 or 26 */
    double tag_tau;          /* a cell belongs to a drop iff c > tag_tau (>= 0) */
    double alpha_fp64_band;  /* mixed path: alpha in double if c < band or
                                c > 1 - band */
    int32_t recolour;        /* 1: run Steps 1-4 after every step of vof_step */
    int32_t vertical_axis;   /* 0, 1, 2: axis theta is measured from */
    int32_t stats_rbins;     /* radial bins of the statistics (plus overflow) */
    int32_t stats_tbins;     /* polar bins over [0, pi] */
    double stats_dr;         /* radial bin width (length units) */
    int32_t stats_every;     /* > 0: vof_step accumulates one statistics event
                                (vof_stats without the read-back) after every
                                stats_every-th step of the context (Section 3
                                samples every 10 steps); 0: off */
} vof_config;

/* Fill `cfg` with defaults: 32^3, K = 1, FP64, h = 1, w = 2, 6-connectivity,
 * tau = 1e-6, band 1e-3, no recolouring, vertical axis z, 1024 x 150 bins of
 * width 0.2, no statistics sampling in vof_step. */
vof_status vof_config_default(vof_config *cfg);

typedef struct vof_ctx vof_ctx;

/* Bytes of device workspace vof_init needs for `cfg` (0 if cfg invalid). */
size_t vof_workspace_size(const vof_config *cfg);

/*
 * Create a context.  c_dev and u_dev are borrowed for the context's
 * lifetime (c is updated in place by vof_step / vof_recolour, u is read
 * only); workspace_dev must hold vof_workspace_size(cfg) bytes and be
 * 256-byte aligned.  Scans u once (synchronising `stream`): VOF_ERR_NONFINITE
 * if it holds NaN/Inf.  Fields k >= k_active must be zero.  All of a
 * context's work is enqueued on `stream` (no other stream is created).
 */
vof_status vof_init(const vof_config *cfg, void *c_dev, const void *u_dev,
                    void *workspace_dev, size_t workspace_bytes, void *stream,
                    vof_ctx **out);

/* Re-scan the borrowed velocity after the caller changed it. */
vof_status vof_set_velocity(vof_ctx *ctx, const void *u_dev);

typedef struct {
    int64_t steps_done;        /* total steps taken by this context */
    double clipped_volume;     /* volume removed by clipping during the call */
    int32_t n_active;          /* active fields N(t) after the call */
    int32_t n_moved;           /* drops moved by Step 4 during the call */
    int32_t near_contact_steps;/* steps whose Step 1 fired somewhere */
    int64_t field_steps;       /* sum over the call's steps of fields advected */
    int64_t faces_network;     /* VOF_MIXED_LEARNED: interfacial faces on the network's normal */
    int64_t faces_myc;         /* ... and on MYC's normal (the fallback) */
    int64_t faces_myc_judged;  /* faces whose MYC normal and residual were evaluated */
    int32_t n_in_use;          /* with recolouring: fields holding at least one occupied
                                  cell at the last step's Step 1, i.e. the tracer count
                                  N(t) of Section 2.3 (fields left empty by Step 4 are
                                  free for later moves); -1 without recolouring */
    int32_t n_in_use_max;      /* largest n_in_use over the call's steps (-1 as above) */
} vof_step_report;

/*
 * Advance every active field by `nsteps` steps of size dt (Section 2.2 /
 * 2.3, the transport equation of each C_i): per step, three split sweeps in
 * the order (x,y,z), (y,z,x), (z,x,y) by step index mod 3, each with
 * Mixed-Youngs-Centred normals and PLIC plane constants recomputed from the
 * current field, face fluxes of the upwind donor's sub-cell, the
 * Weymouth-Yue term c_c (u_hi - u_lo) with c_c = [c > 1/2] of the step's
 * start, and a clip to [0,1] after the third sweep.  With cfg.recolour,
 * Steps 1-4 run after every step (the host waits for Step 1's flags and,
 * where drops are in near contact, for their tag pairs and touch tests).
 * VOF_ERR_CFL if max |u| dt / h > 1/2.  `report` may be NULL.  Asynchronous
 * when recolouring is off and report is NULL.
 */
vof_status vof_step(vof_ctx *ctx, double dt, int32_t nsteps, vof_step_report *report);

/*
 * Learned normal for a VOF_MIXED_LEARNED context (no counterpart in the
 * paper; it replaces the MYC normal of Section 2.2 in the FP32 fluxes).
 * weights_dev: device blob of vof_mlp_weights_size() bytes (see
 * vof_mlp_forward), 16-byte aligned, borrowed until the context is
 * destroyed or the next vof_set_mlp.  In every listed donor stencil the
 * network's normal is kept when the mean residual over the 27 cells of its
 * plane (through the centre cell's fraction, extended over the block) is at
 * most fallback_tol (1e-3 by default) or no larger than MYC's; otherwise
 * MYC's normal is used.  VOF_ERR_ARG for another precision, a null or
 * unaligned blob, or a negative / non-finite tolerance.  vof_step on a
 * VOF_MIXED_LEARNED context without weights returns VOF_ERR_STATE; a
 * timed-out tensor-core wait is reported as VOF_ERR_TIMEOUT by the next
 * vof_step with a report.
 */
vof_status vof_set_mlp(vof_ctx *ctx, const void *weights_dev, double fallback_tol);

/* Step 1 for every active field: flags_host[k] = 1 if field k has a cell
 * with c <= tau whose (2w+1)^3 stencil holds two opposite cells with
 * c > tau (Section 2.3, Step 1; caption of figure fig:criterion).
 * Synchronises.  flags_host has k_capacity entries (inactive fields get 0). */
vof_status vof_near_contact(vof_ctx *ctx, int32_t *flags_host);

/*
 * Tagging (Section 2.3, tag.h): label_dev[nz][ny][nx] (int32, caller-owned)
 * receives 0 for cells with c <= tau and 1..n for the periodic connected
 * components of {c > tau} of field `field`, numbered in the order of each
 * component's smallest linear index.  *n_drops_host = n.  Synchronises.
 */
vof_status vof_label(vof_ctx *ctx, int32_t field, int32_t *label_dev, int32_t *n_drops_host);

/*
 * Tagging without allocation (the paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they need the
 * tags -- plug-ins whose host framework owns every device allocation and
 * passes in only finished buffers, loops whose memory budget is fixed at
 * start-up).  Same result as vof_label on the field c_dev ([nz][ny][nx],
 * double for VOF_FP64 else float; a cell is occupied iff c > tag_tau
 * evaluated in double) with the given connectivity (6 or 26), written to
 * label_dev (int32, caller-owned); *n_drops_host = number of components.
 * Needs no context and no workspace and calls no allocator: scratch is a
 * fixed device array inside the library (about 3 MB per device, kept until
 * the library is unloaded).  nx*ny*nz must not exceed 262144 (64^3): larger
 * grids return VOF_ERR_CAPACITY before anything is launched.  All calls on a
 * device share that array, which keeps the last call's contents (no call
 * reads a word it did not write first): calls that may overlap on the GPU
 * race and must be serialised by the caller.  The first call on each device
 * looks the array up (cudaGetSymbolAddress with that device current) and
 * should be made before any stream capture begins.  Synchronises `stream`.
 */
vof_status vof_label_noalloc(const void *c_dev, int32_t precision, int32_t nx, int32_t ny,
                             int32_t nz, double tag_tau, int32_t connectivity,
                             int32_t *label_dev, int32_t *n_drops_host, void *stream);

/*
 * Steps 1-4 on every active field (Section 2.3).  Steps 1-3 are evaluated on
 * the state at the start of the call; per field, sorted distinct tag pairs
 * (a < b) mark b as moving unless a or b already moves; moving drops, in
 * (field, tag) order, go to the smallest active field other than their own
 * with no occupied cell within Chebyshev distance 2w of the drop (counting
 * drops already moved into it), else to a newly activated field.  Moving
 * adds the drop's c to the target field and zeroes it in the source field.
 * VOF_ERR_NO_FREE_FIELD if some drop found no field with K exhausted (it
 * stays; the rest of the call completes).  Synchronises.
 */
vof_status vof_recolour(vof_ctx *ctx, int32_t *n_moved, int32_t *n_active);

typedef struct {
    int32_t n_drops;      /* drops in all active fields */
    double d;             /* equivalent diameter (6 Vbar / pi)^(1/3) */
    double n_p;           /* number density n_drops / L^3 */
    double volume;        /* total dispersed volume sum_k sum c h^3 */
    double events;        /* accumulated events E (one per drop per call) */
    double M[3];          /* first moment  sum h_ij r / E (accumulated) */
    double R[9];          /* second moment sum h_ij r r^T / E (accumulated) */
    double A[9];          /* R - tr(R)/3 delta */
    double chi_mean;      /* Appendix A: mean aspect ratio chi_p over all drops of all
                             accumulated events */
    double chi_max;       /* largest chi seen */
    double chi_drops;     /* drops whose chi entered the mean */
} vof_stats_out;

/*
 * Nearest-particle statistics (Section 3): tag every active field, compute
 * each drop's volume and centroid (minimum image about the drop's first
 * cell), then for every drop its nearest neighbours among all drops of all
 * fields under the minimum image (ties within 1e-12 d share h_ij = 1/N_i),
 * and accumulate the events into histograms over r (stats_rbins bins of
 * width stats_dr plus an overflow bin) and over (r, theta) with theta the
 * angle to the vertical axis (stats_tbins bins over [0, pi]), and into the
 * moment sums, and each drop's aspect ratio chi (see vof_drop_shape) into
 * the running chi_mean / chi_max.  hist_r_host (stats_rbins + 1 doubles) and hist_rt_host
 * ((stats_rbins + 1) * stats_tbins doubles, r-major) receive the accumulated
 * histograms if not NULL.  reset != 0 clears the accumulators first.
 * Synchronises.
 */
vof_status vof_stats(vof_ctx *ctx, int32_t reset, vof_stats_out *out, double *hist_r_host,
                     double *hist_rt_host);

/*
 * Curvature kappa of field `field` by height functions (Section 2.3: the
 * surface-tension force sums gamma kappa_i grad C_i over the tracers, each
 * curvature computed as for a single tracer).  For every interfacial cell
 * (0 < c < 1): along the axis of the largest |component| of its MYC normal,
 * the 3x3 columns of 7 cells centred on it give heights H = sum of c; if
 * each column's end on the c = 1 side holds more than 1/2 and its other end
 * less than 1/2, kappa = -[H_xx (1 + H_y^2) + H_yy (1 + H_x^2) -
 * 2 H_xy H_x H_y] / (1 + H_x^2 + H_y^2)^(3/2) / h with centred differences
 * (2/R for a drop of radius R), else NaN; NaN for cells that are not
 * interfacial.  kappa_dev [nz][ny][nx] of the context's element type.
 * Asynchronous.
 */
vof_status vof_curvature(vof_ctx *ctx, int32_t field, void *kappa_dev);

/*
 * Surface-tension source f = sum_i gamma kappa_i grad C_i over the active
 * fields (Section 2.3), on the faces of the grid: f_dev [3][nz][ny][nx] of
 * the context's element type receives at the low d-face of cell x
 * sum_i gamma kappa_f,i (C_i(x) - C_i(x - e_d)) / h, kappa_f,i being the mean
 * of the curvatures (vof_curvature) of the face's two cells where both have
 * one, the one that does, or 0.  Uses the workspace's flux buffer as
 * scratch.  VOF_ERR_ARG for a null f_dev or non-finite gamma.  Asynchronous.
 */
vof_status vof_surface_tension(vof_ctx *ctx, double gamma, void *f_dev);

/*
 * Drop shape (Appendix A)/*
 * Drop shape (Appendix A): the inertia tensor of each drop about its centre
 * of mass, I = integral over the drop of [(r.r) delta - r r], r = x - x_cen
 * under the minimum image, for the drop's colour density (each cell of the
 * tag holding its c uniformly: the cell-centre term plus the cube's own
 * c h^5 / 6 on the diagonal), and its aspect ratio chi = sqrt(I_1 / I_2)
 * with I_1, I_2 the largest and smallest eigenvalues.  label_dev: this
 * field's tags (vof_label), cen_dev [n][3] the centroids of vof_drop_table;
 * inertia_dev [n][6] (double) receives xx yy zz xy xz yz, chi_dev [n]
 * (double, may be NULL) chi.  Asynchronous.
 */
vof_status vof_drop_shape(vof_ctx *ctx, int32_t field, const int32_t *label_dev, int32_t n_labels,
                          const double *cen_dev, double *inertia_dev, double *chi_dev);

/* Per-drop table of one field given its labels: vol_dev[n] (double) and
 * cen_dev[n][3] (double, x y z in [0, L h)).  Section 2.3 (drop properties
 * by integrating C_i over the cells of a tag).  Asynchronous. */
vof_status vof_drop_table(vof_ctx *ctx, int32_t field, const int32_t *label_dev,
                          int32_t n_labels, double *vol_dev, double *cen_dev);

/*
 * Stateless nearest-particle statistics of n centroids cen_dev[n][3]
 * (double) in a periodic box box_host[3] (Section 3, eqs. P_nstij, vec_cond,
 * Ptheta_r): accumulates into hist_r_dev[n_rbins+1], hist_rt_dev
 * [(n_rbins+1)*n_tbins] and moments_dev[13] = {sum h r (3), sum h r r^T (9),
 * E}.  Asynchronous on `stream`.
 */
vof_status vof_pair_stats(const double *cen_dev, int64_t n, const double *box_host,
                          int32_t vertical_axis, int32_t n_rbins, double dr, int32_t n_tbins,
                          double dtheta, double tie_tol, double *hist_r_dev,
                          double *hist_rt_dev, double *moments_dev, void *stream);

/* PLIC primitives on n independent cells (Section 2.2): volume of
 * {x in [0,1]^3 : m.x < alpha} and its inverse alpha(m, c).  m is [n][3];
 * all arrays of `precision`'s element type (double for VOF_FP64).  The mixed
 * precisions compute alpha in double when c < band or c > 1 - band.
 * Asynchronous on `stream`. */
vof_status vof_plic_volume(int32_t precision, const void *m_dev, const void *alpha_dev,
                           void *v_dev, int64_t n, void *stream);
vof_status vof_plic_alpha(int32_t precision, const void *m_dev, const void *c_dev,
                          void *alpha_dev, int64_t n, double band, void *stream);

/* Mixed-Youngs-Centred normal of every cell of `field` (m_dev [N][3] of the
 * context's element type; zero where c <= 0 or c >= 1).  Asynchronous. */
vof_status vof_normals(vof_ctx *ctx, int32_t field, void *m_dev);

/*
 * Learned normal estimator (no counterpart in the paper, which uses the PLIC
 * normals this replaces): an MLP 27 -> 64 -> 64 -> 3 with ReLU, BF16 weights
 * and activations, FP32 accumulation on the tensor cores, applied to the
 * 3x3x3 stencil after reflecting it so that every Youngs component is >= 0
 * and permuting its axes by increasing |Youngs component|; input c - 1/2.
 * The weight blob (vof_mlp_weights_size() bytes, device memory) holds
 * W1[64][32], W2[64][64], W3[16][64] (BF16, row = output, zero padding)
 * and b1[64], b2[64], b3[16] (FP32).  Each input x enters as the BF16 pair
 * hi = bf16(x), lo = bf16(x - hi), both multiplied by W1 (16 significant
 * bits of c instead of 8).
 */
size_t vof_mlp_weights_size(void);

/* Normals of n raw stencils (stencils_dev [n][27] float, order
 * (k+1)*9+(j+1)*3+(i+1)) through the network: normals_dev [n][3] float,
 * L2-normalised, pointing out of the c = 1 phase.  Synchronises `stream`;
 * VOF_ERR_TIMEOUT if a tensor-core completion wait gave up. */
vof_status vof_mlp_forward(const void *weights_dev, const float *stencils_dev, float *normals_dev,
                           int64_t n, void *stream);

/* The learned normal exactly as the VOF_MIXED_LEARNED step applies it to a
 * donor stencil (see vof_set_mlp): network, mapped back from the canonical
 * frame, kept when its 27-cell mean residual is <= fallback_tol or no larger
 * than MYC's, else MYC's normal.  stencils_dev float [n][27] as in
 * vof_mlp_forward; normals_dev float [n][3] receives the L1-normalised
 * choice, which_dev int32 [n] 0 (network) or 1 (MYC).  Synchronises
 * `stream`.  VOF_ERR_ARG on a bad pointer, n < 0 or a negative tolerance;
 * VOF_ERR_TIMEOUT on a timed-out tensor-core wait. */
vof_status vof_learned_normals(const void *weights_dev, const float *stencils_dev, int64_t n,
                               double fallback_tol, float *normals_dev, int32_t *which_dev,
                               void *stream);

/* Training on the GPU (forward and backward passes on the tensor cores,
 * Adam on FP32 master weights, cosine learning-rate decay).  Samples are
 * stencils of planes (normal uniform on the sphere, offset so the centre
 * cell is cut, cell fractions from the exact PLIC volume) and of spheres
 * (radius log-uniform in [r_min, r_max] cells, surface within 0.4 cells of
 * the centre cell's centre, half of them inverted, cell fractions by
 * quadrature); the target is the plane normal or the radial direction,
 * pointing out of the c = 1 phase.  Loss 1 - cos(output, target). */
typedef struct {
    int64_t n_train;       /* training stencils (>= 128) */
    int64_t n_test;        /* held-out stencils drawn with another seed */
    int32_t epochs;
    int32_t batch;         /* samples per Adam step, 128 .. 2^20, <= n_train */
    float lr;              /* initial Adam step */
    uint64_t seed;
    float plane_fraction;  /* share of plane samples */
    float r_min, r_max;    /* sphere radii in cells */
} vof_train_params;

typedef struct {
    float final_loss;           /* mean loss over (up to 2^20) training samples */
    int32_t steps;              /* Adam steps taken */
    double test_mean_deg_mlp;   /* held-out mean angular error of the network */
    double test_mean_deg_myc;   /* ... and of MYC on the same stencils */
    double test_p95_deg_mlp;    /* held-out 95th percentiles */
    double test_p95_deg_myc;
    double test_mean_deg_combined; /* network with MYC fallback (residual judge, tol 1e-3) */
    double test_p95_deg_combined;
    double test_network_share;  /* share of held-out stencils that keep the network's normal */
    /* held-out means by class: 0 planes, spheres of radius 1: [2,4), 2: [4,8),
     * 3: [8,16), 4: [16, r_max] cells */
    int64_t bin_count[5];
    double bin_mean_deg_mlp[5];
    double bin_mean_deg_myc[5];
    double bin_mean_deg_combined[5];
} vof_train_report;

vof_status vof_mlp_train_params_default(vof_train_params *tp);
size_t vof_mlp_train_workspace_size(const vof_train_params *tp);
/* Train; weights_dev receives the blob.  Synchronises `stream`. */
vof_status vof_mlp_train(const vof_train_params *tp, void *weights_dev, void *workspace_dev,
                         size_t workspace_bytes, void *stream, vof_train_report *report);
/* Gradient of the mean loss over n stencils (raw frame [n][27], unit targets
 * [n][3]) with respect to the flat FP32 parameters W1[64][32], W2[64][64],
 * W3[16][64], b1[64], b2[64], b3[16] (7312 values): grad_dev; loss_dev[0] =
 * sum of the per-sample losses.  Synchronises `stream`. */
vof_status vof_mlp_grad(const void *weights_dev, const float *stencils_dev, const float *targets_dev,
                        int64_t n, float *grad_dev, float *loss_dev, void *stream);
/* Flat FP32 parameters (order as vof_mlp_grad) -> weight blob.  Async. */
vof_status vof_mlp_params_to_weights(const float *params_dev, void *weights_dev, void *stream);

/* Instrumentation: D[128][n] = A[128][k] B[n][k]^T through one CTA's
 * tensor-core path (operands rounded to BF16, FP32 result), to check the
 * shared-memory operand layout; variant 1 swaps the descriptor's two byte
 * offsets.  k, n in {16, 32, 64}.  Synchronises `stream`. */
vof_status vof_tc_gemm_check(const float *a_dev, const float *b_dev, float *d_dev, int32_t k, int32_t n,
                             int32_t variant, void *stream);

/* Checkpoint: a self-describing blob of the fields, N(t), the step count
 * and the statistics accumulators.  vof_state_size gives its size. */
size_t vof_state_size(const vof_ctx *ctx);
vof_status vof_get_state(vof_ctx *ctx, void *host_buf, size_t bytes);
vof_status vof_set_state(vof_ctx *ctx, const void *host_buf, size_t bytes);

/* Number of kernel launches this context has issued (instrumentation). */
int64_t vof_launch_count(const vof_ctx *ctx);

/*
 * Kernel timing (instrumentation, no counterpart in the paper).  While
 * enabled, every kernel the context launches is bracketed by a pair of CUDA
 * events recorded on the context stream (up to 16384 launches; later ones
 * are not recorded).  vof_profile_read synchronises the stream, writes per
 * kernel class the number of recorded launches and their summed device time
 * in milliseconds (arrays of n entries; classes beyond n are dropped) and
 * clears the record.  vof_profile_class_name names class i (NULL past the
 * last class).  Events are created at the first enable and destroyed by
 * vof_destroy; no device memory is allocated.
 */
vof_status vof_profile_enable(vof_ctx *ctx, int32_t enable);
vof_status vof_profile_read(vof_ctx *ctx, int64_t *launches, double *ms, int32_t n);
const char *vof_profile_class_name(int32_t cls);

/* ------------------------------------------------------------------------
 * Batches of independent boxes (no counterpart in the paper, which
 * advances one box).  Every box follows the arithmetic of vof_step without
 * recolouring: the Section 2.2 split advection of each active field, the
 * Weymouth-Yue term, the clip after the third sweep and the occupancy bits.
 * Each pass of a sweep is one launch covering every field of every box; a
 * step is replayed from a captured CUDA graph (one graph per sweep rotation
 * and list parity, captured on first use); the launch shape of the update
 * pass (warps per block, resident blocks per SM) is chosen by timing the
 * candidates on the batch's own first sweep (vof_batch_tune, run by the
 * first vof_batch_step when cfg.autotune is set).  The library allocates
 * nothing: the caller passes one device workspace.
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t nx, ny, nz;  /* cells; nx a multiple of 4 (FP32) or 2 (FP64) */
    int32_t k_capacity;  /* fields stored in c_dev, 1..16 */
    int32_t k_active;    /* fields advected, 1..k_capacity */
    void *c_dev;         /* [k_capacity][nz][ny][nx], 16-byte aligned, updated in place */
    const void *u_dev;   /* [3][nz][ny][nx] low-face velocities, 16-byte aligned */
    double dt;           /* time step of this box; max |u| dt / h <= 1/2 */
} vof_box_desc;

typedef struct {
    int32_t precision;       /* vof_precision, the same for every box */
    double h;                /* cell size of every box */
    double tag_tau;          /* occupancy threshold of the bits (default 1e-6) */
    double alpha_fp64_band;  /* as in vof_config (FP32 paths) */
    int32_t use_graph;       /* 1: replay captured graphs (default 1) */
    int32_t autotune;        /* 1: tune the update launch shape (default 1) */
} vof_batch_config;

typedef struct {
    int64_t steps_done;
    int32_t n_boxes;
    int64_t cell_fields_per_step;  /* sum over boxes of cells x active fields */
    double clipped_volume[64];     /* per box, accumulated since init */
    int64_t faces_network, faces_myc; /* VOF_MIXED_LEARNED, accumulated */
    int64_t faces_myc_judged;      /* faces whose MYC residual was evaluated */
    int32_t update_warps, update_blocks_per_sm; /* launch shape in use */
    int32_t tune_candidates;       /* shapes timed by the tuner (0: not tuned) */
    float tune_best_ms;            /* median first-sweep time of the chosen shape */
    int64_t graph_launches, direct_steps;
} vof_batch_report_t;

typedef struct vof_batch vof_batch;

vof_status vof_batch_config_default(vof_batch_config *cfg);
/* Bytes of workspace for the batch; 0 for an invalid config or box (see
 * vof_box_desc), or n_boxes outside 1..64. */
size_t vof_batch_workspace_size(const vof_batch_config *cfg, const vof_box_desc *boxes, int32_t n_boxes);
/* Borrows the boxes' c and u and the workspace (256-byte aligned) until
 * vof_batch_destroy.  Scans every velocity: VOF_ERR_NONFINITE, VOF_ERR_CFL
 * (max |u| dt / h > 1/2 in some box), VOF_ERR_WORKSPACE, VOF_ERR_ARG. */
vof_status vof_batch_init(const vof_batch_config *cfg, const vof_box_desc *boxes, int32_t n_boxes,
                          void *workspace_dev, size_t workspace_bytes, void *stream, vof_batch **out);
/* Learned normal for a VOF_MIXED_LEARNED batch (as vof_set_mlp). */
vof_status vof_batch_set_mlp(vof_batch *batch, const void *weights_dev, double fallback_tol);
/* Times the update launch shapes on the batch's first sweep (the state is
 * not modified) and keeps the fastest. */
vof_status vof_batch_tune(vof_batch *batch);
/* nsteps steps of every box, asynchronous on the batch's stream. */
vof_status vof_batch_step(vof_batch *batch, int32_t nsteps);
/* Synchronises; VOF_ERR_TIMEOUT if a tensor-core wait gave up. */
vof_status vof_batch_report(vof_batch *batch, vof_batch_report_t *report);
void vof_batch_destroy(vof_batch *batch);

/* Exercises the bounded device wait of the tensor-core kernels on an
 * mbarrier that nothing arrives at: the wait gives up after poll_limit
 * polls (1..1e8) and the call returns VOF_ERR_TIMEOUT with the device
 * still usable.  For tests of the failure path; no fault is raised. */
vof_status vof_wait_selftest(int64_t poll_limit, void *stream);

const char *vof_status_string(vof_status s);
/* Name of the last CUDA error a call of this thread met and reported as
 * VOF_ERR_CUDA ("no error" if none). */
const char *vof_last_cuda_error(void);
void vof_destroy(vof_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* VOF_H */
