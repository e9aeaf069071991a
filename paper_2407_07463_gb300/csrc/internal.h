// Internal host-side launchers of the GB300 VoF library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

#include <vector>

namespace vof {

// Kernel classes of the launch timer (vof_profile_*).
enum ProfClass {
    P_FIND_FACES = 0,
    P_FACE_FLUX,
    P_UPDATE,
    P_PACK_BITS,
    P_NEAR_CONTACT,
    P_LABEL,
    P_PAIRS,
    P_TOUCH,
    P_MOVE,
    P_STATS,
    P_MISC,
    P_NET_NORMALS,
    P_SCAN,
    P_COUNT
};

// Optional CUDA-event bracketing of kernel launches on one stream.
struct Prof {
    bool on = false;
    int cap = 0, n = 0, pending = -1;
    std::vector<cudaEvent_t> ev;  // 2 * cap
    std::vector<int> cls;         // cap
    cudaStream_t st = nullptr;
    void begin(int c) {
        pending = -1;
        if (!on || n >= cap) return;
        cudaEventRecord(ev[2 * n], st);
        pending = c;
    }
    void end() {
        if (pending < 0) return;
        cudaEventRecord(ev[2 * n + 1], st);
        cls[n] = pending;
        ++n;
        pending = -1;
    }
};

constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kPairCap = 1 << 16;     // distinct tagged near-contact pairs per call
constexpr int kMoveCap = 2048;        // moving drops per recolour call
constexpr int kDropCap = 1 << 20;     // drops over all fields for statistics
constexpr int kSweepBlocks = 152 * 64; // most blocks (and face-list segments) of a sweep (buffer capacity)

// Keeps the name of the last CUDA error a library call met (for
// vof_last_cuda_error); returns the error unchanged.
cudaError_t note_cuda_error(cudaError_t e);
const char* last_cuda_error_name();
struct SweepArgs;
struct MlpBlob;
struct MoveTables;
template <typename T, int NB>
struct BoxSet;
constexpr int kMaxBoxes = 64;
// Largest grid of the list-producing passes.
constexpr int kListBlocks = 2048;
// Learned normal of a box set (FP32 path): network normals of the listed
// faces of one sweep (tensor cores), then their judged fluxes;
// counters[0/1] += faces on the network's / MYC's normal.
template <int NB>
void face_normals_net_set(const BoxSet<float, NB>& S, int d, int sweep, const unsigned long long* list, long long cap,
                          const int* off, int nseg, const int* tile_seg, const MlpBlob* w, int* status,
                          cudaStream_t st);
template <int NB>
void face_flux_judged_set(const BoxSet<float, NB>& S, int d, int sweep, float band, const unsigned long long* list,
                          long long cap, const int* off, int nseg, const int* tile_seg, float tol,
                          unsigned long long* counters, cudaStream_t st);
// nsteps steps of every box of a set (one box: a context; up to kMaxBoxes:
// a batch).
cudaError_t advect_set_fp64(const BoxSet<double, 1>& S, SweepArgs& a, int nsteps);
cudaError_t advect_set_fp32(const BoxSet<float, 1>& S, SweepArgs& a, int nsteps);
cudaError_t advect_set_fp64(const BoxSet<double, kMaxBoxes>& S, SweepArgs& a, int nsteps);
cudaError_t advect_set_fp32(const BoxSet<float, kMaxBoxes>& S, SweepArgs& a, int nsteps);
// After Step 4 moved drops of a context's box: the faces of the current
// list whose donor moved take the drop's target field (d: the direction of
// the sweep the list serves; bits and labels: Step 1's occupancy and Step
// 2's tags; target[m]: the field drop m moved to, or -1).
cudaError_t patch_list_fp32(const BoxSet<float, 1>& S, SweepArgs& a, int d, const uint32_t* bits, const int* labels,
                            const MoveTables& mt, const int* target);
cudaError_t patch_list_fp64(const BoxSet<double, 1>& S, SweepArgs& a, int d, const uint32_t* bits, const int* labels,
                            const MoveTables& mt, const int* target);
// Resident blocks per SM of a batch's update pass with `warps` warps per
// block (0 if the query fails), asked of the unit that launches it.
int update_occupancy(bool fp64, int warps);
int update_occupancy_fp64(int warps);
// Listing and first sweep of a batch only (state untouched; for timing).
cudaError_t advect_first_sweep_fp64(const BoxSet<double, kMaxBoxes>& S, SweepArgs& a);
cudaError_t advect_first_sweep_fp32(const BoxSet<float, kMaxBoxes>& S, SweepArgs& a);
// Face-list entries to reserve per list for K fields of grid g (either
// sweep path, any launch shape the advance may choose): a warp of the
// vectorised passes lists up to 2 faces per cell of every field of each of
// its row chunks, and the segments of a grid carry the slack of their last
// chunks.
inline long long list_reserve(int nx, int ny, int nz, int K, int es) {
    const long long rows = (long long)ny * nz, words = rows * ((nx + 31) / 32);
    const long long scalar = 2LL * 32 * K * (words + kSweepBlocks);
    const long long CH = 512 / es, cpr = (nx + CH - 1) / CH;
    const long long vec = 2LL * CH * K * (rows * cpr + 8LL * kListBlocks);
    return scalar > vec ? scalar : vec;
}

// Exclusive scan of n ints (one block); off[n] = total.
cudaError_t scan_counts(const int* counts, int* off, int n, cudaStream_t st);
// Face lists: consumers take tiles of kFaceTile consecutive entries.
constexpr int kFaceTile = 128;
// Exclusive scan of the segment lengths of a face list, plus tile_seg[t] =
// the segment holding entry t * kFaceTile (t < tile_cap).
cudaError_t scan_face_counts(const int* counts, int* off, int n, int* tile_seg, int tile_cap, cudaStream_t st);
cudaError_t pack_bits(const void* c, bool fp64, uint32_t* bits, const Dims& g, int K, double tau,
                      cudaStream_t st);
// Box dilation (Chebyshev distance reach, periodic) of n bit planes from src
// into dst; tmp: n planes of scratch.
cudaError_t dilate_planes(const uint32_t* src, uint32_t* dst, uint32_t* tmp, int n, const Dims& g, int reach,
                          cudaStream_t st);
// Step 1 per field: flags[f] |= 1 if it fired, |= 2 if the field holds an
// occupied cell (flags cleared by the caller).
cudaError_t near_contact(const uint32_t* bits, uint32_t* ncmap, int* flags, const Dims& g, int K, int w,
                         cudaStream_t st);
// Tags of one field's occupancy bits: label (0 empty, else 1 + the rank of
// the component's root, its smallest cell), *n_out the tag count, root_of[l
// - 1] the root cell of tag l <= root_cap (if not null).  parent, rank,
// block_tot and block_off are scratch: parent does not hold every cell's
// root afterwards.
cudaError_t label_field(const uint32_t* bits_f, const Dims& g, int conn, int* parent, int* rank,
                        int* block_tot, int* block_off, int* label, int* root_of, int root_cap, int* n_out,
                        cudaStream_t st, long long* launches);
// Fields tagged by one chain of launches (slot s = blockIdx.y takes field
// f[s]).  A field's bit plane, near-contact map and labels sit f * words and
// f * N from their bases and its drop count at n_out[f]; a slot's scratch
// sits s * N (parent, rank) and s * (nb + 1) (block totals and offsets, nb =
// ceil(N / 1024)) from theirs.  Labels are complete only at occupied cells
// (empty cells of a row word without an occupied cell keep what they held).
constexpr int kLabelSlots = 16;
struct LabelSlots {
    int n;
    int f[kLabelSlots];
};
cudaError_t label_fields(const uint32_t* bits, const Dims& g, int conn, const LabelSlots& ls, int* parent, int* rank,
                         int* block_tot, int* block_off, int* labels, int* n_out, cudaStream_t st,
                         long long* launches);
// Step 3 for the slots' fields: distinct pairs of the tags of opposite
// occupied cells around every near-contact cell, into the set `table`.
cudaError_t tag_pairs_fields(const uint32_t* ncmap, const uint32_t* bits, const int* labels, const Dims& g, int w,
                             const LabelSlots& ls, unsigned long long* table, int cap, int* overflow,
                             cudaStream_t st);
cudaError_t compact_pairs(const unsigned long long* table, int cap, unsigned long long* out,
                          unsigned long long* count, cudaStream_t st);

// Step 4 helpers.  Moving drops are listed per field in increasing label
// order: mv_label[mv_start[f] .. mv_start[f] + mv_count[f]).
// mv_map: a bit per (field, tag) below kMoveMapTags, set for moving drops
// (a lookup without the search); larger tags are searched.
constexpr int kMoveMapTags = 1 << 16;
constexpr int kMoveMapWords = kMoveMapTags / 32;  // per field
struct MoveTables {
    const int* mv_start;      // [K]
    const int* mv_count;      // [K]
    const int* mv_label;      // [M]
    int M;
    const uint32_t* mv_map;   // [K][kMoveMapWords]
};

#ifdef __CUDACC__
// Index of label l among field f's moving drops, or -1.
__device__ __forceinline__ int moving_index(const MoveTables& mt, int f, int l) {
    int lo = mt.mv_start[f], n = mt.mv_count[f];
    int a = 0, b = n - 1;
    while (a <= b) {
        int mid = (a + b) >> 1;
        int v = mt.mv_label[lo + mid];
        if (v == l) return lo + mid;
        if (v < l) a = mid + 1;
        else b = mid - 1;
    }
    return -1;
}

// Is tag l (> 0) of field f a moving drop?
__device__ __forceinline__ bool is_moving(const MoveTables& mt, int f, int l) {
    if (l <= 0) return false;
    if (l < kMoveMapTags) return (mt.mv_map[(size_t)f * kMoveMapWords + (l >> 5)] >> (l & 31)) & 1u;
    return moving_index(mt, f, l) >= 0;
}
#endif
// Moving-drop bits (mvbits: a plane per field of mv_fields), then touch[m]
// and conflict[m] for every moving drop; dil: scratch of n_active +
// 2 n_mv_fields bit planes; reach <= 16, n_active and n_mv_fields <= 32.
cudaError_t recolour_touch(const int* labels, const uint32_t* bits, uint32_t* mvbits, uint32_t* dil, const Dims& g,
                           int n_active, int reach, MoveTables mt, const int* mv_fields, int n_mv_fields,
                           unsigned* touch, unsigned* conflict, int Mw, cudaStream_t st, long long* launches);
// The bit map of moving tags (mt.mv_map, cleared by the caller) for the
// n_fields fields listed in mv_fields.
cudaError_t move_map(MoveTables mt, uint32_t* map, const int* mv_fields, int n_fields, cudaStream_t st);
// Moves the cells set in mvbits to their drop's target field.
cudaError_t recolour_move(void* c, bool fp64, const int* labels, const uint32_t* mvbits, const Dims& g,
                          MoveTables mt, const int* mv_fields, int n_mv_fields, const int* target, cudaStream_t st);

// Statistics helpers.
// Per tag l <= n_max: the sum of c and its first moments about the tag's
// root cell root_of[l - 1] (minimum image), into S[4 (l - 1) ..].
cudaError_t drop_sums(const void* cf, bool fp64, const int* label_f, const int* root_of, const Dims& g,
                      double* S, int n_max, cudaStream_t st);
cudaError_t drop_finalize(const double* S, const int* root_of, const Dims& g, double h, int n,
                          double* vol, double* cen, cudaStream_t st);
// Height-function curvature of one field (NaN where a cell has none) and
// the surface-tension source f[3][N] = sum over K fields of gamma kappa grad c
// on the low faces (Section 2.3).
cudaError_t curvature_field(bool fp64, const void* cf, const Dims& g, double h, void* kappa, cudaStream_t st);
cudaError_t surface_tension(bool fp64, const void* c, const void* kappa, int K, const Dims& g, double h,
                            double gamma, void* f, cudaStream_t st);
// Drop shape (Appendix A): I[n][6] = xx yy zz xy xz yz about cen (cleared
// first), then chi = sqrt(I_max / I_min) per drop (chi may be null) with
// acc[0] += sum chi, acc[1] += drops, acc[2] = max(acc[2], chi) (acc may be
// null).
cudaError_t drop_inertia(const void* cf, bool fp64, const int* label_f, const Dims& g, double h, const double* cen,
                         int n, double* I, cudaStream_t st);
cudaError_t drop_chi(const double* I, int n, double* chi, double* acc, cudaStream_t st);
cudaError_t pair_stats(const double* cen, long long n, double bx, double by, double bz, int vaxis,
                       int n_rbins, double dr, int n_tbins, double dtheta, double tie_tol, double* hist_r,
                       double* hist_rt, double* moments, cudaStream_t st);

// Learned normal estimator.
struct MlpBlob;
cudaError_t mlp_forward(const MlpBlob* w, const float* st, float* n_out, long long n, int* status,
                        cudaStream_t stream);
cudaError_t mlp_grad_pass(const MlpBlob* w, const float* st, const float* tgt, long long n0, long long n,
                          float inv_batch, float* grad, float* loss_sum, int* status, cudaStream_t stream);
cudaError_t tc_gemm_check(const float* A, const float* B, float* D, int K, int N, int swap, int* status,
                          cudaStream_t st);

// PLIC primitives and normals (tests and tools).
cudaError_t plic_volume_batch(bool fp64, const void* m, const void* alpha, void* v, long long n,
                              cudaStream_t st);
cudaError_t plic_alpha_batch(bool fp64, const void* m, const void* c, void* alpha, long long n,
                             double band, cudaStream_t st);
cudaError_t normals_field(bool fp64, const void* cf, const Dims& g, void* m, cudaStream_t st);
cudaError_t velocity_scan(bool fp64, const void* u, long long n, double* out2, cudaStream_t st);

}  // namespace vof
