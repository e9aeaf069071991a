// C ABI entry points of libvof.so (declared in include/vof.h): argument
// validation, workspace layout and host-side orchestration of the kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "advect_impl.cuh"
#include "internal.h"

using namespace vof;

namespace {

enum Slot {
    S_BUF1,
    S_BUF2,
    S_FLUX,
    S_LIST,
    S_COUNTS,
    S_MISC,
    S_BITS,
    S_CCBITS,
    S_NCMAP,
    S_MVBITS,
    S_DIL,
    S_LABELS,
    S_PARENT,
    S_RANK,
    S_BTOT,
    S_BOFF,
    S_PTABLE,
    S_PLIST,
    S_MV,
    S_MVMAP,
    S_TOUCH,
    S_CONFLICT,
    S_TARGET,
    S_DSUM,
    S_CEN,
    S_VOL,
    S_ROOT,
    S_HIST_R,
    S_HIST_RT,
    S_MOM,
    S_SHAPE,
    S_NET,
    S_TILESEG,
    S_COUNT
};

// MISC slot layout (bytes): counters[8] u64 | flags[16] int | clipped[16] double |
// overflow int | n_out[16] int | vscan[2] u64 | learned-normal status int, face counters[3] u64
constexpr size_t kMiscCounters = 0;
constexpr size_t kMiscFlags = 64;
constexpr size_t kMiscClipped = 128;
constexpr size_t kMiscOverflow = 256;
constexpr size_t kMiscNout = 320;
constexpr size_t kMiscVscan = 448;
constexpr size_t kMiscMlpStatus = 512;
constexpr size_t kMiscMlpCounters = 576;
constexpr size_t kMiscBytes = 640;
constexpr int kMaxK = 16;
constexpr int kMoveWords = (kMoveCap + 31) / 32;

struct Layout {
    size_t off[S_COUNT];
    size_t size[S_COUNT];
    size_t total;
};

bool config_valid(const vof_config* c) {
    if (!c) return false;
    if (c->nx < 1 || c->ny < 1 || c->nz < 1) return false;
    if (c->nx >= (1 << 18) || c->ny >= (1 << 18) || c->nz >= (1 << 18)) return false;
    long long N = (long long)c->nx * c->ny * c->nz;
    if (N >= (1ll << 31)) return false;
    if (c->k_capacity < 1 || c->k_capacity > kMaxK) return false;
    if (c->k_active < 1 || c->k_active > c->k_capacity) return false;
    if (c->precision < VOF_FP64 || c->precision > VOF_MIXED_LEARNED) return false;
    if (!(c->h > 0.0) || !std::isfinite(c->h)) return false;
    if (c->stencil_w < 1 || c->stencil_w > 7) return false;
    if (c->connectivity != 6 && c->connectivity != 26) return false;
    if (!(c->tag_tau >= 0.0 && c->tag_tau < 1.0)) return false;
    if (!(c->alpha_fp64_band >= 0.0 && c->alpha_fp64_band < 0.5)) return false;
    if (c->vertical_axis < 0 || c->vertical_axis > 2) return false;
    if (c->stats_rbins < 1 || c->stats_rbins > (1 << 20)) return false;
    if (c->stats_tbins < 1 || c->stats_tbins > 4096) return false;
    if (!(c->stats_dr > 0.0)) return false;
    if (c->stats_every < 0) return false;
    return true;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Tiles of a face list at its largest (the list's reserved span).
size_t list_entries_for(const vof_config* c) {
    return (size_t)list_reserve(c->nx, c->ny, c->nz, c->k_capacity, c->precision == VOF_FP64 ? 8 : 4);
}
size_t tile_cap_for(const vof_config* c) { return (list_entries_for(c) + kFaceTile - 1) / kFaceTile; }

Layout layout_for(const vof_config* c) {
    Layout L;
    Dims g = make_dims(c->nx, c->ny, c->nz);
    size_t K = (size_t)c->k_capacity, N = (size_t)g.N;
    size_t es = c->precision == VOF_FP64 ? 8 : 4;
    size_t words = (size_t)g.rows * g.W;
    size_t nb = (N + 1023) / 1024;
    L.size[S_BUF1] = K * N * es;
    L.size[S_BUF2] = K * N * es;
    L.size[S_FLUX] = K * N * es;
    // two face lists segmented by block; a segment holds up to 2 faces per
    // cell and field of the block's cells, for any grid the advance picks
    L.size[S_LIST] = 2 * list_entries_for(c) * 8;
    L.size[S_COUNTS] = (3 * (size_t)kSweepBlocks + 1) * 4;
    L.size[S_MISC] = kMiscBytes;
    L.size[S_BITS] = K * words * 4;
    L.size[S_CCBITS] = K * words * 4;
    L.size[S_NCMAP] = K * words * 4;
    L.size[S_MVBITS] = K * words * 4;
    // Step 4: the active fields' and the moving drops' bits dilated, plus scratch
    L.size[S_DIL] = 3 * K * words * 4;
    L.size[S_LABELS] = K * N * 4;
    // labelling scratch, one set per field (Step 2 tags the flagged fields together)
    L.size[S_PARENT] = K * N * 4;
    L.size[S_RANK] = K * N * 4;
    L.size[S_BTOT] = K * (nb + 1) * 4;
    L.size[S_BOFF] = K * (nb + 1) * 4;
    L.size[S_PTABLE] = (size_t)kPairCap * 8;
    L.size[S_PLIST] = (size_t)kPairCap * 8;
    L.size[S_MV] = (size_t)(3 * kMaxK + kMoveCap) * 4;
    L.size[S_MVMAP] = K * (size_t)kMoveMapWords * 4;
    L.size[S_TOUCH] = (size_t)kMoveCap * 4;
    L.size[S_CONFLICT] = (size_t)kMoveCap * kMoveWords * 4;
    L.size[S_TARGET] = (size_t)kMoveCap * 4;
    L.size[S_DSUM] = (size_t)kDropCap * 4 * 8;
    L.size[S_CEN] = (size_t)kDropCap * 3 * 8;
    L.size[S_VOL] = (size_t)kDropCap * 8;
    L.size[S_ROOT] = (size_t)kDropCap * 4;
    L.size[S_HIST_R] = (size_t)(c->stats_rbins + 1) * 8;
    L.size[S_HIST_RT] = (size_t)(c->stats_rbins + 1) * c->stats_tbins * 8;
    L.size[S_MOM] = 16 * 8;
    // per-drop inertia tensor (6) and aspect ratio (1) for the statistics
    L.size[S_SHAPE] = (size_t)kDropCap * 7 * 8;
    // network normal at the cell of every listed face (learned normal only)
    L.size[S_NET] = c->precision == VOF_MIXED_LEARNED ? K * N * 16 : 0;
    // first segment of each tile of kFaceTile entries of a face list
    L.size[S_TILESEG] = (tile_cap_for(c) + 1) * 4;
    size_t o = 0;
    for (int s = 0; s < S_COUNT; ++s) {
        L.off[s] = o;
        o = align256(o + L.size[s]);
    }
    L.total = o;
    return L;
}

}  // namespace

static_assert(kMaxK <= kLabelSlots, "Step 2 tags every flagged field in one chain of launches");

struct vof_ctx {
    vof_config cfg;
    Dims g;
    bool fp64;
    size_t es;
    void* c;
    void* cur;        // buffer holding the state (always c between calls)
    bool bits_valid;  // occupancy bits of the active fields match c
    const void* u;
    char* ws;
    Layout L;
    cudaStream_t stream;
    int n_active;
    int n_in_use = -1;  // fields holding a drop at the last Step 1 (-1: not measured)
    long long step;
    double umax;
    vof_status sticky;
    long long launches;
    Prof prof;
    const void* mlp;  // borrowed weight blob of the learned normal (VOF_MIXED_LEARNED)
    double mlp_tol;
    template <typename P>
    P* slot(int s) const { return (P*)(ws + L.off[s]); }
    char* misc() const { return ws + L.off[S_MISC]; }
};

namespace {

vof_status cuda_fail(vof_ctx* ctx) {
    if (ctx) ctx->sticky = VOF_ERR_CUDA;
    return VOF_ERR_CUDA;
}

#define VOF_CUDA(ctx, expr)                       \
    do {                                          \
        const cudaError_t e_ = (expr);            \
        if (e_ != cudaSuccess) {                  \
            note_cuda_error(e_);                  \
            (void)cudaGetLastError();             \
            return cuda_fail(ctx);                \
        }                                         \
    } while (0)

// Bracket one launcher call with the context's launch timer.
template <typename F>
cudaError_t timed(vof_ctx* ctx, int cls, F&& f) {
    ctx->prof.begin(cls);
    cudaError_t e = f();
    ctx->prof.end();
    return e;
}

// Threshold for the occupancy test c > tau that, applied to the stored
// element type, decides exactly as the comparison in double would: for float
// storage, the largest float not above tau.
double occupancy_tau(const vof_ctx* ctx) {
    double tau = ctx->cfg.tag_tau;
    if (ctx->fp64) return tau;
    float tf = (float)tau;
    if ((double)tf > tau) tf = nextafterf(tf, -1.0f);
    return (double)tf;
}

vof_status check_ctx(vof_ctx* ctx) {
    if (!ctx) return VOF_ERR_ARG;
    return ctx->sticky;
}

vof_status scan_velocity(vof_ctx* ctx) {
    double* vs = (double*)(ctx->misc() + kMiscVscan);
    VOF_CUDA(ctx, velocity_scan(ctx->fp64, ctx->u, 3ll * ctx->g.N, vs, ctx->stream));
    ctx->launches += 1;
    unsigned long long host[2];
    VOF_CUDA(ctx, cudaMemcpyAsync(host, vs, sizeof(host), cudaMemcpyDeviceToHost, ctx->stream));
    VOF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (host[1]) return VOF_ERR_NONFINITE;
    double mx;
    std::memcpy(&mx, &host[0], sizeof(double));
    ctx->umax = mx;
    return VOF_OK;
}

// The context's state as a one-box set.
template <typename T>
static BoxSet<T, 1> ctx_box_set(vof_ctx* ctx, double* clipped, double dt) {
    BoxSet<T, 1> S;
    BoxDev<T>& B = S.b[0];
    const Dims& g = ctx->g;
    const int CH = 32 * VecOf<T>::W;
    B.g = g;
    B.K = ctx->n_active;
    B.item0 = 0;
    B.chunk0 = 0;
    B.cpr = (g.nx + CH - 1) / CH;
    B.divK = fastdiv_make((uint32_t)B.K);
    B.divcpr = fastdiv_make((uint32_t)B.cpr);
    B.divny = fastdiv_make((uint32_t)g.ny);
    B.sfac = (T)(dt / ctx->cfg.h);
    B.c = (T*)ctx->c;
    B.b1 = ctx->slot<T>(S_BUF1);
    B.b2 = ctx->slot<T>(S_BUF2);
    B.flux = ctx->slot<T>(S_FLUX);
    B.u = (const T*)ctx->u;
    B.net = ctx->cfg.precision == VOF_MIXED_LEARNED ? ctx->slot<float4>(S_NET) : nullptr;
    B.ccbits = ctx->slot<uint32_t>(S_CCBITS);
    B.occbits = ctx->slot<uint32_t>(S_BITS);
    B.clipped = clipped;
    S.n = 1;
    S.items = B.K * g.rows * B.cpr;
    S.chunks = g.rows * B.cpr;
    return S;
}

// Steps 1-4 on the current state (see vof_recolour).  patch (inside
// vof_step): the sweep arguments whose current face list is rewritten for
// the moved drops instead of being listed again.
vof_status recolour_impl(vof_ctx* ctx, int* moved_out, int* fired_out, SweepArgs* patch = nullptr,
                         double dt = 0.0) {
    const Dims& g = ctx->g;
    const vof_config& cf = ctx->cfg;
    cudaStream_t st = ctx->stream;
    int K = cf.k_capacity;
    int na0 = ctx->n_active;
    size_t words = (size_t)g.rows * g.W;
    uint32_t* bits = ctx->slot<uint32_t>(S_BITS);
    uint32_t* ncmap = ctx->slot<uint32_t>(S_NCMAP);
    int* flags = (int*)(ctx->misc() + kMiscFlags);
    *moved_out = 0;
    if (fired_out) *fired_out = 0;

    // Step 1 on the snapshot
    if (!ctx->bits_valid) {
        VOF_CUDA(ctx, timed(ctx, P_PACK_BITS, [&] { return pack_bits(ctx->cur, ctx->fp64, bits, g, na0, occupancy_tau(ctx), st); }));
        ctx->launches += 1;
    }
    if (na0 < K) VOF_CUDA(ctx, cudaMemsetAsync(bits + (size_t)na0 * words, 0, (size_t)(K - na0) * words * 4, st));
    VOF_CUDA(ctx, cudaMemsetAsync(flags, 0, kMaxK * sizeof(int), st));
    VOF_CUDA(ctx, timed(ctx, P_NEAR_CONTACT, [&] {
                 return near_contact(bits, ncmap, flags, g, na0, cf.stencil_w, st);
             }));
    ctx->launches += 1;
    int hflags[kMaxK];
    VOF_CUDA(ctx, cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
    VOF_CUDA(ctx, cudaStreamSynchronize(st));
    std::vector<int> flagged;
    int in_use = 0;
    for (int f = 0; f < na0; ++f) {
        if (hflags[f] & 1) flagged.push_back(f);
        in_use += (hflags[f] & 2) ? 1 : 0;
    }
    ctx->n_in_use = in_use;
    if (flagged.empty()) return VOF_OK;
    if (fired_out) *fired_out = 1;

    // Step 2: tag the flagged fields; Step 3: tagged pairs
    int* labels = ctx->slot<int>(S_LABELS);
    unsigned long long* table = ctx->slot<unsigned long long>(S_PTABLE);
    unsigned long long* plist = ctx->slot<unsigned long long>(S_PLIST);
    unsigned long long* counters = (unsigned long long*)(ctx->misc() + kMiscCounters);
    int* overflow = (int*)(ctx->misc() + kMiscOverflow);
    int* nout = (int*)(ctx->misc() + kMiscNout);
    VOF_CUDA(ctx, cudaMemsetAsync(table, 0xff, (size_t)kPairCap * 8, st));
    VOF_CUDA(ctx, cudaMemsetAsync(overflow, 0, sizeof(int), st));
    VOF_CUDA(ctx, cudaMemsetAsync(counters + 1, 0, sizeof(unsigned long long), st));
    // the flagged fields are tagged (and their pairs inserted) together: one
    // chain of launches whose blocks take a field each (blockIdx.y), with a
    // labelling scratch set per flagged field
    LabelSlots ls{};
    ls.n = (int)flagged.size();
    for (int i = 0; i < ls.n; ++i) ls.f[i] = flagged[i];
    VOF_CUDA(ctx, timed(ctx, P_LABEL, [&]() -> cudaError_t {
                 cudaError_t e = label_fields(bits, g, cf.connectivity, ls, ctx->slot<int>(S_PARENT),
                                              ctx->slot<int>(S_RANK), ctx->slot<int>(S_BTOT),
                                              ctx->slot<int>(S_BOFF), labels, nout, st, &ctx->launches);
                 if (e == cudaSuccess)
                     e = tag_pairs_fields(ncmap, bits, labels, g, cf.stencil_w, ls, table, kPairCap, overflow, st);
                 ctx->launches += 1;
                 return e;
             }));
    VOF_CUDA(ctx, timed(ctx, P_PAIRS, [&] { return compact_pairs(table, kPairCap, plist, counters + 1, st); }));
    ctx->launches += 1;
    // the pair count, the overflow flag and the first kFastPairs keys come
    // back with one synchronisation (the rest, rarely, with a second)
    constexpr size_t kFastPairs = 1024;
    unsigned long long npairs = 0;
    int hover = 0;
    std::vector<unsigned long long> keys(kFastPairs);
    VOF_CUDA(ctx, cudaMemcpyAsync(&npairs, counters + 1, 8, cudaMemcpyDeviceToHost, st));
    VOF_CUDA(ctx, cudaMemcpyAsync(&hover, overflow, 4, cudaMemcpyDeviceToHost, st));
    VOF_CUDA(ctx, cudaMemcpyAsync(keys.data(), plist, kFastPairs * 8, cudaMemcpyDeviceToHost, st));
    VOF_CUDA(ctx, cudaStreamSynchronize(st));
    if (hover) return VOF_ERR_CAPACITY;
    if (npairs == 0) return VOF_OK;
    keys.resize(npairs);
    if (npairs > kFastPairs) {
        VOF_CUDA(ctx, cudaMemcpyAsync(keys.data() + kFastPairs, plist + kFastPairs, (npairs - kFastPairs) * 8,
                                      cudaMemcpyDeviceToHost, st));
        VOF_CUDA(ctx, cudaStreamSynchronize(st));
    }
    std::sort(keys.begin(), keys.end());

    // moving drops per field: pairs (a < b) in order mark b unless a or b moves
    std::vector<std::vector<int>> moving(K);
    {
        size_t p = 0;
        while (p < keys.size()) {
            int f = (int)(keys[p] >> 60);
            std::vector<int> mv;  // sorted insertion not needed for membership tests
            std::vector<char> seen;
            size_t q = p;
            while (q < keys.size() && (int)(keys[q] >> 60) == f) ++q;
            int maxl = 0;
            for (size_t r = p; r < q; ++r) maxl = std::max(maxl, (int)(keys[r] & 0x3fffffffull));
            seen.assign((size_t)maxl + 1, 0);
            for (size_t r = p; r < q; ++r) {
                int a = (int)((keys[r] >> 30) & 0x3fffffffull), b = (int)(keys[r] & 0x3fffffffull);
                if (!seen[a] && !seen[b]) seen[b] = 1;
            }
            for (int l = 1; l <= maxl; ++l)
                if (seen[l]) moving[f].push_back(l);
            p = q;
        }
    }
    std::vector<int> hstart(kMaxK, 0), hcount(kMaxK, 0), hlabel, hfields, mfield;
    for (int f = 0; f < K; ++f) {
        hstart[f] = (int)hlabel.size();
        hcount[f] = (int)moving[f].size();
        for (int l : moving[f]) {
            hlabel.push_back(l);
            mfield.push_back(f);
        }
        if (!moving[f].empty()) hfields.push_back(f);
    }
    int M = (int)hlabel.size();
    if (M == 0) return VOF_OK;
    if (M > kMoveCap) return VOF_ERR_CAPACITY;
    int* mv = ctx->slot<int>(S_MV);
    int* d_start = mv;
    int* d_count = mv + kMaxK;
    int* d_fields = mv + 2 * kMaxK;
    int* d_label = mv + 3 * kMaxK;
    VOF_CUDA(ctx, cudaMemcpyAsync(d_start, hstart.data(), kMaxK * 4, cudaMemcpyHostToDevice, st));
    VOF_CUDA(ctx, cudaMemcpyAsync(d_count, hcount.data(), kMaxK * 4, cudaMemcpyHostToDevice, st));
    VOF_CUDA(ctx, cudaMemcpyAsync(d_fields, hfields.data(), hfields.size() * 4, cudaMemcpyHostToDevice, st));
    VOF_CUDA(ctx, cudaMemcpyAsync(d_label, hlabel.data(), (size_t)M * 4, cudaMemcpyHostToDevice, st));
    uint32_t* mv_map = ctx->slot<uint32_t>(S_MVMAP);
    MoveTables mt{d_start, d_count, d_label, M, mv_map};
    VOF_CUDA(ctx, cudaMemsetAsync(mv_map, 0, ctx->L.size[S_MVMAP], st));
    VOF_CUDA(ctx, move_map(mt, mv_map, d_fields, (int)hfields.size(), st));
    ctx->launches += 1;
    unsigned* touch = ctx->slot<unsigned>(S_TOUCH);
    unsigned* conflict = ctx->slot<unsigned>(S_CONFLICT);
    VOF_CUDA(ctx, cudaMemsetAsync(touch, 0, (size_t)M * 4, st));
    VOF_CUDA(ctx, cudaMemsetAsync(conflict, 0, (size_t)M * kMoveWords * 4, st));
    VOF_CUDA(ctx, timed(ctx, P_TOUCH, [&] {
                 return recolour_touch(labels, bits, ctx->slot<uint32_t>(S_MVBITS), ctx->slot<uint32_t>(S_DIL), g,
                                       na0, 2 * cf.stencil_w, mt, d_fields, (int)hfields.size(), touch, conflict,
                                       kMoveWords, st, &ctx->launches);
             }));
    std::vector<unsigned> htouch(M), hconf((size_t)M * kMoveWords);
    VOF_CUDA(ctx, cudaMemcpyAsync(htouch.data(), touch, (size_t)M * 4, cudaMemcpyDeviceToHost, st));
    VOF_CUDA(ctx, cudaMemcpyAsync(hconf.data(), conflict, (size_t)M * kMoveWords * 4, cudaMemcpyDeviceToHost, st));
    VOF_CUDA(ctx, cudaStreamSynchronize(st));

    // Step 4 greedy in (field, label) order
    std::vector<int> target(M, -1);
    vof_status status = VOF_OK;
    int moved = 0;
    for (int m = 0; m < M; ++m) {
        int f = mfield[m];
        int tg = -1;
        for (int n = 0; n < ctx->n_active && tg < 0; ++n) {
            if (n == f) continue;
            if ((htouch[m] >> n) & 1u) continue;
            bool clash = false;
            for (int q = 0; q < m && !clash; ++q)
                if (target[q] == n && ((hconf[(size_t)q * kMoveWords + (m >> 5)] >> (m & 31)) & 1u)) clash = true;
            if (!clash) tg = n;
        }
        if (tg < 0) {
            if (ctx->n_active < K) {
                tg = ctx->n_active++;
            } else {
                status = VOF_ERR_NO_FREE_FIELD;
                continue;
            }
        }
        target[m] = tg;
        ++moved;
    }
    int* d_target = ctx->slot<int>(S_TARGET);
    VOF_CUDA(ctx, cudaMemcpyAsync(d_target, target.data(), (size_t)M * 4, cudaMemcpyHostToDevice, st));
    VOF_CUDA(ctx, timed(ctx, P_MOVE, [&] {
                 return recolour_move(ctx->cur, ctx->fp64, labels, ctx->slot<uint32_t>(S_MVBITS), g, mt, d_fields,
                                     (int)hfields.size(), d_target, st);
             }));
    ctx->launches += 1;
    if (patch && moved > 0 && ctx->n_active != na0) {
        // a newly activated field changes the list's segment geometry (its
        // capacity per segment grows with the fields): list again
        patch->list_valid = false;
    } else if (patch && moved > 0) {
        // the list serves the first sweep of the next step
        double* clipped = (double*)(ctx->misc() + kMiscClipped);
        const int d = (int)(ctx->step % 3);
        VOF_CUDA(ctx, timed(ctx, P_FIND_FACES, [&] {
                     return ctx->fp64 ? patch_list_fp64(ctx_box_set<double>(ctx, clipped, dt), *patch, d, bits, labels,
                                                        mt, d_target)
                                      : patch_list_fp32(ctx_box_set<float>(ctx, clipped, dt), *patch, d, bits, labels,
                                                        mt, d_target);
                 }));
    }
    ctx->bits_valid = false;
    // vof_recolour returns with the work done; inside vof_step the next
    // step's launches follow on the same stream without a wait
    if (!patch) VOF_CUDA(ctx, cudaStreamSynchronize(st));
    *moved_out = moved;
    return status;
}

// One statistics event (Section 3) of every active field into the context's
// accumulators: tags, drop volumes and centroids, the drops' inertia
// tensors and aspect ratios (Appendix A; sum, count and maximum of chi in
// the moments slot), then the nearest-particle histograms and moments.
// Synchronises.  *D_out / *vtot_out: drops and their total volume.
vof_status stats_accumulate(vof_ctx* ctx, long long* D_out, double* vtot_out) {
    const Dims& g = ctx->g;
    const vof_config& cf = ctx->cfg;
    cudaStream_t st = ctx->stream;
    size_t words = (size_t)g.rows * g.W;
    double* hr = ctx->slot<double>(S_HIST_R);
    double* hrt = ctx->slot<double>(S_HIST_RT);
    double* mom = ctx->slot<double>(S_MOM);
    uint32_t* bits = ctx->slot<uint32_t>(S_BITS);
    int* labels = ctx->slot<int>(S_LABELS);
    int* nout = (int*)(ctx->misc() + kMiscNout);
    double* S = ctx->slot<double>(S_DSUM);
    double* cen = ctx->slot<double>(S_CEN);
    double* vol = ctx->slot<double>(S_VOL);
    double* shape = ctx->slot<double>(S_SHAPE);  // [D][6] tensors, then [D] chi
    int* root = ctx->slot<int>(S_ROOT);
    VOF_CUDA(ctx, pack_bits(ctx->c, ctx->fp64, bits, g, ctx->n_active, occupancy_tau(ctx), st));
    ctx->launches += 1;
    long long D = 0;
    for (int f = 0; f < ctx->n_active; ++f) {
        const char* cfp = (const char*)ctx->c + (size_t)f * g.N * ctx->es;
        int* lab = labels + (size_t)f * g.N;
        VOF_CUDA(ctx, label_field(bits + (size_t)f * words, g, cf.connectivity, ctx->slot<int>(S_PARENT),
                                  ctx->slot<int>(S_RANK), ctx->slot<int>(S_BTOT), ctx->slot<int>(S_BOFF), lab,
                                  root + D, (int)(kDropCap - D), nout + f, st, &ctx->launches));
        int n = 0;
        VOF_CUDA(ctx, cudaMemcpyAsync(&n, nout + f, 4, cudaMemcpyDeviceToHost, st));
        VOF_CUDA(ctx, cudaStreamSynchronize(st));
        if (D + n > kDropCap) return VOF_ERR_CAPACITY;
        if (n > 0) {
            VOF_CUDA(ctx, cudaMemsetAsync(S + 4 * D, 0, (size_t)n * 4 * 8, st));
            VOF_CUDA(ctx, drop_sums(cfp, ctx->fp64, lab, root + D, g, S + 4 * D, n, st));
            VOF_CUDA(ctx, drop_finalize(S + 4 * D, root + D, g, cf.h, n, vol + D, cen + 3 * D, st));
            VOF_CUDA(ctx, drop_inertia(cfp, ctx->fp64, lab, g, cf.h, cen + 3 * D, n, shape + 6 * D, st));
            ctx->launches += 4;
        }
        D += n;
    }
    VOF_CUDA(ctx, drop_chi(shape, (int)D, shape + 6 * (size_t)kDropCap, mom + 13, st));
    std::vector<double> hvol((size_t)D);
    if (D) VOF_CUDA(ctx, cudaMemcpyAsync(hvol.data(), vol, (size_t)D * 8, cudaMemcpyDeviceToHost, st));
    VOF_CUDA(ctx, cudaStreamSynchronize(st));
    double vtot = 0.0;
    for (double v : hvol) vtot += v;
    double dd = D ? std::cbrt(6.0 * (vtot / (double)D) / M_PI) : 0.0;
    double Lx = g.nx * cf.h, Ly = g.ny * cf.h, Lz = g.nz * cf.h;
    VOF_CUDA(ctx, pair_stats(cen, D, Lx, Ly, Lz, cf.vertical_axis, cf.stats_rbins, cf.stats_dr, cf.stats_tbins,
                             M_PI / cf.stats_tbins, 1e-12 * dd, hr, hrt, mom, st));
    ctx->launches += 2;
    if (D_out) *D_out = D;
    if (vtot_out) *vtot_out = vtot;
    return VOF_OK;
}

}  // namespace

extern "C" {

vof_status vof_config_default(vof_config* cfg) {
    if (!cfg) return VOF_ERR_ARG;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->nx = cfg->ny = cfg->nz = 32;
    cfg->k_capacity = 1;
    cfg->k_active = 1;
    cfg->precision = VOF_FP64;
    cfg->h = 1.0;
    cfg->stencil_w = 2;
    cfg->connectivity = 6;
    cfg->tag_tau = 1e-6;
    cfg->alpha_fp64_band = 1e-3;
    cfg->recolour = 0;
    cfg->vertical_axis = 2;
    cfg->stats_rbins = 1024;
    cfg->stats_tbins = 150;
    cfg->stats_dr = 0.2;
    cfg->stats_every = 0;
    return VOF_OK;
}

size_t vof_workspace_size(const vof_config* cfg) {
    if (!config_valid(cfg)) return 0;
    return layout_for(cfg).total;
}

vof_status vof_init(const vof_config* cfg, void* c_dev, const void* u_dev, void* workspace_dev,
                    size_t workspace_bytes, void* stream, vof_ctx** out) {
    if (!out) return VOF_ERR_ARG;
    *out = nullptr;
    if (!config_valid(cfg) || !c_dev || !u_dev || !workspace_dev) return VOF_ERR_ARG;
    if (((uintptr_t)workspace_dev & 255) != 0) return VOF_ERR_ARG;
    Layout L = layout_for(cfg);
    if (workspace_bytes < L.total) return VOF_ERR_WORKSPACE;
    vof_ctx* ctx = new (std::nothrow) vof_ctx();
    if (!ctx) return VOF_ERR_ARG;
    ctx->cfg = *cfg;
    ctx->g = make_dims(cfg->nx, cfg->ny, cfg->nz);
    ctx->fp64 = cfg->precision == VOF_FP64;
    ctx->es = ctx->fp64 ? 8 : 4;
    ctx->c = c_dev;
    ctx->cur = c_dev;
    ctx->bits_valid = false;
    ctx->u = u_dev;
    ctx->ws = (char*)workspace_dev;
    ctx->L = L;
    ctx->stream = (cudaStream_t)stream;
    ctx->n_active = cfg->k_active;
    ctx->step = 0;
    ctx->sticky = VOF_OK;
    ctx->launches = 0;
    ctx->prof.st = ctx->stream;
    ctx->mlp = nullptr;
    ctx->mlp_tol = 1e-3;
    if (cudaMemsetAsync(ctx->ws + L.off[S_MISC], 0, kMiscBytes, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->ws + L.off[S_HIST_R], 0, L.size[S_HIST_R], ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->ws + L.off[S_HIST_RT], 0, L.size[S_HIST_RT], ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->ws + L.off[S_MOM], 0, L.size[S_MOM], ctx->stream) != cudaSuccess) {
        (void)cudaGetLastError();
        delete ctx;
        return VOF_ERR_CUDA;
    }
    vof_status s = scan_velocity(ctx);
    if (s != VOF_OK) {
        delete ctx;
        return s;
    }
    *out = ctx;
    return VOF_OK;
}

vof_status vof_set_velocity(vof_ctx* ctx, const void* u_dev) {
    vof_status s = check_ctx(ctx);
    if (s != VOF_OK) return s;
    if (!u_dev) return VOF_ERR_ARG;
    ctx->u = u_dev;
    return scan_velocity(ctx);
}

}  // extern "C"

extern "C" {

vof_status vof_set_mlp(vof_ctx* ctx, const void* weights_dev, double fallback_tol) {
    vof_status s = check_ctx(ctx);
    if (s != VOF_OK) return s;
    if (ctx->cfg.precision != VOF_MIXED_LEARNED || !weights_dev || ((uintptr_t)weights_dev & 15) != 0 ||
        !(fallback_tol >= 0.0) || !std::isfinite(fallback_tol))
        return VOF_ERR_ARG;
    ctx->mlp = weights_dev;
    ctx->mlp_tol = fallback_tol;
    return VOF_OK;
}

vof_status vof_step(vof_ctx* ctx, double dt, int32_t nsteps, vof_step_report* report) {
    vof_status s = check_ctx(ctx);
    if (s != VOF_OK) return s;
    if (!(dt >= 0.0) || !std::isfinite(dt) || nsteps < 0) return VOF_ERR_ARG;
    if (ctx->umax * dt / ctx->cfg.h > 0.5) return VOF_ERR_CFL;
    if (ctx->cfg.precision == VOF_MIXED_LEARNED && !ctx->mlp) return VOF_ERR_STATE;
    double* clipped = (double*)(ctx->misc() + kMiscClipped);
    unsigned long long* mlp_counters = (unsigned long long*)(ctx->misc() + kMiscMlpCounters);
    if (report) {
        VOF_CUDA(ctx, cudaMemsetAsync(clipped, 0, kMaxK * sizeof(double), ctx->stream));
        VOF_CUDA(ctx, cudaMemsetAsync(mlp_counters, 0, 3 * sizeof(unsigned long long), ctx->stream));
    }
    SweepArgs a;
    a.list = ctx->slot<unsigned long long>(S_LIST);
    a.list_entries = (long long)list_entries_for(&ctx->cfg);
    a.counts = ctx->slot<int>(S_COUNTS);
    a.offsets = ctx->slot<int>(S_COUNTS) + 2 * kSweepBlocks;
    a.tile_seg = ctx->slot<int>(S_TILESEG);
    a.tile_cap = (int)std::min<size_t>(tile_cap_for(&ctx->cfg), (size_t)INT32_MAX);
    a.tau = occupancy_tau(ctx);
    a.list_valid = false;
    a.list_cur = 0;
    a.band = ctx->cfg.alpha_fp64_band;
    a.stream = ctx->stream;
    a.launches = &ctx->launches;
    a.prof = &ctx->prof;
    a.mlp = (const MlpBlob*)ctx->mlp;
    a.mlp_tol = (float)ctx->mlp_tol;
    a.mlp_status = (int*)(ctx->misc() + kMiscMlpStatus);
    a.mlp_counters = mlp_counters;
    a.update_warps = 0;
    a.update_blocks_per_sm = 0;
    int moved_total = 0, fired_steps = 0, in_use_max = -1;
    long long field_steps = 0;
    vof_status result = VOF_OK;
    const int every = ctx->cfg.stats_every;
    for (int done = 0; done < nsteps;) {
        // one step at a time with Steps 1-4, and never past a sampling step
        int n = ctx->cfg.recolour ? 1 : nsteps - done;
        if (every > 0) n = std::min(n, every - (int)(ctx->step % every));
        a.step = ctx->step;
        field_steps += (long long)ctx->n_active * n;
        if (ctx->fp64) {
            const BoxSet<double, 1> S = ctx_box_set<double>(ctx, clipped, dt);
            VOF_CUDA(ctx, advect_set_fp64(S, a, n));
        } else {
            const BoxSet<float, 1> S = ctx_box_set<float>(ctx, clipped, dt);
            VOF_CUDA(ctx, advect_set_fp32(S, a, n));
        }
        ctx->bits_valid = true;
        ctx->step += n;
        if (ctx->cfg.recolour) {
            int moved = 0, fired = 0;
            // the face list of the next sweep is patched for moved drops
            vof_status r = recolour_impl(ctx, &moved, &fired, &a, dt);
            if (r != VOF_OK && r != VOF_ERR_NO_FREE_FIELD) return r;
            if (r == VOF_ERR_NO_FREE_FIELD) result = r;
            moved_total += moved;
            fired_steps += fired;
            in_use_max = std::max(in_use_max, ctx->n_in_use);
        }
        // statistics events every `every` steps (Section 3 samples them every
        // 10 steps), accumulated into the context's histograms and moments
        if (every > 0 && ctx->step % every == 0) {
            vof_status r = stats_accumulate(ctx, nullptr, nullptr);
            if (r != VOF_OK) return r;
        }
        done += n;
    }
    if (report) {
        double hc[kMaxK];
        unsigned long long hm[3];
        int mst = 0;
        VOF_CUDA(ctx, cudaMemcpyAsync(hc, clipped, sizeof(hc), cudaMemcpyDeviceToHost, ctx->stream));
        VOF_CUDA(ctx, cudaMemcpyAsync(hm, mlp_counters, sizeof(hm), cudaMemcpyDeviceToHost, ctx->stream));
        VOF_CUDA(ctx, cudaMemcpyAsync(&mst, a.mlp_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        VOF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (mst) return ctx->sticky = VOF_ERR_TIMEOUT;
        report->faces_network = (int64_t)hm[0];
        report->faces_myc = (int64_t)hm[1];
        report->faces_myc_judged = (int64_t)hm[2];
        double tot = 0.0;
        for (int f = 0; f < ctx->cfg.k_capacity; ++f) tot += hc[f];
        report->steps_done = ctx->step;
        report->clipped_volume = tot * ctx->cfg.h * ctx->cfg.h * ctx->cfg.h;
        report->n_active = ctx->n_active;
        report->n_moved = moved_total;
        report->near_contact_steps = fired_steps;
        report->field_steps = field_steps;
        report->n_in_use = ctx->cfg.recolour ? ctx->n_in_use : -1;
        report->n_in_use_max = in_use_max;
    }
    return result;
}

vof_status vof_near_contact(vof_ctx* ctx, int32_t* flags_host) {
    vof_status s = check_ctx(ctx);
    if (s != VOF_OK) return s;
    if (!flags_host) return VOF_ERR_ARG;
    const Dims& g = ctx->g;
    uint32_t* bits = ctx->slot<uint32_t>(S_BITS);
    int* flags = (int*)(ctx->misc() + kMiscFlags);
    VOF_CUDA(ctx, pack_bits(ctx->c, ctx->fp64, bits, g, ctx->n_active, occupancy_tau(ctx), ctx->stream));
    VOF_CUDA(ctx, cudaMemsetAsync(flags, 0, kMaxK * sizeof(int), ctx->stream));
    VOF_CUDA(ctx, near_contact(bits, ctx->slot<uint32_t>(S_NCMAP), flags, g, ctx->n_active, ctx->cfg.stencil_w,
                               ctx->stream));
    ctx->launches += 2;
    int h[kMaxK];
    VOF_CUDA(ctx, cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    VOF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int f = 0; f < ctx->cfg.k_capacity; ++f) flags_host[f] = f < ctx->n_active ? (h[f] & 1) : 0;
    return VOF_OK;
}

vof_status vof_label(vof_ctx* ctx, int32_t field, int32_t* label_dev, int32_t* n_drops_host) {
    vof_status s = check_ctx(ctx);
    if (s != VOF_OK) return s;
    if (field < 0 || field >= ctx->cfg.k_capacity || !label_dev || !n_drops_host) return VOF_ERR_ARG;
    const Dims& g = ctx->g;
    size_t words = (size_t)g.rows * g.W;
    uint32_t* bits = ctx->slot<uint32_t>(S_BITS);
    const char* cf = (const char*)ctx->c + (size_t)field * g.N * ctx->es;
    int* nout = (int*)(ctx->misc() + kMiscNout);
    VOF_CUDA(ctx, pack_bits(cf, ctx->fp64, bits + (size_t)field * words, g, 1, occupancy_tau(ctx), ctx->stream));
    ctx->launches += 1;
    VOF_CUDA(ctx, label_field(bits + (size_t)field * words, g, ctx->cfg.connectivity, ctx->slot<int>(S_PARENT),
                              ctx->slot<int>(S_RANK), ctx->slot<int>(S_BTOT), ctx->slot<int>(S_BOFF), label_dev,
                              nullptr, 0, nout + field, ctx->stream, &ctx->launches));
    int n = 0;
    VOF_CUDA(ctx, cudaMemcpyAsync(&n, nout + field, 4, cudaMemcpyDeviceToHost, ctx->stream));
    VOF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *n_drops_host = n;
    return VOF_OK;
}

vof_status vof_recolour(vof_ctx* ctx, int32_t* n_moved, int32_t* n_active) {
    vof_status s = check_ctx(ctx);
    if (s != VOF_OK) return s;
    int moved = 0;
    vof_status r = recolour_impl(ctx, &moved, nullptr);
    if (n_moved) *n_moved = moved;
    if (n_active) *n_active = ctx->n_active;
    return r;
}

vof_status vof_drop_table(vof_ctx* ctx, int32_t field, const int32_t* label_dev, int32_t n_labels,
                          double* vol_dev, double* cen_dev) {
    vof_status s = check_ctx(ctx);
    if (s != VOF_OK) return s;
    if (field < 0 || field >= ctx->cfg.k_capacity || !label_dev || n_labels < 0 || n_labels > kDropCap ||
        (n_labels > 0 && (!vol_dev || !cen_dev)))
        return VOF_ERR_ARG;
    const Dims& g = ctx->g;
    size_t words = (size_t)g.rows * g.W;
    uint32_t* bits = ctx->slot<uint32_t>(S_BITS);
    const char* cf = (const char*)ctx->c + (size_t)field * g.N * ctx->es;
    int* nout = (int*)(ctx->misc() + kMiscNout);
    int* tmp_label = ctx->slot<int>(S_LABELS) + (size_t)field * g.N;
    // re-derive the roots (the caller's labels must be this field's tags)
    VOF_CUDA(ctx, pack_bits(cf, ctx->fp64, bits + (size_t)field * words, g, 1, occupancy_tau(ctx), ctx->stream));
    VOF_CUDA(ctx, label_field(bits + (size_t)field * words, g, ctx->cfg.connectivity, ctx->slot<int>(S_PARENT),
                              ctx->slot<int>(S_RANK), ctx->slot<int>(S_BTOT), ctx->slot<int>(S_BOFF), tmp_label,
                              ctx->slot<int>(S_ROOT), kDropCap, nout + field, ctx->stream, &ctx->launches));
    double* S = ctx->slot<double>(S_DSUM);
    VOF_CUDA(ctx, cudaMemsetAsync(S, 0, (size_t)n_labels * 4 * 8, ctx->stream));
    VOF_CUDA(ctx, drop_sums(cf, ctx->fp64, label_dev, ctx->slot<int>(S_ROOT), g, S, n_labels, ctx->stream));
    VOF_CUDA(ctx, drop_finalize(S, ctx->slot<int>(S_ROOT), g, ctx->cfg.h, n_labels, vol_dev, cen_dev, ctx->stream));
    ctx->launches += 3;
    return VOF_OK;
}

vof_status vof_stats(vof_ctx* ctx, int32_t reset, vof_stats_out* out, double* hist_r_host,
                     double* hist_rt_host) {
    vof_status s = check_ctx(ctx);
    if (s != VOF_OK) return s;
    if (!out) return VOF_ERR_ARG;
    const Dims& g = ctx->g;
    const vof_config& cf = ctx->cfg;
    cudaStream_t st = ctx->stream;
    double* hr = ctx->slot<double>(S_HIST_R);
    double* hrt = ctx->slot<double>(S_HIST_RT);
    double* mom = ctx->slot<double>(S_MOM);
    if (reset) {
        VOF_CUDA(ctx, cudaMemsetAsync(hr, 0, ctx->L.size[S_HIST_R], st));
        VOF_CUDA(ctx, cudaMemsetAsync(hrt, 0, ctx->L.size[S_HIST_RT], st));
        VOF_CUDA(ctx, cudaMemsetAsync(mom, 0, ctx->L.size[S_MOM], st));
    }
    long long D = 0;
    double vtot = 0.0;
    s = stats_accumulate(ctx, &D, &vtot);
    if (s != VOF_OK) return s;
    double dd = D ? std::cbrt(6.0 * (vtot / (double)D) / M_PI) : 0.0;
    double Lx = g.nx * cf.h, Ly = g.ny * cf.h, Lz = g.nz * cf.h;
    double hm[16];
    VOF_CUDA(ctx, cudaMemcpyAsync(hm, mom, sizeof(hm), cudaMemcpyDeviceToHost, st));
    if (hist_r_host) VOF_CUDA(ctx, cudaMemcpyAsync(hist_r_host, hr, ctx->L.size[S_HIST_R], cudaMemcpyDeviceToHost, st));
    if (hist_rt_host)
        VOF_CUDA(ctx, cudaMemcpyAsync(hist_rt_host, hrt, ctx->L.size[S_HIST_RT], cudaMemcpyDeviceToHost, st));
    VOF_CUDA(ctx, cudaStreamSynchronize(st));
    out->n_drops = (int32_t)D;
    out->d = dd;
    out->n_p = (double)D / (Lx * Ly * Lz);
    out->volume = vtot;
    out->events = hm[12];
    double E = hm[12] > 0 ? hm[12] : 1.0;
    for (int a = 0; a < 3; ++a) out->M[a] = hm[a] / E;
    for (int q = 0; q < 9; ++q) out->R[q] = hm[3 + q] / E;
    double tr = out->R[0] + out->R[4] + out->R[8];
    for (int q = 0; q < 9; ++q) out->A[q] = out->R[q] - ((q % 4 == 0) ? tr / 3.0 : 0.0);
    out->chi_drops = hm[14];
    out->chi_mean = hm[14] > 0 ? hm[13] / hm[14] : 0.0;
    out->chi_max = hm[15];
    return VOF_OK;
}

vof_status vof_curvature(vof_ctx* ctx, int32_t field, void* kappa_dev) {
    vof_status s = check_ctx(ctx);
    if (s != VOF_OK) return s;
    if (field < 0 || field >= ctx->cfg.k_capacity || !kappa_dev) return VOF_ERR_ARG;
    const char* cf = (const char*)ctx->c + (size_t)field * ctx->g.N * ctx->es;
    VOF_CUDA(ctx, timed(ctx, P_MISC, [&] {
        return curvature_field(ctx->fp64, cf, ctx->g, ctx->cfg.h, kappa_dev, ctx->stream);
    }));
    ctx->launches += 1;
    return VOF_OK;
}

vof_status vof_surface_tension(vof_ctx* ctx, double gamma, void* f_dev) {
    vof_status s = check_ctx(ctx);
    if (s != VOF_OK) return s;
    if (!f_dev || !std::isfinite(gamma)) return VOF_ERR_ARG;
    const Dims& g = ctx->g;
    // the flux buffer ([K][N], the state's element type) is free between
    // calls: it holds the curvature of every active field here
    char* kap = ctx->slot<char>(S_FLUX);
    for (int f = 0; f < ctx->n_active; ++f) {
        const char* cf = (const char*)ctx->c + (size_t)f * g.N * ctx->es;
        VOF_CUDA(ctx, timed(ctx, P_MISC, [&] {
            return curvature_field(ctx->fp64, cf, g, ctx->cfg.h, kap + (size_t)f * g.N * ctx->es, ctx->stream);
        }));
    }
    VOF_CUDA(ctx, timed(ctx, P_MISC, [&] {
        return surface_tension(ctx->fp64, ctx->c, kap, ctx->n_active, g, ctx->cfg.h, gamma, f_dev, ctx->stream);
    }));
    ctx->launches += ctx->n_active + 1;
    return VOF_OK;
}

vof_status vof_drop_shape(vof_ctx* ctx, int32_t field, const int32_t* label_dev, int32_t n_labels,
                          const double* cen_dev, double* inertia_dev, double* chi_dev) {
    vof_status s = check_ctx(ctx);
    if (s != VOF_OK) return s;
    if (field < 0 || field >= ctx->cfg.k_capacity || !label_dev || n_labels < 0 || n_labels > kDropCap ||
        (n_labels > 0 && (!cen_dev || !inertia_dev)))
        return VOF_ERR_ARG;
    const char* cf = (const char*)ctx->c + (size_t)field * ctx->g.N * ctx->es;
    VOF_CUDA(ctx, drop_inertia(cf, ctx->fp64, label_dev, ctx->g, ctx->cfg.h, cen_dev, n_labels, inertia_dev,
                               ctx->stream));
    VOF_CUDA(ctx, drop_chi(inertia_dev, n_labels, chi_dev, nullptr, ctx->stream));
    ctx->launches += 2;
    return VOF_OK;
}

vof_status vof_pair_stats(const double* cen_dev, int64_t n, const double* box_host, int32_t vertical_axis,
                          int32_t n_rbins, double dr, int32_t n_tbins, double dtheta, double tie_tol,
                          double* hist_r_dev, double* hist_rt_dev, double* moments_dev, void* stream) {
    if (n < 0 || (n > 0 && !cen_dev) || !box_host || vertical_axis < 0 || vertical_axis > 2 || n_rbins < 1 ||
        n_tbins < 1 || !(dr > 0) || !(dtheta > 0) || !(tie_tol >= 0) || !hist_r_dev || !hist_rt_dev || !moments_dev)
        return VOF_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!(box_host[a] > 0)) return VOF_ERR_ARG;
    if (pair_stats(cen_dev, n, box_host[0], box_host[1], box_host[2], vertical_axis, n_rbins, dr, n_tbins, dtheta,
                   tie_tol, hist_r_dev, hist_rt_dev, moments_dev, (cudaStream_t)stream) != cudaSuccess)
        return VOF_ERR_CUDA;
    return VOF_OK;
}

vof_status vof_plic_volume(int32_t precision, const void* m_dev, const void* alpha_dev, void* v_dev, int64_t n,
                           void* stream) {
    if (precision < VOF_FP64 || precision > VOF_MIXED_LEARNED || n < 0) return VOF_ERR_ARG;
    if (n > 0 && (!m_dev || !alpha_dev || !v_dev)) return VOF_ERR_ARG;
    if (plic_volume_batch(precision == VOF_FP64, m_dev, alpha_dev, v_dev, n, (cudaStream_t)stream) != cudaSuccess)
        return VOF_ERR_CUDA;
    return VOF_OK;
}

vof_status vof_plic_alpha(int32_t precision, const void* m_dev, const void* c_dev, void* alpha_dev, int64_t n,
                          double band, void* stream) {
    if (precision < VOF_FP64 || precision > VOF_MIXED_LEARNED || n < 0 || !(band >= 0 && band < 0.5))
        return VOF_ERR_ARG;
    if (n > 0 && (!m_dev || !c_dev || !alpha_dev)) return VOF_ERR_ARG;
    if (plic_alpha_batch(precision == VOF_FP64, m_dev, c_dev, alpha_dev, n, band, (cudaStream_t)stream) !=
        cudaSuccess)
        return VOF_ERR_CUDA;
    return VOF_OK;
}

vof_status vof_normals(vof_ctx* ctx, int32_t field, void* m_dev) {
    vof_status s = check_ctx(ctx);
    if (s != VOF_OK) return s;
    if (field < 0 || field >= ctx->cfg.k_capacity || !m_dev) return VOF_ERR_ARG;
    const char* cf = (const char*)ctx->c + (size_t)field * ctx->g.N * ctx->es;
    VOF_CUDA(ctx, normals_field(ctx->fp64, cf, ctx->g, m_dev, ctx->stream));
    ctx->launches += 1;
    return VOF_OK;
}

namespace {
struct StateHeader {
    char magic[8];
    int32_t version, nx, ny, nz, k_capacity, precision, n_active, stats_rbins, stats_tbins, pad;
    int64_t step;
};
}  // namespace

size_t vof_state_size(const vof_ctx* ctx) {
    if (!ctx) return 0;
    return sizeof(StateHeader) + (size_t)ctx->cfg.k_capacity * ctx->g.N * ctx->es + ctx->L.size[S_HIST_R] +
           ctx->L.size[S_HIST_RT] + ctx->L.size[S_MOM];
}

vof_status vof_get_state(vof_ctx* ctx, void* host_buf, size_t bytes) {
    vof_status s = check_ctx(ctx);
    if (s != VOF_OK) return s;
    if (!host_buf || bytes < vof_state_size(ctx)) return VOF_ERR_ARG;
    StateHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "VOFSTAT1", 8);
    h.version = 1;
    h.nx = ctx->cfg.nx;
    h.ny = ctx->cfg.ny;
    h.nz = ctx->cfg.nz;
    h.k_capacity = ctx->cfg.k_capacity;
    h.precision = ctx->cfg.precision;
    h.n_active = ctx->n_active;
    h.stats_rbins = ctx->cfg.stats_rbins;
    h.stats_tbins = ctx->cfg.stats_tbins;
    h.step = ctx->step;
    char* p = (char*)host_buf;
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    size_t cb = (size_t)ctx->cfg.k_capacity * ctx->g.N * ctx->es;
    VOF_CUDA(ctx, cudaMemcpyAsync(p, ctx->c, cb, cudaMemcpyDeviceToHost, ctx->stream));
    p += cb;
    const int slots[3] = {S_HIST_R, S_HIST_RT, S_MOM};
    for (int q = 0; q < 3; ++q) {
        VOF_CUDA(ctx, cudaMemcpyAsync(p, ctx->ws + ctx->L.off[slots[q]], ctx->L.size[slots[q]], cudaMemcpyDeviceToHost,
                                      ctx->stream));
        p += ctx->L.size[slots[q]];
    }
    VOF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return VOF_OK;
}

vof_status vof_set_state(vof_ctx* ctx, const void* host_buf, size_t bytes) {
    vof_status s = check_ctx(ctx);
    if (s != VOF_OK) return s;
    if (!host_buf || bytes < sizeof(StateHeader)) return VOF_ERR_ARG;
    StateHeader h;
    std::memcpy(&h, host_buf, sizeof(h));
    if (std::memcmp(h.magic, "VOFSTAT1", 8) != 0 || h.version != 1 || h.nx != ctx->cfg.nx || h.ny != ctx->cfg.ny ||
        h.nz != ctx->cfg.nz || h.k_capacity != ctx->cfg.k_capacity || h.precision != ctx->cfg.precision ||
        h.stats_rbins != ctx->cfg.stats_rbins || h.stats_tbins != ctx->cfg.stats_tbins || h.n_active < 1 ||
        h.n_active > ctx->cfg.k_capacity || bytes < vof_state_size(ctx))
        return VOF_ERR_STATE;
    const char* p = (const char*)host_buf + sizeof(h);
    size_t cb = (size_t)ctx->cfg.k_capacity * ctx->g.N * ctx->es;
    VOF_CUDA(ctx, cudaMemcpyAsync(ctx->c, p, cb, cudaMemcpyHostToDevice, ctx->stream));
    p += cb;
    const int slots[3] = {S_HIST_R, S_HIST_RT, S_MOM};
    for (int q = 0; q < 3; ++q) {
        VOF_CUDA(ctx, cudaMemcpyAsync(ctx->ws + ctx->L.off[slots[q]], p, ctx->L.size[slots[q]], cudaMemcpyHostToDevice,
                                      ctx->stream));
        p += ctx->L.size[slots[q]];
    }
    VOF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->n_active = h.n_active;
    ctx->step = h.step;
    ctx->bits_valid = false;
    return VOF_OK;
}

int64_t vof_launch_count(const vof_ctx* ctx) { return ctx ? ctx->launches : 0; }

const char* vof_status_string(vof_status s) {
    switch (s) {
        case VOF_OK: return "ok";
        case VOF_ERR_ARG: return "invalid argument";
        case VOF_ERR_CUDA: return "CUDA error";
        case VOF_ERR_WORKSPACE: return "workspace too small";
        case VOF_ERR_NO_FREE_FIELD: return "no free colour field";
        case VOF_ERR_CFL: return "CFL number above 1/2";
        case VOF_ERR_TIMEOUT: return "bounded device wait timed out";
        case VOF_ERR_STATE: return "state blob does not match the context";
        case VOF_ERR_NONFINITE: return "non-finite velocity";
        case VOF_ERR_CAPACITY: return "fixed-capacity list overflowed";
    }
    return "unknown status";
}

vof_status vof_profile_enable(vof_ctx* ctx, int32_t enable) {
    if (!ctx) return VOF_ERR_ARG;
    Prof& p = ctx->prof;
    if (enable && p.cap == 0) {
        const int cap = 16384;
        p.ev.resize(2 * (size_t)cap);
        for (auto& e : p.ev)
            if (cudaEventCreate(&e) != cudaSuccess) {
                (void)cudaGetLastError();
                return cuda_fail(ctx);
            }
        p.cls.assign(cap, 0);
        p.cap = cap;
    }
    p.on = enable != 0;
    return VOF_OK;
}

vof_status vof_profile_read(vof_ctx* ctx, int64_t* launches, double* ms, int32_t n) {
    if (!ctx || n < 0 || (n > 0 && (!launches || !ms))) return VOF_ERR_ARG;
    Prof& p = ctx->prof;
    for (int c = 0; c < n; ++c) {
        launches[c] = 0;
        ms[c] = 0.0;
    }
    VOF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int q = 0; q < p.n; ++q) {
        float t = 0.f;
        VOF_CUDA(ctx, cudaEventElapsedTime(&t, p.ev[2 * q], p.ev[2 * q + 1]));
        int c = p.cls[q];
        if (c < n) {
            launches[c] += 1;
            ms[c] += (double)t;
        }
    }
    p.n = 0;
    return VOF_OK;
}

const char* vof_last_cuda_error(void) { return vof::last_cuda_error_name(); }

const char* vof_profile_class_name(int32_t cls) {
    static const char* names[P_COUNT] = {"list_faces", "face_flux", "update", "pack_bits", "near_contact",
                                         "label",      "pairs",     "touch",  "move",      "stats",
                                         "misc",       "net_normals", "scan"};
    if (cls < 0 || cls >= P_COUNT) return nullptr;
    return names[cls];
}

void vof_destroy(vof_ctx* ctx) {
    if (!ctx) return;
    for (auto& e : ctx->prof.ev) cudaEventDestroy(e);
    delete ctx;
}

}  // extern "C"
