// Batched advance of many independent boxes (C ABI, declared in
// include/vof.h): every pass of a sweep is one launch over every field of
// every box (see boxes.cuh), a step is replayed from a captured CUDA graph,
// and the launch shape of the update pass is chosen at init by timing the
// candidates on the batch itself.
//
// The paper advances one box; batching independent boxes is a throughput
// device of this library: each box follows exactly the arithmetic of a
// single context (Section 2.2 split advection with the Weymouth & Yue term,
// the clip after the third sweep), so a box advanced in a batch equals the
// same box advanced alone.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "advect_impl.cuh"
#include "internal.h"

namespace {

using namespace vof;

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

bool fp64_batch(const vof_batch_config* c) { return c->precision == VOF_FP64; }

bool box_valid(const vof_box_desc& b, int es) {
    if (b.nx < 1 || b.ny < 1 || b.nz < 1) return false;
    if (b.nx >= (1 << 18) || b.ny >= (1 << 18) || b.nz >= (1 << 18)) return false;
    if ((long long)b.nx * b.ny * b.nz >= (1ll << 31)) return false;
    if (b.k_capacity < 1 || b.k_capacity > 16 || b.k_active < 1 || b.k_active > b.k_capacity) return false;
    if (b.nx % (16 / es) != 0) return false;  // whole 16-byte lanes per row
    if (!b.c_dev || !b.u_dev || ((uintptr_t)b.c_dev & 15) || ((uintptr_t)b.u_dev & 15)) return false;
    if (!(b.dt >= 0.0) || !std::isfinite(b.dt)) return false;
    return true;
}

bool batch_config_valid(const vof_batch_config* c) {
    if (!c) return false;
    if (c->precision < VOF_FP64 || c->precision > VOF_MIXED_LEARNED) return false;
    if (!(c->h > 0.0) || !std::isfinite(c->h)) return false;
    if (!(c->tag_tau >= 0.0 && c->tag_tau < 1.0)) return false;
    if (!(c->alpha_fp64_band >= 0.0 && c->alpha_fp64_band < 0.5)) return false;
    return true;
}

// Per-box slices and shared buffers of the batch workspace.
struct BatchLayout {
    std::vector<size_t> b1, b2, flux, net, ccbits, occbits;
    size_t clipped, list, counts, tile_seg, misc, vscan, total;
    long long list_entries, items;
    int tile_cap;
};

BatchLayout batch_layout(const vof_batch_config* cfg, const vof_box_desc* boxes, int n) {
    BatchLayout L;
    const size_t es = cfg->precision == VOF_FP64 ? 8 : 4;
    const int CH = (int)(512 / es);
    size_t o = 0;
    long long items = 0, chunks = 0, kmax = 1;
    for (int b = 0; b < n; ++b) {
        const vof_box_desc& d = boxes[b];
        const size_t N = (size_t)d.nx * d.ny * d.nz, K = (size_t)d.k_capacity;
        const size_t words = (size_t)d.ny * d.nz * ((d.nx + 31) / 32);
        L.b1.push_back(o), o = al256(o + K * N * es);
        L.b2.push_back(o), o = al256(o + K * N * es);
        L.flux.push_back(o), o = al256(o + K * N * es);
        L.net.push_back(o), o = al256(o + (cfg->precision == VOF_MIXED_LEARNED ? K * N * 16 : 0));
        L.ccbits.push_back(o), o = al256(o + K * words * 4);
        L.occbits.push_back(o), o = al256(o + K * words * 4);
        items += (long long)d.k_capacity * d.ny * d.nz * ((d.nx + CH - 1) / CH);
        chunks += (long long)d.ny * d.nz * ((d.nx + CH - 1) / CH);
        kmax = std::max<long long>(kmax, d.k_capacity);
    }
    L.items = items;
    // a warp of the update pass lists up to 2 faces per cell of every field
    // of each of its row chunks
    L.list_entries = 2LL * CH * kmax * (chunks + 8LL * kListBlocks);
    L.tile_cap = (int)std::min<long long>((L.list_entries + kFaceTile - 1) / kFaceTile, INT32_MAX);
    L.clipped = o, o = al256(o + (size_t)n * 16 * 8);
    L.list = o, o = al256(o + 2 * (size_t)L.list_entries * 8);
    L.counts = o, o = al256(o + (3 * (size_t)kSweepBlocks + 1) * 4);
    L.tile_seg = o, o = al256(o + ((size_t)L.tile_cap + 1) * 4);
    L.misc = o, o = al256(o + 64);  // [0] tensor-core status, [8..32) face counters
    L.vscan = o, o = al256(o + 16);
    L.total = o;
    return L;
}

}  // namespace

struct vof_batch {
    vof_batch_config cfg;
    std::vector<vof_box_desc> boxes;
    BatchLayout L;
    char* ws;
    cudaStream_t stream;
    long long step;
    bool list_valid;
    int list_cur;
    const void* mlp;
    double mlp_tol;
    int update_warps, update_blocks_per_sm;
    float tune_ms_best;
    int tune_candidates;
    cudaGraphExec_t graphs[3][2];  // by sweep rotation and current list
    cudaStream_t cap_stream;       // capture only (the caller's stream may be the legacy default one)
    long long graph_launches, direct_steps;
    vof_status sticky;
};

namespace {

template <typename T>
BoxSet<T, kMaxBoxes> batch_set(vof_batch* B) {
    BoxSet<T, kMaxBoxes> S;
    const int CH = 32 * VecOf<T>::W;
    int item = 0, chunk = 0;
    S.n = (int)B->boxes.size();
    for (int b = 0; b < S.n; ++b) {
        const vof_box_desc& d = B->boxes[b];
        BoxDev<T>& X = S.b[b];
        X.g = make_dims(d.nx, d.ny, d.nz);
        X.K = d.k_active;
        X.item0 = item;
        X.chunk0 = chunk;
        X.cpr = (d.nx + CH - 1) / CH;
        X.divK = fastdiv_make((uint32_t)X.K);
        X.divcpr = fastdiv_make((uint32_t)X.cpr);
        X.divny = fastdiv_make((uint32_t)d.ny);
        X.sfac = (T)(d.dt / B->cfg.h);
        X.c = (T*)d.c_dev;
        X.b1 = (T*)(B->ws + B->L.b1[b]);
        X.b2 = (T*)(B->ws + B->L.b2[b]);
        X.flux = (T*)(B->ws + B->L.flux[b]);
        X.u = (const T*)d.u_dev;
        X.net = B->cfg.precision == VOF_MIXED_LEARNED ? (float4*)(B->ws + B->L.net[b]) : nullptr;
        X.ccbits = (uint32_t*)(B->ws + B->L.ccbits[b]);
        X.occbits = (uint32_t*)(B->ws + B->L.occbits[b]);
        X.clipped = (double*)(B->ws + B->L.clipped) + 16 * b;
        item += X.K * X.g.rows * X.cpr;
        chunk += X.g.rows * X.cpr;
    }
    S.items = item;
    S.chunks = chunk;
    return S;
}

SweepArgs batch_args(vof_batch* B) {
    SweepArgs a;
    a.list = (unsigned long long*)(B->ws + B->L.list);
    a.list_entries = B->L.list_entries;
    a.counts = (int*)(B->ws + B->L.counts);
    a.offsets = a.counts + 2 * kSweepBlocks;
    a.tile_seg = (int*)(B->ws + B->L.tile_seg);
    a.tile_cap = B->L.tile_cap;
    a.step = B->step;
    a.band = B->cfg.alpha_fp64_band;
    // occupancy threshold as in a context: the largest value of the element
    // type that is <= tau (c > t in the element type iff c > tau)
    if (B->cfg.precision == VOF_FP64) {
        a.tau = B->cfg.tag_tau;
    } else {
        float t = (float)B->cfg.tag_tau;
        if ((double)t > B->cfg.tag_tau) t = std::nextafter(t, -1.0f);
        a.tau = (double)t;
    }
    a.list_valid = B->list_valid;
    a.list_cur = B->list_cur;
    a.stream = B->stream;
    a.launches = nullptr;
    a.prof = nullptr;
    a.mlp = (const MlpBlob*)B->mlp;
    a.mlp_tol = (float)B->mlp_tol;
    a.mlp_status = (int*)(B->ws + B->L.misc);
    a.mlp_counters = (unsigned long long*)(B->ws + B->L.misc + 8);
    a.update_warps = B->update_warps;
    a.update_blocks_per_sm = B->update_blocks_per_sm;
    return a;
}

cudaError_t advance(vof_batch* B, SweepArgs& a, int nsteps) {
    if (B->cfg.precision == VOF_FP64) return advect_set_fp64(batch_set<double>(B), a, nsteps);
    return advect_set_fp32(batch_set<float>(B), a, nsteps);
}

vof_status fail(vof_batch* B, vof_status s) {
    note_cuda_error(cudaGetLastError());
    if (B && (s == VOF_ERR_CUDA || s == VOF_ERR_TIMEOUT)) B->sticky = s;
    return s;
}

// One step replayed from the graph of (rotation, current list), captured on
// first use.  The graph holds every launch of the step; the box table is a
// kernel parameter, so nothing else has to stay alive.
cudaError_t graph_step(vof_batch* B) {
    const int rot = (int)(B->step % 3), cur = B->list_cur;
    cudaGraphExec_t& ex = B->graphs[rot][cur];
    if (!ex) {
        cudaGraph_t graph = nullptr;
        if (!B->cap_stream) {
            cudaError_t e = cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        SweepArgs a = batch_args(B);
        a.stream = B->cap_stream;
        cudaError_t e1 = advance(B, a, 1);
        cudaError_t e2 = cudaStreamEndCapture(B->cap_stream, &graph);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return e1 != cudaSuccess ? e1 : e2;
        }
        e = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            ex = nullptr;
            return e;
        }
    }
    cudaError_t e = cudaGraphLaunch(ex, B->stream);
    if (e != cudaSuccess) return e;
    B->graph_launches += 1;
    B->step += 1;
    B->list_cur = 1 - B->list_cur;  // three sweeps flip the current list
    return cudaSuccess;
}

// Median time of `reps` first-sweep passes (listing, fluxes, update into the
// first scratch buffer) with one launch shape; the state is not modified.
float time_shape(vof_batch* B, int warps, int per_sm, int reps) {
    B->update_warps = warps;
    B->update_blocks_per_sm = per_sm;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<float> t;
    for (int r = 0; r < reps + 1; ++r) {
        SweepArgs a = batch_args(B);
        a.list_valid = false;  // list the first sweep from c, then one sweep only
        cudaEventRecord(e0, B->stream);
        cudaError_t err = cudaSuccess;
        if (B->cfg.precision == VOF_FP64)
            err = advect_first_sweep_fp64(batch_set<double>(B), a);
        else
            err = advect_first_sweep_fp32(batch_set<float>(B), a);
        cudaEventRecord(e1, B->stream);
        if (err != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            note_cuda_error(err != cudaSuccess ? err : cudaGetLastError());
            t.assign(1, INFINITY);
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) t.push_back(ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

}  // namespace

extern "C" {

size_t vof_batch_workspace_size(const vof_batch_config* cfg, const vof_box_desc* boxes, int32_t n_boxes) {
    if (!batch_config_valid(cfg) || !boxes || n_boxes < 1 || n_boxes > kMaxBoxes) return 0;
    const int es = cfg->precision == VOF_FP64 ? 8 : 4;
    for (int b = 0; b < n_boxes; ++b)
        if (!box_valid(boxes[b], es)) return 0;
    return batch_layout(cfg, boxes, n_boxes).total;
}

vof_status vof_batch_config_default(vof_batch_config* cfg) {
    if (!cfg) return VOF_ERR_ARG;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->precision = VOF_MIXED;
    cfg->h = 1.0;
    cfg->tag_tau = 1e-6;
    cfg->alpha_fp64_band = 1e-3;
    cfg->use_graph = 1;
    cfg->autotune = 1;
    return VOF_OK;
}

vof_status vof_batch_init(const vof_batch_config* cfg, const vof_box_desc* boxes, int32_t n_boxes,
                          void* workspace_dev, size_t workspace_bytes, void* stream, vof_batch** out) {
    if (!out) return VOF_ERR_ARG;
    *out = nullptr;
    const size_t need = vof_batch_workspace_size(cfg, boxes, n_boxes);
    if (need == 0 || !workspace_dev || ((uintptr_t)workspace_dev & 255)) return VOF_ERR_ARG;
    if (workspace_bytes < need) return VOF_ERR_WORKSPACE;
    vof_batch* B = new (std::nothrow) vof_batch();
    if (!B) return VOF_ERR_ARG;
    B->cfg = *cfg;
    B->boxes.assign(boxes, boxes + n_boxes);
    B->L = batch_layout(cfg, boxes, n_boxes);
    B->ws = (char*)workspace_dev;
    B->stream = (cudaStream_t)stream;
    B->step = 0;
    B->list_valid = false;
    B->list_cur = 0;
    B->mlp = nullptr;
    B->mlp_tol = 1e-3;
    // default launch shape of the update pass: 8 warps, one resident wave
    B->update_warps = 8;
    B->update_blocks_per_sm = 1;
    {
        const int occ = update_occupancy(fp64_batch(cfg), 8);
        if (occ > 0) B->update_blocks_per_sm = occ;
    }
    B->tune_ms_best = 0.f;
    B->tune_candidates = 0;
    std::memset(B->graphs, 0, sizeof(B->graphs));
    B->cap_stream = nullptr;
    B->graph_launches = 0;
    B->direct_steps = 0;
    B->sticky = VOF_OK;
    // velocities: finite, and the time step of each box within CFL 1/2
    const bool fp64 = cfg->precision == VOF_FP64;
    double* vs = (double*)(B->ws + B->L.vscan);
    for (int b = 0; b < n_boxes; ++b) {
        const vof_box_desc& d = boxes[b];
        unsigned long long host[2];
        if (velocity_scan(fp64, d.u_dev, 3ll * d.nx * d.ny * d.nz, vs, B->stream) != cudaSuccess ||
            cudaMemcpyAsync(host, vs, sizeof(host), cudaMemcpyDeviceToHost, B->stream) != cudaSuccess ||
            cudaStreamSynchronize(B->stream) != cudaSuccess) {
            (void)cudaGetLastError();
            delete B;
            return VOF_ERR_CUDA;
        }
        double mx;
        std::memcpy(&mx, &host[0], sizeof(double));
        vof_status s = host[1] ? VOF_ERR_NONFINITE : (mx * d.dt / cfg->h > 0.5 ? VOF_ERR_CFL : VOF_OK);
        if (s != VOF_OK) {
            delete B;
            return s;
        }
    }
    if (cudaMemsetAsync(B->ws + B->L.clipped, 0, (size_t)n_boxes * 16 * 8, B->stream) != cudaSuccess ||
        cudaMemsetAsync(B->ws + B->L.misc, 0, 64, B->stream) != cudaSuccess) {
        (void)cudaGetLastError();
        delete B;
        return VOF_ERR_CUDA;
    }
    *out = B;
    return VOF_OK;
}

vof_status vof_batch_set_mlp(vof_batch* B, const void* weights_dev, double fallback_tol) {
    if (!B) return VOF_ERR_ARG;
    if (B->sticky != VOF_OK) return B->sticky;
    if (B->cfg.precision != VOF_MIXED_LEARNED || !weights_dev || ((uintptr_t)weights_dev & 15) ||
        !(fallback_tol >= 0.0) || !std::isfinite(fallback_tol))
        return VOF_ERR_ARG;
    B->mlp = weights_dev;
    B->mlp_tol = fallback_tol;
    for (auto& r : B->graphs)
        for (auto& g : r)
            if (g) cudaGraphExecDestroy(g), g = nullptr;
    return VOF_OK;
}

vof_status vof_batch_tune(vof_batch* B) {
    if (!B) return VOF_ERR_ARG;
    if (B->sticky != VOF_OK) return B->sticky;
    if (B->cfg.precision == VOF_MIXED_LEARNED && !B->mlp) return VOF_ERR_STATE;
    // candidates: warps per block x resident blocks per SM
    float best = INFINITY;
    int bw = 8, bp = 0, n = 0;
    const int warps_c[2] = {4, 8};
    for (int w : warps_c) {
        const int occ = update_occupancy(B->cfg.precision == VOF_FP64, w);
        for (int p = 1; p <= std::max(1, occ); p = p < 2 ? 2 : p + 2) {
            const float ms = time_shape(B, w, p, 3);
            ++n;
            if (ms < best) best = ms, bw = w, bp = p;
        }
    }
    (void)cudaGetLastError();
    if (!std::isfinite(best)) return fail(B, VOF_ERR_CUDA);
    B->update_warps = bw;
    B->update_blocks_per_sm = bp;
    B->tune_ms_best = best;
    B->tune_candidates = n;
    // the timed sweeps counted faces: start the counters afresh
    if (cudaMemsetAsync(B->ws + B->L.misc + 8, 0, 24, B->stream) != cudaSuccess) return fail(B, VOF_ERR_CUDA);
    for (auto& r : B->graphs)
        for (auto& g : r)
            if (g) cudaGraphExecDestroy(g), g = nullptr;
    return VOF_OK;
}

vof_status vof_batch_step(vof_batch* B, int32_t nsteps) {
    if (!B || nsteps < 0) return VOF_ERR_ARG;
    if (B->sticky != VOF_OK) return B->sticky;
    if (B->cfg.precision == VOF_MIXED_LEARNED && !B->mlp) return VOF_ERR_STATE;
    if (B->cfg.autotune && B->tune_candidates == 0) {
        vof_status s = vof_batch_tune(B);
        if (s != VOF_OK) return s;
    }
    int done = 0;
    if (!B->list_valid && nsteps > 0) {
        // the first step lists its first sweep's faces from c: run it directly
        SweepArgs a = batch_args(B);
        const cudaError_t e = advance(B, a, 1);
        if (e != cudaSuccess) return note_cuda_error(e), fail(B, VOF_ERR_CUDA);
        B->list_valid = true;
        B->list_cur = a.list_cur;
        B->step += 1;
        B->direct_steps += 1;
        done = 1;
    }
    for (; done < nsteps; ++done) {
        if (B->cfg.use_graph) {
            const cudaError_t e = graph_step(B);
            if (e != cudaSuccess) return note_cuda_error(e), fail(B, VOF_ERR_CUDA);
        } else {
            SweepArgs a = batch_args(B);
            const cudaError_t e = advance(B, a, 1);
            if (e != cudaSuccess) return note_cuda_error(e), fail(B, VOF_ERR_CUDA);
            B->list_cur = a.list_cur;
            B->step += 1;
            B->direct_steps += 1;
        }
    }
    return VOF_OK;
}

vof_status vof_batch_report(vof_batch* B, vof_batch_report_t* r) {
    if (!B || !r) return VOF_ERR_ARG;
    const int n = (int)B->boxes.size();
    std::vector<double> cl((size_t)n * 16);
    unsigned long long cnt[3];
    int st = 0;
    if (cudaMemcpyAsync(cl.data(), B->ws + B->L.clipped, cl.size() * 8, cudaMemcpyDeviceToHost, B->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(cnt, B->ws + B->L.misc + 8, 24, cudaMemcpyDeviceToHost, B->stream) != cudaSuccess ||
        cudaMemcpyAsync(&st, B->ws + B->L.misc, 4, cudaMemcpyDeviceToHost, B->stream) != cudaSuccess ||
        cudaStreamSynchronize(B->stream) != cudaSuccess)
        return fail(B, VOF_ERR_CUDA);
    if (st) return fail(B, VOF_ERR_TIMEOUT);
    std::memset(r, 0, sizeof(*r));
    r->steps_done = B->step;
    r->n_boxes = n;
    for (int b = 0; b < n; ++b) {
        double s = 0.0;
        for (int f = 0; f < 16; ++f) s += cl[(size_t)b * 16 + f];
        r->clipped_volume[b] = s * B->cfg.h * B->cfg.h * B->cfg.h;
    }
    long long fs = 0;
    for (const auto& d : B->boxes) fs += (long long)d.nx * d.ny * d.nz * d.k_active;
    r->cell_fields_per_step = fs;
    r->faces_network = (int64_t)cnt[0];
    r->faces_myc = (int64_t)cnt[1];
    r->faces_myc_judged = (int64_t)cnt[2];
    r->update_warps = B->update_warps;
    r->update_blocks_per_sm = B->update_blocks_per_sm;
    r->tune_candidates = B->tune_candidates;
    r->tune_best_ms = B->tune_ms_best;
    r->graph_launches = B->graph_launches;
    r->direct_steps = B->direct_steps;
    return VOF_OK;
}

void vof_batch_destroy(vof_batch* B) {
    if (!B) return;
    for (auto& r : B->graphs)
        for (auto& g : r)
            if (g) cudaGraphExecDestroy(g);
    if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
    delete B;
}

}  // extern "C"
