// Learned interface normal: an MLP 27 -> 64 -> 64 -> 3 (ReLU) on the
// canonicalised 3x3x3 volume-fraction stencil, BF16 weights, every layer
// input as a BF16 (hi, lo) pair, FP32 accumulation in tensor memory
// (tcgen05), used in place of MYC with MYC as the fallback.  (No counterpart in the paper; the paper's PLIC
// normals are the method it replaces.)
//
// Canonical frame: the stencil is reflected so that every Youngs component
// is >= 0 and its axes are permuted so that |m_x| <= |m_y| <= |m_z| (ties to
// the lower axis); the network sees c - 1/2 in that frame and its output is
// mapped back.  One CTA of 128 threads runs 128 stencils per tile, thread t
// owning row t of every matrix and lane t of tensor memory.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"
#include "mlp.cuh"
#include "mlp_tile.cuh"
#include "plic.cuh"
#include "tc.cuh"

namespace vof {

// ---------------------------------------------------------------------------
// tensor-core layout self-check: D[128][n] = A[128][k] B[n][k]^T in BF16

__global__ void __launch_bounds__(128) k_tc_gemm_check(const float* __restrict__ A, const float* __restrict__ B,
                                                       float* __restrict__ D, int K, int N, int swap,
                                                       int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* As = smem;                       // 128 x K
    unsigned char* Bs = smem + 128 * K * 2;         // N x K
    __shared__ uint64_t bar;
    __shared__ uint32_t tbase;
    const int t = threadIdx.x;
    for (int k = 0; k < K; ++k) tc::store_bf16(As, t, k, K, A[t * K + k]);
    for (int idx = t; idx < N * K; idx += 128) tc::store_bf16(Bs, idx / K, idx % K, K, B[idx]);
    if (t == 0) tc::mbar_init(&bar, 1);
    if (t < 32) {
        tc::tmem_alloc(&tbase, 256);
        tc::tmem_relinquish();
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tbase;
    if (t == 0) {
        const uint32_t idesc = tc::idesc_bf16(128, N);
        for (int s = 0; s < K / 16; ++s) {
            uint64_t ad = tc::sdesc(tc::smem_u32(As) + s * 256, K, swap);
            uint64_t bd = tc::sdesc(tc::smem_u32(Bs) + s * 256, K, swap);
            tc::mma_bf16(taddr, ad, bd, idesc, s > 0);
        }
        tc::mma_commit(&bar);
    }
    bool ok = tc::mbar_wait(&bar, 0);
    tc::fence_after_sync();
    if (!ok) {
        if (t == 0) atomicExch(status, 1);
    } else {
        const int w = t >> 5;
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc::tmem_ld16(taddr + ((uint32_t)(32 * w) << 16) + c0, v);
            for (int q = 0; q < 16; ++q)
                if (c0 + q < N) D[t * N + c0 + q] = v[q];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (t < 32) tc::tmem_dealloc(taddr, 256);
}

cudaError_t tc_gemm_check(const float* A, const float* B, float* D, int K, int N, int swap, int* status,
                          cudaStream_t st) {
    size_t smem = (size_t)(128 + N) * K * 2;
    cudaFuncSetAttribute(k_tc_gemm_check, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_tc_gemm_check<<<1, 128, smem, st>>>(A, B, D, K, N, swap, status);
    return cudaGetLastError();
}

// Normal of each raw stencil st[n][27] (float): canonicalise, run the
// network, map back, L2-normalise.  Output n_out[n][3].
__global__ void __launch_bounds__(128, 4) k_mlp_forward(const MlpBlob* __restrict__ w, const float* __restrict__ st,
                                                        float* __restrict__ n_out, long long n,
                                                        int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    MlpSmem& s = *reinterpret_cast<MlpSmem*>(smem_raw);
    mlp_cta_begin(s, w);
    const uint32_t taddr = s.tbase;
    uint32_t phase = 0;
    const int t = threadIdx.x;
    for (long long base = (long long)blockIdx.x * 128; base < n; base += (long long)gridDim.x * 128) {
        const long long r = base + t;
        float sv[27];
        CanonFrame fr;
        if (r < n) {
            for (int q = 0; q < 27; ++q) sv[q] = st[r * 27 + q];
        } else {
            for (int q = 0; q < 27; ++q) sv[q] = 0.f;
        }
        canon_frame(sv, fr);
        float x[27];
        canon_input(sv, fr, x);
        store_input_row(s, t, x);
        float oc[3];
        if (!mlp_tile_forward(s, taddr, phase, oc)) break;
        float nn[3];
        canon_output(oc, fr, nn);
        float nrm = sqrtf(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
        if (r < n) {
            float inv = nrm > 0.f ? 1.f / nrm : 0.f;
            n_out[r * 3 + 0] = nn[0] * inv;
            n_out[r * 3 + 1] = nn[1] * inv;
            n_out[r * 3 + 2] = nn[2] * inv;
        }
    }
    mlp_cta_end(s, status);
}

// The judged learned normal of each raw stencil (the estimator exactly as
// the learned step applies it to a donor): m_out[n][3] L1-normalised,
// which_out[n] = 0 network kept, 1 MYC.
__global__ void __launch_bounds__(128, 3) k_learned_normals(const MlpBlob* __restrict__ w,
                                                            const float* __restrict__ st, float tol,
                                                            float* __restrict__ m_out,
                                                            int* __restrict__ which_out, long long n,
                                                            int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    MlpSmem& s = *reinterpret_cast<MlpSmem*>(smem_raw);
    mlp_cta_begin(s, w);
    const uint32_t taddr = s.tbase;
    uint32_t phase = 0;
    const int t = threadIdx.x;
    for (long long base = (long long)blockIdx.x * 128; base < n; base += (long long)gridDim.x * 128) {
        const long long r = base + t;
        float sv[27];
        for (int q = 0; q < 27; ++q) sv[q] = r < n ? st[r * 27 + q] : 0.5f;
        CanonFrame fr;
        canon_frame(sv, fr);
        float x[27];
        canon_input(sv, fr, x);
        store_input_row(s, t, x);
        float oc[3];
        if (!mlp_tile_forward(s, taddr, phase, oc)) break;
        if (r < n) {
            float nn[3], m[3];
            canon_output(oc, fr, nn);
            const bool keep = judged_normal(sv, nn, tol, m);
            m_out[r * 3 + 0] = m[0];
            m_out[r * 3 + 1] = m[1];
            m_out[r * 3 + 2] = m[2];
            which_out[r] = keep ? 0 : 1;
        }
    }
    mlp_cta_end(s, status);
}

cudaError_t learned_normals(const MlpBlob* w, const float* st, float tol, float* m_out, int* which_out,
                            long long n, int* status, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    cudaFuncSetAttribute(k_learned_normals, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpSmem));
    const int blocks = (int)std::min<long long>((n + 127) / 128, (long long)sm_count() * 3);
    k_learned_normals<<<blocks, 128, sizeof(MlpSmem), stream>>>(w, st, tol, m_out, which_out, n, status);
    return cudaGetLastError();
}

cudaError_t mlp_forward(const MlpBlob* w, const float* st, float* n_out, long long n, int* status,
                        cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpSmem));
    long long tiles = (n + 127) / 128;
    int blocks = (int)std::min<long long>(tiles, (long long)sm_count() * 4);
    k_mlp_forward<<<blocks, 128, sizeof(MlpSmem), stream>>>(w, st, n_out, n, status);
    return cudaGetLastError();
}

}  // namespace vof

namespace {
__device__ int g_mlp_status;

vof_status read_status(cudaStream_t st) {
    int h = 0;
    if (cudaMemcpyFromSymbolAsync(&h, g_mlp_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        (void)cudaGetLastError();
        return VOF_ERR_CUDA;
    }
    return h ? VOF_ERR_TIMEOUT : VOF_OK;
}

int* status_ptr() {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_mlp_status) != cudaSuccess) return nullptr;
    return (int*)p;
}
}  // namespace

extern "C" size_t vof_mlp_weights_size(void) { return sizeof(vof::MlpBlob); }

extern "C" vof_status vof_mlp_forward(const void* weights_dev, const float* stencils_dev, float* normals_dev,
                                      int64_t n, void* stream) {
    if (n < 0 || (n > 0 && (!weights_dev || !stencils_dev || !normals_dev))) return VOF_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int* sp = status_ptr();
    if (!sp || cudaMemsetAsync(sp, 0, sizeof(int), st) != cudaSuccess) return VOF_ERR_CUDA;
    if (vof::mlp_forward((const vof::MlpBlob*)weights_dev, stencils_dev, normals_dev, n, sp, st) != cudaSuccess) {
        (void)cudaGetLastError();
        return VOF_ERR_CUDA;
    }
    return read_status(st);
}

extern "C" vof_status vof_learned_normals(const void* weights_dev, const float* stencils_dev, int64_t n,
                                          double fallback_tol, float* normals_dev, int32_t* which_dev,
                                          void* stream) {
    if (n < 0 || (n > 0 && (!weights_dev || !stencils_dev || !normals_dev || !which_dev)) ||
        !(fallback_tol >= 0.0) || !std::isfinite(fallback_tol))
        return VOF_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int* sp = status_ptr();
    if (!sp || cudaMemsetAsync(sp, 0, sizeof(int), st) != cudaSuccess) return VOF_ERR_CUDA;
    if (vof::learned_normals((const vof::MlpBlob*)weights_dev, stencils_dev, (float)fallback_tol, normals_dev,
                             which_dev, n, sp, st) != cudaSuccess) {
        (void)cudaGetLastError();
        return VOF_ERR_CUDA;
    }
    return read_status(st);
}

namespace vof {
// An mbarrier that nothing arrives at, waited on with the bounded wait the
// tensor-core kernels use: the wait gives up after `limit` polls and the
// kernel reports it, the context stays usable.
__global__ void k_wait_selftest(long long limit, int* __restrict__ status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) tc::mbar_init(&bar, 1);
    __syncthreads();
    const bool ok = tc::mbar_wait(&bar, 0u, limit);
    if (!__syncthreads_and(ok) && threadIdx.x == 0) atomicExch(status, 1);
}
}  // namespace vof

extern "C" vof_status vof_wait_selftest(int64_t poll_limit, void* stream) {
    if (poll_limit < 1 || poll_limit > 100000000LL) return VOF_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int* sp = status_ptr();
    if (!sp || cudaMemsetAsync(sp, 0, sizeof(int), st) != cudaSuccess) return VOF_ERR_CUDA;
    vof::k_wait_selftest<<<1, 32, 0, st>>>(poll_limit, sp);
    if (cudaGetLastError() != cudaSuccess) return VOF_ERR_CUDA;
    return read_status(st);
}

extern "C" vof_status vof_tc_gemm_check(const float* a_dev, const float* b_dev, float* d_dev, int32_t k,
                                        int32_t n, int32_t variant, void* stream) {
    if (!a_dev || !b_dev || !d_dev || (k != 16 && k != 32 && k != 64) || (n != 16 && n != 32 && n != 64))
        return VOF_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int* sp = status_ptr();
    if (!sp || cudaMemsetAsync(sp, 0, sizeof(int), st) != cudaSuccess) return VOF_ERR_CUDA;
    if (vof::tc_gemm_check(a_dev, b_dev, d_dev, k, n, variant, sp, st) != cudaSuccess) {
        (void)cudaGetLastError();
        return VOF_ERR_CUDA;
    }
    return read_status(st);
}
