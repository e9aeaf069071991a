// Learned interface normal: an MLP 27 -> 64 -> 64 -> 3 (ReLU) on the
// canonicalised 3x3x3 volume-fraction stencil, BF16 weights and activations,
// FP32 accumulation in tensor memory (tcgen05), used in place of MYC with
// MYC as the fallback.  (No counterpart in the paper; the paper's PLIC
// normals are the method it replaces.)
//
// Canonical frame: the stencil is reflected so that every Youngs component
// is >= 0 and its axes are permuted so that |m_x| <= |m_y| <= |m_z| (ties to
// the lower axis); the network sees c - 1/2 in that frame and its output is
// mapped back.  One CTA of 128 threads runs 128 stencils per tile, thread t
// owning row t of every matrix and lane t of tensor memory.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "mlp.cuh"
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

// ---------------------------------------------------------------------------
// one CTA-wide forward pass over a tile of 128 canonical inputs

// Shared-memory image of the network plus activation tiles.
struct MlpSmem {
    unsigned char X[128 * kInHL * 2];    // 128 x 64 (hi | lo)
    unsigned char H[128 * kHid * 2];     // 128 x 64
    unsigned char W1[kHid * kInHL * 2];  // 64 x 64 (W1 | W1)
    unsigned char W2[kHid * kHid * 2];   // 64 x 64
    unsigned char W3[kOutP * kHid * 2];  // 16 x 64
    float b1[kHid], b2[kHid], b3[kOutP];
    uint64_t bar;
    uint32_t tbase;
    int timeout;
};

__device__ void load_weights(MlpSmem& s, const MlpBlob* __restrict__ w) {
    for (int idx = threadIdx.x; idx < kHid * kIn; idx += blockDim.x) {
        const int o = idx / kIn, i = idx % kIn;
        *reinterpret_cast<__nv_bfloat16*>(s.W1 + tc::kmajor_offset(o, i, kInHL)) = w->W1[idx];
        *reinterpret_cast<__nv_bfloat16*>(s.W1 + tc::kmajor_offset(o, kIn + i, kInHL)) = w->W1[idx];
    }
    for (int idx = threadIdx.x; idx < kHid * kHid; idx += blockDim.x)
        *reinterpret_cast<__nv_bfloat16*>(s.W2 + tc::kmajor_offset(idx / kHid, idx % kHid, kHid)) = w->W2[idx];
    for (int idx = threadIdx.x; idx < kOutP * kHid; idx += blockDim.x)
        *reinterpret_cast<__nv_bfloat16*>(s.W3 + tc::kmajor_offset(idx / kHid, idx % kHid, kHid)) = w->W3[idx];
    for (int idx = threadIdx.x; idx < kHid; idx += blockDim.x) {
        s.b1[idx] = w->b1[idx];
        s.b2[idx] = w->b2[idx];
    }
    for (int idx = threadIdx.x; idx < kOutP; idx += blockDim.x) s.b3[idx] = w->b3[idx];
}

// Row t of the layer-1 input tile: BF16 high parts, then low parts.
__device__ __forceinline__ void store_input_row(unsigned char* X, int t, const float x[27]) {
    for (int q = 0; q < kIn; ++q) {
        __nv_bfloat16 hi, lo;
        split_bf16(q < 27 ? x[q] : 0.f, hi, lo);
        *reinterpret_cast<__nv_bfloat16*>(X + tc::kmajor_offset(t, q, kInHL)) = hi;
        *reinterpret_cast<__nv_bfloat16*>(X + tc::kmajor_offset(t, kIn + q, kInHL)) = lo;
    }
}

// Tensor-memory columns of the three layer outputs.
// D3 reuses D1's columns (D1 is in registers before layer 2 is issued), so
// four CTAs fit the 512 columns of an SM.
constexpr uint32_t kColD1 = 0, kColD2 = 64, kColD3 = 0, kTmemCols = 128;

// Issue one layer (thread 0): D = A * W^T over K in steps of 16.
__device__ __forceinline__ void issue_layer(uint32_t d, const unsigned char* A, const unsigned char* W, int K, int N,
                                            uint64_t* bar) {
    const uint32_t idesc = tc::idesc_bf16(128, N);
    for (int s = 0; s < K / 16; ++s)
        tc::mma_bf16(d, tc::sdesc(tc::smem_u32(A) + s * 256, K), tc::sdesc(tc::smem_u32(W) + s * 256, K), idesc,
                     s > 0);
    tc::mma_commit(bar);
}

// Wait for the layer, bring its row into registers.  Returns false on a
// timed-out wait (the caller stops and reports it).
__device__ __forceinline__ bool finish_layer(MlpSmem& s, uint32_t& phase) {
    const bool ok = tc::mbar_wait(&s.bar, phase & 1u);
    phase += 1;
    // every thread takes the same decision (no thread may stop at a
    // different barrier than the others)
    const int failed = __syncthreads_or(!ok);
    tc::fence_after_sync();
    if (failed) {
        if (threadIdx.x == 0) s.timeout = 1;
        return false;
    }
    return true;
}

// Forward pass of the tile whose canonical inputs are in s.X.  out[3] gets
// this thread's canonical output.  Every thread of the CTA must call it.
__device__ bool mlp_tile_forward(MlpSmem& s, uint32_t taddr, uint32_t& phase, float out[3]) {
    const int t = threadIdx.x;
    const uint32_t lane_off = (uint32_t)(32 * (t >> 5)) << 16;
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) issue_layer(taddr + kColD1, s.X, s.W1, kInHL, kHid, &s.bar);
    if (!finish_layer(s, phase)) return false;
    for (int c0 = 0; c0 < kHid; c0 += 16) {
        float v[16];
        tc::tmem_ld16(taddr + lane_off + kColD1 + c0, v);
        for (int q = 0; q < 16; ++q) tc::store_bf16(s.H, t, c0 + q, kHid, fmaxf(v[q] + s.b1[c0 + q], 0.f));
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) issue_layer(taddr + kColD2, s.H, s.W2, kHid, kHid, &s.bar);
    if (!finish_layer(s, phase)) return false;
    float h2[kHid];
    for (int c0 = 0; c0 < kHid; c0 += 16) {
        float v[16];
        tc::tmem_ld16(taddr + lane_off + kColD2 + c0, v);
        for (int q = 0; q < 16; ++q) h2[c0 + q] = fmaxf(v[q] + s.b2[c0 + q], 0.f);
    }
    // layer 2 has finished reading H: reuse it for layer 3's input
    for (int q = 0; q < kHid; ++q) tc::store_bf16(s.H, t, q, kHid, h2[q]);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) issue_layer(taddr + kColD3, s.H, s.W3, kHid, kOutP, &s.bar);
    if (!finish_layer(s, phase)) return false;
    float v[16];
    tc::tmem_ld16(taddr + lane_off + kColD3, v);
    out[0] = v[0] + s.b3[0];
    out[1] = v[1] + s.b3[1];
    out[2] = v[2] + s.b3[2];
    return true;
}

__device__ void mlp_cta_begin(MlpSmem& s, const MlpBlob* w) {
    load_weights(s, w);
    if (threadIdx.x == 0) {
        tc::mbar_init(&s.bar, 1);
        s.timeout = 0;
    }
    if (threadIdx.x < 32) {
        tc::tmem_alloc(&s.tbase, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

__device__ void mlp_cta_end(MlpSmem& s, int* status) {
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x < 32) tc::tmem_dealloc(s.tbase, kTmemCols);
    if (threadIdx.x == 0 && s.timeout && status) atomicExch(status, 1);
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
        store_input_row(s.X, t, x);
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

cudaError_t mlp_forward(const MlpBlob* w, const float* st, float* n_out, long long n, int* status,
                        cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpSmem));
    long long tiles = (n + 127) / 128;
    int blocks = (int)std::min<long long>(tiles, 152LL * 4);
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
