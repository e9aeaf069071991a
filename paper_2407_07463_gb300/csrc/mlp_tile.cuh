// One CTA-wide forward pass of the learned normal estimator over a tile of
// 128 canonical stencils on the tensor cores (internal): weights staged in
// shared memory, each layer one tcgen05 MMA chain (M = 128, BF16 operands,
// FP32 accumulation in tensor memory) issued by one thread, bias + ReLU in
// the epilogue of the thread that owns the row.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "mlp.cuh"
#include "mlp_judge.cuh"
#include "plic.cuh"
#include "tc.cuh"

namespace vof {

// Shared-memory image of the network plus activation tiles.
// H holds the layer-1 input (128 x 64, hi | lo) at its start, then each
// hidden activation tile (128 x 128, hi | lo) once the layer reading the
// previous content has completed.  The weights are held once: the MMA
// chain over the hi and lo halves of K reads the same weight columns.
struct MlpSmem {
    unsigned char H[128 * kHidHL * 2];   // 128 x 128
    unsigned char W1[kHid * kIn * 2];    // 64 x 32
    unsigned char W2[kHid * kHid * 2];   // 64 x 64
    unsigned char W3[kOutP * kHid * 2];  // 16 x 64
    float b1[kHid], b2[kHid], b3[kOutP];
    uint64_t bar;
    uint32_t tbase;
    int timeout;
};

__device__ __forceinline__ void load_weights(MlpSmem& s, const MlpBlob* __restrict__ w) {
    for (int idx = threadIdx.x; idx < kHid * kIn; idx += blockDim.x)
        *reinterpret_cast<__nv_bfloat16*>(s.W1 + tc::kmajor_offset(idx / kIn, idx % kIn, kIn)) = w->W1[idx];
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
__device__ __forceinline__ void store_input_row(MlpSmem& s, int t, const float x[27]) {
#pragma unroll
    for (int k0 = 0; k0 < kIn; k0 += 8) {
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = k0 + q < 27 ? x[k0 + q] : 0.f;
        store_pairs8(s.H, t, k0, kIn, kInHL, v);
    }
}

// Float scratch [27][128] in the upper half of H (bytes 16 K .. 30 K), free
// while the layer-1 input (the lower 16 K) is being written: a stencil per
// thread column, read back with the frame's offsets.
__device__ __forceinline__ float* stencil_scratch(MlpSmem& s) {
    return reinterpret_cast<float*>(s.H + 128 * kInHL * 2);
}

// Tensor-memory columns of the three layer outputs.
// D3 reuses D1's columns (D1 is in shared memory before layer 2 is issued),
// so four CTAs fit the 512 columns of an SM.
constexpr uint32_t kColD1 = 0, kColD2 = 64, kColD3 = 0, kTmemCols = 128;

// Issue one layer (thread 0): D = [A_hi | A_lo] * [W | W]^T, i.e. the K
// steps of 16 run over the KA = 2 KW columns of A while the weight
// descriptor wraps around W's KW columns.
__device__ __forceinline__ void issue_layer(uint32_t d, const unsigned char* A, int KA, const unsigned char* W, int KW,
                                            int N, uint64_t* bar) {
    const uint32_t idesc = tc::idesc_bf16(128, N);
    const int ws = KW / 16;
    for (int s = 0; s < KA / 16; ++s)
        tc::mma_bf16(d, tc::sdesc(tc::smem_u32(A) + s * 256, KA), tc::sdesc(tc::smem_u32(W) + (s % ws) * 256, KW),
                     idesc, s > 0);
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

// Forward pass of the tile whose canonical inputs are in s.H.  out[3] gets
// this thread's canonical output.  Every thread of the CTA must call it.
__device__ __forceinline__ bool mlp_tile_forward(MlpSmem& s, uint32_t taddr, uint32_t& phase, float out[3]) {
    const int t = threadIdx.x;
    const uint32_t lane_off = (uint32_t)(32 * (t >> 5)) << 16;
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) issue_layer(taddr + kColD1, s.H, kInHL, s.W1, kIn, kHid, &s.bar);
    if (!finish_layer(s, phase)) return false;
    for (int c0 = 0; c0 < kHid; c0 += 32) {
        float v[32];
        tc::tmem_ld32(taddr + lane_off + kColD1 + c0, v);
#pragma unroll
        for (int q = 0; q < 32; ++q) v[q] = fmaxf(v[q] + s.b1[c0 + q], 0.f);
#pragma unroll
        for (int k8 = 0; k8 < 32; k8 += 8) store_pairs8(s.H, t, c0 + k8, kHid, kHidHL, v + k8);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) issue_layer(taddr + kColD2, s.H, kHidHL, s.W2, kHid, kHid, &s.bar);
    if (!finish_layer(s, phase)) return false;
    // layer 2 has finished reading H: its output goes there as layer 3's input
    for (int c0 = 0; c0 < kHid; c0 += 32) {
        float v[32];
        tc::tmem_ld32(taddr + lane_off + kColD2 + c0, v);
#pragma unroll
        for (int q = 0; q < 32; ++q) v[q] = fmaxf(v[q] + s.b2[c0 + q], 0.f);
#pragma unroll
        for (int k8 = 0; k8 < 32; k8 += 8) store_pairs8(s.H, t, c0 + k8, kHid, kHidHL, v + k8);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) issue_layer(taddr + kColD3, s.H, kHidHL, s.W3, kHid, kOutP, &s.bar);
    if (!finish_layer(s, phase)) return false;
    float v[16];
    tc::tmem_ld16(taddr + lane_off + kColD3, v);
    out[0] = v[0] + s.b3[0];
    out[1] = v[1] + s.b3[1];
    out[2] = v[2] + s.b3[2];
    return true;
}

__device__ __forceinline__ void mlp_cta_begin(MlpSmem& s, const MlpBlob* w) {
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

__device__ __forceinline__ void mlp_cta_end(MlpSmem& s, int* status) {
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x < 32) tc::tmem_dealloc(s.tbase, kTmemCols);
    if (threadIdx.x == 0 && s.timeout && status) atomicExch(status, 1);
}

}  // namespace vof
