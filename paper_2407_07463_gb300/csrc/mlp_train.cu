// Training of the learned normal estimator on the GPU (no counterpart in
// the paper): stencils of exact planes and spheres generated on the device,
// forward and backward passes on the tensor cores (tcgen05, BF16 operands,
// FP32 accumulation in tensor memory), Adam on FP32 master weights.
//
// Every layer input (stencil, H1, H2) enters the forward pass as the BF16
// pair (hi, lo) against the weights held twice along K, as in inference.
// Backward of a tile of 128 samples (thread b owns sample b):
//   dY3 = d loss / d out                      (registers)
//   dH2 = dY3 W3,   dA2 = dH2 [a2 > 0]        (MMA, A = dY3, B = W3^T)
//   dH1 = dA2 W2,   dA1 = dH1 [a1 > 0]        (MMA, A = dA2, B = W2^T)
//   dW3^T += H2^T dY3, dW2^T += H1^T dA2, dW1^T += X^T dA1
//                                             (MMA, K = the 128 samples; the
//                                              hi and lo rows are summed on
//                                              the way out)
// The weight gradients accumulate in tensor memory over a CTA's tiles and
// are added to the global FP32 gradient once per launch.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "mlp.cuh"
#include "plic.cuh"
#include "tc.cuh"

namespace vof {

constexpr int kNParam = kHid * kIn + kHid * kHid + kOutP * kHid + kHid + kHid + kOutP;
constexpr int kOffW1 = 0, kOffW2 = kHid * kIn, kOffW3 = kOffW2 + kHid * kHid, kOffB1 = kOffW3 + kOutP * kHid,
              kOffB2 = kOffB1 + kHid, kOffB3 = kOffB2 + kHid;

// ---------------------------------------------------------------------------
// counter-based random numbers (SplitMix64 finaliser)

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double urand(uint64_t seed, uint64_t sample, int k) {
    return (double)(mix64(seed ^ mix64(sample * 64ull + (uint64_t)k)) >> 11) * (1.0 / 9007199254740992.0);
}
__device__ __forceinline__ void unit_vector(uint64_t seed, uint64_t s, int k0, double v[3]) {
    // uniform on the sphere: z uniform in [-1, 1], azimuth uniform
    double z = 2.0 * urand(seed, s, k0) - 1.0;
    double ph = 6.283185307179586 * urand(seed, s, k0 + 1);
    double r = sqrt(fmax(0.0, 1.0 - z * z));
    v[0] = r * cos(ph);
    v[1] = r * sin(ph);
    v[2] = z;
}

// ---------------------------------------------------------------------------
// training data: stencil of a plane or a sphere around the centre cell

// Volume fraction of the cell [i-1/2, i+1/2] x ... (centre cell at the
// origin) inside the ball |x - C| < R: Gauss quadrature over (x, y) of the
// analytic chord along z.
__device__ double sphere_fraction(const double C[3], double R, int i, int j, int k) {
    const double gx[4] = {0.0694318442029737, 0.3300094782075719, 0.6699905217924281, 0.9305681557970263};
    const double gw[4] = {0.1739274225687269, 0.3260725774312731, 0.3260725774312731, 0.1739274225687269};
    const int NS = 3;  // sub-intervals per axis
    double x0 = i - 0.5 - C[0], y0 = j - 0.5 - C[1], z0 = k - 0.5 - C[2];
    // whole cell outside / inside
    double dn[3] = {fmin(fmax(0.0, x0), x0 + 1.0), fmin(fmax(0.0, y0), y0 + 1.0), fmin(fmax(0.0, z0), z0 + 1.0)};
    if (dn[0] * dn[0] + dn[1] * dn[1] + dn[2] * dn[2] >= R * R) return 0.0;
    double fx = fmax(fabs(x0), fabs(x0 + 1.0)), fy = fmax(fabs(y0), fabs(y0 + 1.0)),
           fz = fmax(fabs(z0), fabs(z0 + 1.0));
    if (fx * fx + fy * fy + fz * fz <= R * R) return 1.0;
    double acc = 0.0;
    for (int a = 0; a < NS; ++a)
        for (int p = 0; p < 4; ++p) {
            double x = x0 + (a + gx[p]) / NS;
            for (int b = 0; b < NS; ++b)
                for (int q = 0; q < 4; ++q) {
                    double y = y0 + (b + gx[q]) / NS;
                    double h2 = R * R - x * x - y * y;
                    if (h2 <= 0.0) continue;
                    double hw = sqrt(h2);
                    double seg = fmin(z0 + 1.0, hw) - fmax(z0, -hw);
                    if (seg > 0.0) acc += gw[p] * gw[q] * seg;
                }
        }
    return fmin(1.0, acc / (NS * NS));
}

// rad (may be null) receives each sample's sphere radius, 0 for a plane.
__global__ void k_mlp_gen(float* __restrict__ st, float* __restrict__ tgt, float* __restrict__ rad, long long n,
                          uint64_t seed, double plane_frac, double r_min, double r_max) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        double t[3];
        float* o = st + s * 27;
        if (urand(seed, s, 0) < plane_frac) {
            double nv[3];
            unit_vector(seed, s, 1, nv);
            double half = 0.5 * (fabs(nv[0]) + fabs(nv[1]) + fabs(nv[2]));
            double a0 = (2.0 * urand(seed, s, 3) - 1.0) * 0.98 * half;
            for (int k = -1; k <= 1; ++k)
                for (int j = -1; j <= 1; ++j)
                    for (int i = -1; i <= 1; ++i) {
                        double al = a0 - (nv[0] * (i - 0.5) + nv[1] * (j - 0.5) + nv[2] * (k - 0.5));
                        o[(k + 1) * 9 + (j + 1) * 3 + (i + 1)] = (float)plic_volume<double>(nv[0], nv[1], nv[2], al);
                    }
            t[0] = nv[0];
            t[1] = nv[1];
            t[2] = nv[2];
            if (rad) rad[s] = 0.f;
        } else {
            double R = exp(log(r_min) + urand(seed, s, 4) * (log(r_max) - log(r_min)));
            double dir[3];
            unit_vector(seed, s, 5, dir);
            double dl = (2.0 * urand(seed, s, 7) - 1.0) * 0.4;
            double C[3] = {-(R + dl) * dir[0], -(R + dl) * dir[1], -(R + dl) * dir[2]};
            bool inv = urand(seed, s, 8) < 0.5;
            for (int k = -1; k <= 1; ++k)
                for (int j = -1; j <= 1; ++j)
                    for (int i = -1; i <= 1; ++i) {
                        double c = sphere_fraction(C, R, i, j, k);
                        o[(k + 1) * 9 + (j + 1) * 3 + (i + 1)] = (float)(inv ? 1.0 - c : c);
                    }
            // out of the liquid: away from the centre for a drop, towards it when inverted
            double sg = inv ? -1.0 : 1.0;
            t[0] = sg * dir[0];
            t[1] = sg * dir[1];
            t[2] = sg * dir[2];
            if (rad) rad[s] = (float)R;
        }
        tgt[s * 3 + 0] = (float)t[0];
        tgt[s * 3 + 1] = (float)t[1];
        tgt[s * 3 + 2] = (float)t[2];
    }
}

// ---------------------------------------------------------------------------
// forward + backward of tiles of 128 samples

struct TrainSmem {
    unsigned char W1[kHid * kInHL * 2];    // 64 x 64 (B of layer 1: W1 | W1)
    unsigned char W2[kHid * kHidHL * 2];   // 64 x 128 (W2 | W2)
    unsigned char W3[kOutP * kHidHL * 2];  // 16 x 128 (W3 | W3)
    unsigned char W2T[kHid * kHid * 2];    // 64 x 64: W2^T (B of dH1 = dA2 W2)
    unsigned char W3T[kHid * kOutP * 2];   // 64 x 16: W3^T (B of dH2 = dY3 W3)
    unsigned char X[128 * kInHL * 2];      // 128 x 64 (hi | lo)
    unsigned char H1[128 * kHidHL * 2];    // 128 x 128 (hi | lo)
    unsigned char H2[128 * kHidHL * 2];    // 128 x 128 (hi | lo)
    unsigned char T[128 * 128 * 2];        // 128 x 128: X^T, H1^T or H2^T (rows = hi/lo features)
    unsigned char DY[128 * kOutP * 2];    // 128 x 16: dY3
    unsigned char DYT[kOutP * 128 * 2];   // 16 x 128: dY3^T
    unsigned char DA[128 * kHid * 2];     // 128 x 64: dA2
    unsigned char DAT[kHid * 128 * 2];    // 64 x 128: dA2^T then dA1^T
    float b1[kHid], b2[kHid], b3[kOutP];
    float gb1[kHid], gb2[kHid], gb3[kOutP];
    float loss;
    uint64_t bar;
    uint32_t tbase;
    int timeout;
};

// tensor-memory columns
constexpr uint32_t kTD1 = 0, kTD2 = 64, kTD3 = 128, kTdH2 = 144, kTdH1 = 208, kTgW3 = 272, kTgW2 = 288,
                   kTgW1 = 352, kTrainCols = 512;

__device__ __forceinline__ float bf(const unsigned char* tile, int r, int k, int kext) {
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(tile + tc::kmajor_offset(r, k, kext)));
}

// one MMA chain D (+)= A B^T over K in steps of 16 (A: M=128 rows, B: N rows)
__device__ __forceinline__ void chain(uint32_t d, const unsigned char* A, int kextA, const unsigned char* B,
                                      int kextB, int K, int N, bool acc_first) {
    const uint32_t idesc = tc::idesc_bf16(128, N);
    for (int s = 0; s < K / 16; ++s)
        tc::mma_bf16(d, tc::sdesc(tc::smem_u32(A) + s * 256, kextA), tc::sdesc(tc::smem_u32(B) + s * 256, kextB),
                     idesc, (acc_first || s > 0) ? 1u : 0u);
}

__device__ __forceinline__ void publish_smem() {
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// thread 0 commits; everybody waits (uniform decision).  false on timeout.
__device__ __forceinline__ bool commit_wait(TrainSmem& s, uint32_t& phase) {
    if (threadIdx.x == 0) tc::mma_commit(&s.bar);
    const bool ok = tc::mbar_wait(&s.bar, phase & 1u);
    phase += 1;
    const int failed = __syncthreads_or(!ok);
    tc::fence_after_sync();
    if (failed && threadIdx.x == 0) s.timeout = 1;
    return !failed;
}

__global__ void __launch_bounds__(128, 1) k_mlp_train(const MlpBlob* __restrict__ w, const float* __restrict__ st,
                                                      const float* __restrict__ tgt, long long n0, long long n,
                                                      float inv_batch, float* __restrict__ grad,
                                                      float* __restrict__ loss_sum, int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TrainSmem& s = *reinterpret_cast<TrainSmem*>(smem_raw);
    const int t = threadIdx.x;
    // weights (forward and transposed copies), zeroed scratch
    load_weight_pair(s.W1, w->W1, kHid, kIn, t, 128);
    load_weight_pair(s.W2, w->W2, kHid, kHid, t, 128);
    load_weight_pair(s.W3, w->W3, kOutP, kHid, t, 128);
    for (int idx = t; idx < kHid * kHid; idx += 128) {
        const int o = idx / kHid, i = idx % kHid;
        *reinterpret_cast<__nv_bfloat16*>(s.W2T + tc::kmajor_offset(i, o, kHid)) = w->W2[idx];
    }
    for (int idx = t; idx < kOutP * kHid; idx += 128) {
        const int o = idx / kHid, i = idx % kHid;
        *reinterpret_cast<__nv_bfloat16*>(s.W3T + tc::kmajor_offset(i, o, kOutP)) = w->W3[idx];
    }
    for (int idx = t; idx < kHid; idx += 128) {
        s.b1[idx] = w->b1[idx];
        s.b2[idx] = w->b2[idx];
        s.gb1[idx] = 0.f;
        s.gb2[idx] = 0.f;
    }
    if (t < kOutP) {
        s.b3[t] = w->b3[t];
        s.gb3[t] = 0.f;
    }
    for (int idx = t; idx < 128 * 128 * 2 / 4; idx += 128) reinterpret_cast<uint32_t*>(s.T)[idx] = 0u;
    for (int idx = t; idx < kOutP * 128 * 2 / 4; idx += 128) reinterpret_cast<uint32_t*>(s.DYT)[idx] = 0u;
    if (t == 0) {
        s.loss = 0.f;
        s.timeout = 0;
        tc::mbar_init(&s.bar, 1);
    }
    if (t < 32) {
        tc::tmem_alloc(&s.tbase, kTrainCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = s.tbase;
    const uint32_t lane = (uint32_t)(32 * (t >> 5)) << 16;
    uint32_t phase = 0;
    bool first = true;
    bool alive = true;
    for (long long base = n0 + (long long)blockIdx.x * 128; base < n0 + n && alive;
         base += (long long)gridDim.x * 128) {
        const long long r = base + t;
        const bool valid = r < n0 + n;
        // canonical input and target
        float sv[27], tr[3] = {0.f, 0.f, 0.f};
        for (int q = 0; q < 27; ++q) sv[q] = valid ? st[r * 27 + q] : 0.f;
        if (valid) {
            tr[0] = tgt[r * 3];
            tr[1] = tgt[r * 3 + 1];
            tr[2] = tgt[r * 3 + 2];
        }
        CanonFrame fr;
        canon_frame(sv, fr);
        float x[27], tc3[3];
        canon_input(sv, fr, x);
        for (int q = 0; q < 3; ++q) tc3[q] = (float)pick3(fr.sign, fr.perm[q]) * pick3(tr, fr.perm[q]);
        for (int q = 0; q < kIn; ++q) store_pair(s.X, t, q, kIn, kInHL, (q < 27 && valid) ? x[q] : 0.f);
        // ---- forward
        publish_smem();
        if (t == 0) chain(tm + kTD1, s.X, kInHL, s.W1, kInHL, kInHL, kHid, false);
        if (!(alive = commit_wait(s, phase))) break;
        for (int c0 = 0; c0 < kHid; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tm + lane + kTD1 + c0, v);
            for (int q = 0; q < 16; ++q) store_pair(s.H1, t, c0 + q, kHid, kHidHL, fmaxf(v[q] + s.b1[c0 + q], 0.f));
        }
        publish_smem();
        if (t == 0) chain(tm + kTD2, s.H1, kHidHL, s.W2, kHidHL, kHidHL, kHid, false);
        if (!(alive = commit_wait(s, phase))) break;
        for (int c0 = 0; c0 < kHid; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tm + lane + kTD2 + c0, v);
            for (int q = 0; q < 16; ++q) store_pair(s.H2, t, c0 + q, kHid, kHidHL, fmaxf(v[q] + s.b2[c0 + q], 0.f));
        }
        publish_smem();
        if (t == 0) chain(tm + kTD3, s.H2, kHidHL, s.W3, kHidHL, kHidHL, kOutP, false);
        if (!(alive = commit_wait(s, phase))) break;
        float out[3];
        {
            float v[16];
            tc::tmem_ld16(tm + lane + kTD3, v);
            for (int q = 0; q < 3; ++q) out[q] = v[q] + s.b3[q];
        }
        // ---- loss 1 - cos(out, t) and its gradient
        float dy[3] = {0.f, 0.f, 0.f};
        if (valid) {
            const float nrm = sqrtf(out[0] * out[0] + out[1] * out[1] + out[2] * out[2]);
            const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
            const float nh[3] = {out[0] * inv, out[1] * inv, out[2] * inv};
            const float cs = nh[0] * tc3[0] + nh[1] * tc3[1] + nh[2] * tc3[2];
            atomicAdd(&s.loss, 1.f - cs);
            for (int q = 0; q < 3; ++q) dy[q] = -(tc3[q] - cs * nh[q]) * inv * inv_batch;
        }
        for (int q = 0; q < kOutP; ++q) {
            const float v = q < 3 ? dy[q] : 0.f;
            tc::store_bf16(s.DY, t, q, kOutP, v);
            if (q < 3) tc::store_bf16(s.DYT, q, t, 128, v);
        }
        for (int q = 0; q < 3; ++q) atomicAdd(&s.gb3[q], dy[q]);
        for (int i = 0; i < kHidHL; ++i) tc::store_bf16(s.T, i, t, 128, bf(s.H2, t, i, kHidHL));  // H2^T
        // ---- dH2 = dY3 W3 ; dW3^T += H2^T dY3
        publish_smem();
        if (t == 0) {
            chain(tm + kTdH2, s.DY, kOutP, s.W3T, kOutP, kOutP, kHid, false);
            chain(tm + kTgW3, s.T, 128, s.DYT, 128, 128, kOutP, !first);
        }
        if (!(alive = commit_wait(s, phase))) break;
        for (int c0 = 0; c0 < kHid; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tm + lane + kTdH2 + c0, v);
            for (int q = 0; q < 16; ++q) {
                const int i = c0 + q;
                const float da = bf(s.H2, t, i, kHidHL) > 0.f ? v[q] : 0.f;
                tc::store_bf16(s.DA, t, i, kHid, da);
                tc::store_bf16(s.DAT, i, t, 128, da);
                atomicAdd(&s.gb2[i], da);
            }
        }
        for (int i = 0; i < kHidHL; ++i) tc::store_bf16(s.T, i, t, 128, bf(s.H1, t, i, kHidHL));  // H1^T
        // ---- dH1 = dA2 W2 ; dW2^T += H1^T dA2
        publish_smem();
        if (t == 0) {
            chain(tm + kTdH1, s.DA, kHid, s.W2T, kHid, kHid, kHid, false);
            chain(tm + kTgW2, s.T, 128, s.DAT, 128, 128, kHid, !first);
        }
        if (!(alive = commit_wait(s, phase))) break;
        for (int c0 = 0; c0 < kHid; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tm + lane + kTdH1 + c0, v);
            for (int q = 0; q < 16; ++q) {
                const int i = c0 + q;
                const float da = bf(s.H1, t, i, kHidHL) > 0.f ? v[q] : 0.f;
                tc::store_bf16(s.DAT, i, t, 128, da);
                atomicAdd(&s.gb1[i], da);
            }
        }
        for (int i = 0; i < kInHL; ++i) tc::store_bf16(s.T, i, t, 128, bf(s.X, t, i, kInHL));  // [hi|lo]^T
        // ---- dW1^T += X^T dA1
        publish_smem();
        if (t == 0) chain(tm + kTgW1, s.T, 128, s.DAT, 128, 128, kHid, !first);
        if (!(alive = commit_wait(s, phase))) break;
        first = false;
    }
    // ---- gradients of this CTA to global memory
    if (alive && !first) {
        float v[16];
        // row t = hi (t < 64) or lo (t >= 64) part of input t mod 64 of W3 / W2
        tc::tmem_ld16(tm + lane + kTgW3, v);
        for (int o = 0; o < 3; ++o) atomicAdd(&grad[kOffW3 + o * kHid + (t & 63)], v[o]);
        for (int c0 = 0; c0 < kHid; c0 += 16) {
            tc::tmem_ld16(tm + lane + kTgW2 + c0, v);
            for (int q = 0; q < 16; ++q) atomicAdd(&grad[kOffW2 + (c0 + q) * kHid + (t & 63)], v[q]);
            // rows 0..31 (high parts) and 32..63 (low parts) both feed W1[o][row mod 32]
            tc::tmem_ld16(tm + lane + kTgW1 + c0, v);
            if ((t & 31) < 27 && t < kInHL)
                for (int q = 0; q < 16; ++q) atomicAdd(&grad[kOffW1 + (c0 + q) * kIn + (t & 31)], v[q]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (!first) {
        for (int idx = t; idx < kHid; idx += 128) {
            atomicAdd(&grad[kOffB1 + idx], s.gb1[idx]);
            atomicAdd(&grad[kOffB2 + idx], s.gb2[idx]);
        }
        if (t < 3) atomicAdd(&grad[kOffB3 + t], s.gb3[t]);
        if (t == 0) atomicAdd(loss_sum, s.loss);
    }
    if (t < 32) tc::tmem_dealloc(tm, kTrainCols);
    if (t == 0 && s.timeout) atomicExch(status, 1);
}

// ---------------------------------------------------------------------------
// Adam on the FP32 master weights; writes the BF16/FP32 blob

__global__ void k_adam(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       MlpBlob* __restrict__ blob, float lr, float b1, float b2, float eps, float bc1, float bc2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParam; i += gridDim.x * blockDim.x) {
        // padding entries (W1 columns 27..31, W3 rows 3..15, b3[3..15]) stay zero
        bool pad = (i < kOffW2 && (i % kIn) >= 27) || (i >= kOffW3 && i < kOffB1 && (i - kOffW3) / kHid >= 3) ||
                   (i >= kOffB3 && i - kOffB3 >= 3);
        float gi = pad ? 0.f : g[i];
        float mi = b1 * m[i] + (1.f - b1) * gi;
        float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        float pi = pad ? 0.f : p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        p[i] = pi;
        g[i] = 0.f;
        if (i < kOffW2) blob->W1[i] = __float2bfloat16_rn(pi);
        else if (i < kOffW3) blob->W2[i - kOffW2] = __float2bfloat16_rn(pi);
        else if (i < kOffB1) blob->W3[i - kOffW3] = __float2bfloat16_rn(pi);
        else if (i < kOffB2) blob->b1[i - kOffB1] = pi;
        else if (i < kOffB3) blob->b2[i - kOffB2] = pi;
        else blob->b3[i - kOffB3] = pi;
    }
}

// FP32 parameters -> blob
__global__ void k_params_to_blob(const float* __restrict__ p, MlpBlob* __restrict__ blob) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParam; i += gridDim.x * blockDim.x) {
        float pi = p[i];
        if (i < kOffW2) blob->W1[i] = __float2bfloat16_rn(pi);
        else if (i < kOffW3) blob->W2[i - kOffW2] = __float2bfloat16_rn(pi);
        else if (i < kOffB1) blob->W3[i - kOffW3] = __float2bfloat16_rn(pi);
        else if (i < kOffB2) blob->b1[i - kOffB1] = pi;
        else if (i < kOffB3) blob->b2[i - kOffB2] = pi;
        else blob->b3[i - kOffB3] = pi;
    }
}

// ---------------------------------------------------------------------------
// held-out evaluation: angle (degrees) between target and MLP / MYC normals

// Class of a held-out sample: 0 plane, 1..4 sphere radius in [2,4), [4,8),
// [8,16), [16, inf).
__device__ __forceinline__ int radius_bin(float r) {
    return r <= 0.f ? 0 : (r < 4.f ? 1 : (r < 8.f ? 2 : (r < 16.f ? 3 : 4)));
}

__global__ void k_mlp_eval_angles(const float* __restrict__ st, const float* __restrict__ tgt,
                                  const float* __restrict__ rad, const float* __restrict__ n_mlp, long long n,
                                  float tol, unsigned* __restrict__ hist_mlp, unsigned* __restrict__ hist_myc,
                                  unsigned* __restrict__ hist_cmb, double* __restrict__ sums,
                                  double* __restrict__ bins) {
    double s_mlp = 0.0, s_myc = 0.0, s_cmb = 0.0, s_used = 0.0;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        float sv[27];
        for (int q = 0; q < 27; ++q) sv[q] = st[r * 27 + q];
        float m[3];
        myc_normal(sv, m);
        const float tx = tgt[r * 3], ty = tgt[r * 3 + 1], tz = tgt[r * 3 + 2];
        const float nm = sqrtf(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
        float c1 = (m[0] * tx + m[1] * ty + m[2] * tz) / nm;
        float c2 = n_mlp[r * 3] * tx + n_mlp[r * 3 + 1] * ty + n_mlp[r * 3 + 2] * tz;
        c1 = fminf(1.f, fmaxf(-1.f, c1));
        c2 = fminf(1.f, fmaxf(-1.f, c2));
        const float a1 = acosf(c1) * 57.29577951308232f, a2 = acosf(c2) * 57.29577951308232f;
        // the estimator as the method uses it: the network unless its plane
        // explains the neighbours worse than MYC's and than the tolerance
        const float nn[3] = {n_mlp[r * 3], n_mlp[r * 3 + 1], n_mlp[r * 3 + 2]};
        float mj[3];
        const bool use = judged_normal(sv, nn, tol, mj);
        const float a3 = use ? a2 : a1;
        // per class: count, mean angle of the network, of MYC, of the judged estimator
        double* bq = bins + 4 * radius_bin(rad[r]);
        atomicAdd(bq, 1.0);
        atomicAdd(bq + 1, (double)a2);
        atomicAdd(bq + 2, (double)a1);
        atomicAdd(bq + 3, (double)a3);
        s_myc += a1;
        s_mlp += a2;
        s_cmb += a3;
        s_used += use ? 1.0 : 0.0;
        atomicAdd(&hist_myc[min(17999, (int)(a1 * 100.f))], 1u);
        atomicAdd(&hist_mlp[min(17999, (int)(a2 * 100.f))], 1u);
        atomicAdd(&hist_cmb[min(17999, (int)(a3 * 100.f))], 1u);
    }
    atomicAdd(&sums[0], s_mlp);
    atomicAdd(&sums[1], s_myc);
    atomicAdd(&sums[2], s_cmb);
    atomicAdd(&sums[3], s_used);
}

cudaError_t mlp_grad_pass(const MlpBlob* w, const float* st, const float* tgt, long long n0, long long n,
                          float inv_batch, float* grad, float* loss_sum, int* status, cudaStream_t stream) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(TrainSmem));
    if (e != cudaSuccess) return e;
    long long tiles = (n + 127) / 128;
    int blocks = (int)std::min<long long>(tiles, 148LL);
    k_mlp_train<<<blocks, 128, sizeof(TrainSmem), stream>>>(w, st, tgt, n0, n, inv_batch, grad, loss_sum, status);
    return cudaGetLastError();
}

}  // namespace vof

using namespace vof;

namespace {
__device__ int g_train_status;

int* train_status_ptr() {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_train_status) != cudaSuccess) return nullptr;
    return (int*)p;
}

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

struct TrainLayout {
    size_t st, tgt, test_st, test_tgt, test_n, p, g, m, v, loss, hist, sums, bins, test_rad, total;
};

TrainLayout train_layout(const vof_train_params* tp) {
    TrainLayout L;
    size_t o = 0;
    L.st = o; o = align_up(o + (size_t)tp->n_train * 27 * 4);
    L.tgt = o; o = align_up(o + (size_t)tp->n_train * 3 * 4);
    L.test_st = o; o = align_up(o + (size_t)tp->n_test * 27 * 4);
    L.test_tgt = o; o = align_up(o + (size_t)tp->n_test * 3 * 4);
    L.test_n = o; o = align_up(o + (size_t)tp->n_test * 3 * 4);
    L.p = o; o = align_up(o + kNParam * 4);
    L.g = o; o = align_up(o + kNParam * 4);
    L.m = o; o = align_up(o + kNParam * 4);
    L.v = o; o = align_up(o + kNParam * 4);
    L.loss = o; o = align_up(o + 8);
    L.hist = o; o = align_up(o + 3 * 18000 * 4);
    L.sums = o; o = align_up(o + 4 * 8);
    L.bins = o; o = align_up(o + 5 * 4 * 8);
    L.test_rad = o; o = align_up(o + (size_t)tp->n_test * 4);
    L.total = o;
    return L;
}

bool train_params_valid(const vof_train_params* tp) {
    return tp && tp->n_train >= 128 && tp->n_test >= 0 && tp->epochs >= 1 && tp->batch >= 128 &&
           tp->batch <= (1 << 20) && tp->batch <= tp->n_train && tp->lr > 0.f && tp->plane_fraction >= 0.f && tp->plane_fraction <= 1.f &&
           tp->r_min > 0.f && tp->r_max >= tp->r_min;
}

uint64_t host_mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
}  // namespace

extern "C" vof_status vof_mlp_train_params_default(vof_train_params* tp) {
    if (!tp) return VOF_ERR_ARG;
    tp->n_train = 10000000;
    tp->n_test = 1000000;
    tp->epochs = 4;
    tp->batch = 16384;
    tp->lr = 3e-3f;
    tp->seed = 12345;
    tp->plane_fraction = 0.5f;
    tp->r_min = 2.f;
    tp->r_max = 32.f;
    return VOF_OK;
}

extern "C" size_t vof_mlp_train_workspace_size(const vof_train_params* tp) {
    if (!train_params_valid(tp)) return 0;
    return train_layout(tp).total;
}

extern "C" vof_status vof_mlp_train(const vof_train_params* tp, void* weights_dev, void* workspace_dev,
                                    size_t workspace_bytes, void* stream, vof_train_report* report) {
    if (!train_params_valid(tp) || !weights_dev || !workspace_dev) return VOF_ERR_ARG;
    TrainLayout L = train_layout(tp);
    if (workspace_bytes < L.total) return VOF_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)workspace_dev;
    float* dst = (float*)(ws + L.st);
    float* dtg = (float*)(ws + L.tgt);
    float* tst = (float*)(ws + L.test_st);
    float* ttg = (float*)(ws + L.test_tgt);
    float* tnm = (float*)(ws + L.test_n);
    float* p = (float*)(ws + L.p);
    float* g = (float*)(ws + L.g);
    float* m = (float*)(ws + L.m);
    float* v = (float*)(ws + L.v);
    float* loss = (float*)(ws + L.loss);
    unsigned* hist = (unsigned*)(ws + L.hist);
    double* sums = (double*)(ws + L.sums);
    MlpBlob* blob = (MlpBlob*)weights_dev;
    int* status = train_status_ptr();
    if (!status) return VOF_ERR_CUDA;
#define TRY(x)                               \
    do {                                     \
        if ((x) != cudaSuccess) {            \
            (void)cudaGetLastError();        \
            return VOF_ERR_CUDA;             \
        }                                    \
    } while (0)
    TRY(cudaMemsetAsync(status, 0, 4, st));
    // data
    k_mlp_gen<<<sm_count() * 16, 128, 0, st>>>(dst, dtg, nullptr, tp->n_train, tp->seed, tp->plane_fraction, tp->r_min,
                                        tp->r_max);
    if (tp->n_test > 0)
        k_mlp_gen<<<sm_count() * 16, 128, 0, st>>>(tst, ttg, (float*)(ws + L.test_rad), tp->n_test, host_mix64(tp->seed + 1),
                                            tp->plane_fraction, tp->r_min, tp->r_max);
    TRY(cudaGetLastError());
    // initial weights: He-normal hidden layers (Box-Muller on a counter RNG), zero biases
    std::vector<float> hp(kNParam, 0.f);
    auto gauss = [&](uint64_t i) {
        double u1 = ((host_mix64(tp->seed * 7919ull + 2 * i) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
        double u2 = (host_mix64(tp->seed * 7919ull + 2 * i + 1) >> 11) * (1.0 / 9007199254740992.0);
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    };
    for (int o = 0; o < kHid; ++o)
        for (int i = 0; i < 27; ++i) hp[kOffW1 + o * kIn + i] = (float)(gauss(kOffW1 + o * kIn + i) * std::sqrt(2.0 / 27));
    for (int o = 0; o < kHid; ++o)
        for (int i = 0; i < kHid; ++i)
            hp[kOffW2 + o * kHid + i] = (float)(gauss(kOffW2 + o * kHid + i) * std::sqrt(2.0 / kHid));
    for (int o = 0; o < 3; ++o)
        for (int i = 0; i < kHid; ++i)
            hp[kOffW3 + o * kHid + i] = (float)(gauss(kOffW3 + o * kHid + i) * std::sqrt(1.0 / kHid));
    TRY(cudaMemcpyAsync(p, hp.data(), kNParam * 4, cudaMemcpyHostToDevice, st));
    TRY(cudaMemsetAsync(g, 0, kNParam * 4, st));
    TRY(cudaMemsetAsync(m, 0, kNParam * 4, st));
    TRY(cudaMemsetAsync(v, 0, kNParam * 4, st));
    TRY(cudaMemsetAsync(loss, 0, 8, st));
    k_params_to_blob<<<64, 128, 0, st>>>(p, blob);
    // Adam with cosine learning-rate decay
    const long long nb = tp->n_train / tp->batch;
    const long long total_steps = nb * tp->epochs;
    long long step = 0;
    const float b1 = 0.9f, b2 = 0.999f;
    for (int ep = 0; ep < tp->epochs; ++ep) {
        for (long long b = 0; b < nb; ++b, ++step) {
            TRY(mlp_grad_pass(blob, dst, dtg, b * tp->batch, tp->batch, 1.f / (float)tp->batch, g, loss, status, st));
            const float frac = (float)step / (float)std::max<long long>(1, total_steps - 1);
            const float lr = tp->lr * (0.01f + 0.99f * 0.5f * (1.f + std::cos(3.14159265f * frac)));
            const float bc1 = 1.f - std::pow(b1, (float)(step + 1));
            const float bc2 = 1.f - std::pow(b2, (float)(step + 1));
            k_adam<<<64, 128, 0, st>>>(p, g, m, v, blob, lr, b1, b2, 1e-8f, bc1, bc2);
            TRY(cudaGetLastError());
        }
    }
    // final epoch's mean loss: one more gradient pass over the last batches is
    // not needed; report the loss of the last epoch (accumulated below)
    TRY(cudaMemsetAsync(loss, 0, 8, st));
    TRY(cudaMemsetAsync(g, 0, kNParam * 4, st));
    const long long n_eval = std::min<long long>(tp->n_train, 1 << 20);
    TRY(mlp_grad_pass(blob, dst, dtg, 0, n_eval, 0.f, g, loss, status, st));
    TRY(cudaMemsetAsync(g, 0, kNParam * 4, st));
    float hloss = 0.f;
    TRY(cudaMemcpyAsync(&hloss, loss, 4, cudaMemcpyDeviceToHost, st));
    double hs[4] = {0.0, 0.0, 0.0, 0.0};
    double hb[5][4] = {};
    std::vector<unsigned> hh(54000, 0u);
    if (tp->n_test > 0) {
        int* fstat = status;
        TRY(mlp_forward(blob, tst, tnm, tp->n_test, fstat, st));
        TRY(cudaMemsetAsync(hist, 0, 3 * 18000 * 4, st));
        TRY(cudaMemsetAsync(sums, 0, 32, st));
        TRY(cudaMemsetAsync(ws + L.bins, 0, 5 * 4 * 8, st));
        k_mlp_eval_angles<<<sm_count() * 8, 128, 0, st>>>(tst, ttg, (const float*)(ws + L.test_rad), tnm, tp->n_test,
                                                   1e-3f, hist, hist + 18000, hist + 36000, sums,
                                                   (double*)(ws + L.bins));
        TRY(cudaGetLastError());
        TRY(cudaMemcpyAsync(hs, sums, 32, cudaMemcpyDeviceToHost, st));
        TRY(cudaMemcpyAsync(hb, ws + L.bins, sizeof(hb), cudaMemcpyDeviceToHost, st));
        TRY(cudaMemcpyAsync(hh.data(), hist, 54000 * 4, cudaMemcpyDeviceToHost, st));
    }
    int hstat = 0;
    TRY(cudaMemcpyAsync(&hstat, status, 4, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
#undef TRY
    if (hstat) return VOF_ERR_TIMEOUT;
    if (report) {
        report->final_loss = hloss / (float)n_eval;
        report->steps = (int32_t)total_steps;
        report->test_mean_deg_mlp = tp->n_test ? hs[0] / tp->n_test : 0.0;
        report->test_mean_deg_myc = tp->n_test ? hs[1] / tp->n_test : 0.0;
        auto p95 = [&](const unsigned* h) {
            long long acc = 0, want = (long long)(0.95 * tp->n_test);
            for (int i = 0; i < 18000; ++i) {
                acc += h[i];
                if (acc >= want) return (i + 1) / 100.0;
            }
            return 180.0;
        };
        report->test_p95_deg_mlp = tp->n_test ? p95(hh.data()) : 0.0;
        report->test_p95_deg_myc = tp->n_test ? p95(hh.data() + 18000) : 0.0;
        report->test_mean_deg_combined = tp->n_test ? hs[2] / tp->n_test : 0.0;
        report->test_p95_deg_combined = tp->n_test ? p95(hh.data() + 36000) : 0.0;
        report->test_network_share = tp->n_test ? hs[3] / tp->n_test : 0.0;
        for (int b = 0; b < 5; ++b) {
            const double cnt = hb[b][0];
            report->bin_count[b] = (int64_t)cnt;
            report->bin_mean_deg_mlp[b] = cnt > 0 ? hb[b][1] / cnt : 0.0;
            report->bin_mean_deg_myc[b] = cnt > 0 ? hb[b][2] / cnt : 0.0;
            report->bin_mean_deg_combined[b] = cnt > 0 ? hb[b][3] / cnt : 0.0;
        }
    }
    return VOF_OK;
}

extern "C" vof_status vof_mlp_grad(const void* weights_dev, const float* stencils_dev, const float* targets_dev,
                                   int64_t n, float* grad_dev, float* loss_dev, void* stream) {
    if (!weights_dev || !stencils_dev || !targets_dev || !grad_dev || !loss_dev || n < 1) return VOF_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int* status = train_status_ptr();
    if (!status) return VOF_ERR_CUDA;
    if (cudaMemsetAsync(status, 0, 4, st) != cudaSuccess || cudaMemsetAsync(grad_dev, 0, kNParam * 4, st) != cudaSuccess ||
        cudaMemsetAsync(loss_dev, 0, 4, st) != cudaSuccess ||
        mlp_grad_pass((const MlpBlob*)weights_dev, stencils_dev, targets_dev, 0, n, 1.f / (float)n, grad_dev, loss_dev,
                      status, st) != cudaSuccess) {
        (void)cudaGetLastError();
        return VOF_ERR_CUDA;
    }
    int h = 0;
    if (cudaMemcpyAsync(&h, status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        (void)cudaGetLastError();
        return VOF_ERR_CUDA;
    }
    return h ? VOF_ERR_TIMEOUT : VOF_OK;
}

extern "C" vof_status vof_mlp_params_to_weights(const float* params_dev, void* weights_dev, void* stream) {
    if (!params_dev || !weights_dev) return VOF_ERR_ARG;
    k_params_to_blob<<<64, 128, 0, (cudaStream_t)stream>>>(params_dev, (MlpBlob*)weights_dev);
    if (cudaGetLastError() != cudaSuccess) return VOF_ERR_CUDA;
    return VOF_OK;
}
