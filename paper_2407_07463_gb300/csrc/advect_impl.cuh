// Directionally split geometric advection of K colour fields, one sweep per
// three launches (Section 2.2 transport of every C_i, Section 2.3 "we solve
// N(t) transport equations"):
//   1. find_faces: list the faces whose upwind donor is interfacial
//      (0 < c < 1) -- compaction keeps the costly reconstruction on full
//      warps (FP64 issues at a small fraction of the FP32 rate on GB300);
//   2. face_flux: per listed face, MYC normal + plane constant of the donor
//      and the PLIC volume of the swept sub-cell;
//   3. update: c <- c - (F_hi - F_lo) + c_c (s_hi - s_lo) with c_c = [c^n > 1/2]
//      (Weymouth & Yue 2010); empty/full donors give F = 0 / s without
//      reconstruction; after the third sweep the result is clipped to [0,1].
#pragma once

#include "common.cuh"
#include "internal.h"
#include "plic.cuh"

namespace vof {

struct AdvectArgs {
    Dims g;
    int K;                       // fields advected (the active ones)
    void* c;                     // [K][N] state, updated in place
    const void* u;               // [3][N]
    void* buf1;                  // [K][N] scratch
    void* buf2;                  // [K][N] scratch
    void* flux;                  // [K][N] scratch (interfacial faces only)
    unsigned long long* list;    // [K*N] scratch
    unsigned long long* counter; // 1 scratch word
    double* clipped;             // [K] accumulated clip volume
    double dt, h;
    long long step;
    double band;
    cudaStream_t stream;
    long long* launches;
    Prof* prof;
};

template <typename T>
__global__ void __launch_bounds__(256) k_find_faces(const T* __restrict__ cin, const T* __restrict__ ud,
                                                    Dims g, int K, int d,
                                                    unsigned long long* __restrict__ list,
                                                    unsigned long long* __restrict__ count) {
    long long total = (long long)K * g.N;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += stride) {
        long long t = base + threadIdx.x;
        bool flag = false;
        if (t < total) {
            int f = (int)(t / g.N);
            int x = (int)(t - (long long)f * g.N);
            int sg = vsign(ud[x]);
            if (sg != 0) {
                int i, j, k;
                decode(x, g, i, j, k);
                int donor = sg > 0 ? step_cell(x, i, j, k, d, -1, g) : x;
                flag = vclass(cin[(size_t)f * g.N + donor]) == 1;
            }
        }
        long long slot = warp_append(flag, count);
        if (slot >= 0) list[slot] = (unsigned long long)t;
    }
}

template <typename T>
__device__ __forceinline__ void gather_stencil(const T* __restrict__ cf, int x, const Dims& g, T st[27]) {
    int i, j, k;
    decode(x, g, i, j, k);
    int im = i == 0 ? g.nx - 1 : i - 1, ip = i == g.nx - 1 ? 0 : i + 1;
    int jm = j == 0 ? g.ny - 1 : j - 1, jp = j == g.ny - 1 ? 0 : j + 1;
    int km = k == 0 ? g.nz - 1 : k - 1, kp = k == g.nz - 1 ? 0 : k + 1;
    const int is[3] = {im, i, ip}, js[3] = {jm, j, jp}, ks[3] = {km, k, kp};
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) st[c * 9 + b * 3 + a] = cf[cell(is[a], js[b], ks[c], g)];
}

template <typename T>
__global__ void __launch_bounds__(128) k_face_flux(const T* __restrict__ cin, const T* __restrict__ ud,
                                                   Dims g, int d, T sfac, T band,
                                                   const unsigned long long* __restrict__ list,
                                                   const unsigned long long* __restrict__ count,
                                                   T* __restrict__ flux) {
    unsigned long long n = *count;
    for (unsigned long long idx = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (unsigned long long)gridDim.x * blockDim.x) {
        unsigned long long t = list[idx];
        int f = (int)(t / (unsigned long long)g.N);
        int x = (int)(t - (unsigned long long)f * g.N);
        T uv = ud[x];
        T s = uv * sfac;
        int i, j, k;
        decode(x, g, i, j, k);
        int donor = vsign(uv) > 0 ? step_cell(x, i, j, k, d, -1, g) : x;
        const T* cf = cin + (size_t)f * g.N;
        T st[27];
        gather_stencil(cf, donor, g, st);
        T m[3];
        myc_normal(st, m);
        T alpha = plic_alpha_banded(m[0], m[1], m[2], st[13], band);
        flux[t] = face_flux(m, alpha, d, s);
    }
}

template <typename T>
__device__ __forceinline__ T face_value(int kind, T s, const T* __restrict__ flux, size_t t) {
    return kind == 0 ? T(0) : (kind == 2 ? s : flux[t]);
}

template <typename T>
__global__ void __launch_bounds__(256) k_update(const T* __restrict__ cin, const T* cstart, T* cout,
                                                const T* __restrict__ ud, Dims g, int K, int d,
                                                T sfac, const T* __restrict__ flux, int clip,
                                                double* __restrict__ clipped) {
    long long total = (long long)K * g.N;
    long long stride = (long long)gridDim.x * blockDim.x;
    double removed = 0.0;
    int fcur = -1;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        int f = (int)(t / g.N);
        int x = (int)(t - (long long)f * g.N);
        if (clip && f != fcur) {
            if (fcur >= 0 && removed != 0.0) atomicAdd(&clipped[fcur], removed);
            removed = 0.0;
            fcur = f;
        }
        int i, j, k;
        decode(x, g, i, j, k);
        int xh = step_cell(x, i, j, k, d, +1, g);
        size_t base = (size_t)f * g.N;
        T u_lo = ud[x], u_hi = ud[xh];
        T cx = cin[base + x];
        int sl = vsign(u_lo), sh = vsign(u_hi);
        int kl = 0, kh = 0;
        if (sl > 0) kl = vclass(cin[base + step_cell(x, i, j, k, d, -1, g)]);
        else if (sl < 0) kl = vclass(cx);
        if (sh > 0) kh = vclass(cx);
        else if (sh < 0) kh = vclass(cin[base + xh]);
        bool cc = above_half(cstart[base + x]);
        T v;
        if (kl == 0 && kh == 0 && !cc && is_exact_zero(cx)) {
            v = cx;
        } else {
            T s_lo = u_lo * sfac, s_hi = u_hi * sfac;
            T F_lo = face_value(kl, s_lo, flux, base + x);
            T F_hi = face_value(kh, s_hi, flux, base + xh);
            T ccv = cc ? T(1) : T(0);
            v = cx - (F_hi - F_lo) + ccv * (s_hi - s_lo);
            if (clip) {
                T cl = v < T(0) ? T(0) : (v > T(1) ? T(1) : v);
                removed += (double)v - (double)cl;
                v = cl;
            }
        }
        cout[base + x] = v;
    }
    if (clip && fcur >= 0 && removed != 0.0) atomicAdd(&clipped[fcur], removed);
}

template <typename T>
cudaError_t advect_steps_t(const AdvectArgs& a, int nsteps) {
    const Dims& g = a.g;
    long long total = (long long)a.K * g.N;
    if (total == 0 || nsteps <= 0) return cudaSuccess;
    T sfac = (T)(a.dt / a.h);
    T band = (T)a.band;
    const T* u = (const T*)a.u;
    T* c = (T*)a.c;
    T* b1 = (T*)a.buf1;
    T* b2 = (T*)a.buf2;
    T* fl = (T*)a.flux;
    int gu = grid_for(total, 256);
    int gf = 152 * 8;
    for (int s = 0; s < nsteps; ++s) {
        long long step = a.step + s;
        int rot = (int)(step % 3);
        const T* ins[3] = {c, b1, b2};
        T* outs[3] = {b1, b2, c};
        for (int sw = 0; sw < 3; ++sw) {
            int d = (rot + sw) % 3;
            const T* ud = u + (size_t)d * g.N;
            cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), a.stream);
            if (a.prof) a.prof->begin(P_FIND_FACES);
            k_find_faces<T><<<gu, 256, 0, a.stream>>>(ins[sw], ud, g, a.K, d, a.list, a.counter);
            if (a.prof) { a.prof->end(); a.prof->begin(P_FACE_FLUX); }
            k_face_flux<T><<<gf, 128, 0, a.stream>>>(ins[sw], ud, g, d, sfac, band, a.list, a.counter, fl);
            if (a.prof) { a.prof->end(); a.prof->begin(P_UPDATE); }
            k_update<T><<<gu, 256, 0, a.stream>>>(ins[sw], c, outs[sw], ud, g, a.K, d, sfac, fl,
                                                   sw == 2, a.clipped);
            if (a.prof) a.prof->end();
            if (a.launches) *a.launches += 3;
        }
    }
    return cudaGetLastError();
}

}  // namespace vof
