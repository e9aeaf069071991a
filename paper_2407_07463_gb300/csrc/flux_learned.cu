// Face fluxes of one split sweep with the learned normal (FP32 path; the
// normal estimator itself has no counterpart in the paper, the fluxes are
// those of Section 2.2).
//
// A CTA of 128 threads takes 128 listed faces at a time.  Each thread
// gathers the 3x3x3 stencil of its face's upwind donor and writes the
// canonical input row; the CTA runs the network on the tensor cores; each
// thread maps its output back and judges it: the network's normal is kept
// when its plane explains the stencil with a mean residual of at most `tol`,
// or no worse than MYC's plane does, otherwise MYC's normal is used.  Then
// the plane constant (FP64 refinement near c = 0 or 1) and the PLIC volume
// of the swept sub-cell, as in the MYC path.
#include "advect_impl.cuh"
#include "mlp.cuh"
#include "mlp_tile.cuh"

namespace vof {

__global__ void __launch_bounds__(128, 3) k_face_flux_learned(const float* __restrict__ cin,
                                                              const float* __restrict__ ud, Dims g, int d,
                                                              float sfac, float band,
                                                              const unsigned long long* __restrict__ list,
                                                              long long cap, const int* __restrict__ off, int nseg,
                                                              float* __restrict__ flux,
                                                              const MlpBlob* __restrict__ w, float tol,
                                                              int* __restrict__ status,
                                                              unsigned long long* __restrict__ counters) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    MlpSmem& s = *reinterpret_cast<MlpSmem*>(smem_raw);
    mlp_cta_begin(s, w);
    const uint32_t taddr = s.tbase;
    uint32_t phase = 0;
    const int t = threadIdx.x;
    const int n = off[nseg];
    unsigned n_net = 0, n_myc = 0;
    // the loop bound is the same for every thread of the CTA
    for (int base = blockIdx.x * 128; base < n; base += gridDim.x * 128) {
        const int e = base + t;
        const bool valid = e < n;
        float st[27];
        float sv = 0.f;
        size_t fi = 0;
        if (valid) {
            const int sgi = segment_of(off, nseg, e);
            const unsigned long long key = list[(size_t)sgi * cap + (e - off[sgi])];
            const int f = (int)(key >> 54);
            const int k = (int)((key >> 36) & 0x3ffffu);
            const int j = (int)((key >> 18) & 0x3ffffu);
            const int i = (int)(key & 0x3ffffu);
            const int x = cell(i, j, k, g);
            fi = (size_t)f * g.N + x;
            const float uv = ud[x];
            sv = uv * sfac;
            const int donor = vsign(uv) > 0 ? step_cell(x, i, j, k, d, -1, g) : x;
            gather_stencil(cin + (size_t)f * g.N, donor, g, st);
        } else {
#pragma unroll
            for (int q = 0; q < 27; ++q) st[q] = 0.5f;
        }
        CanonFrame fr;
        canon_frame(st, fr);
        float x[27];
        canon_input(st, fr, x);
        store_input_row(s, t, x);
        float oc[3];
        if (!mlp_tile_forward(s, taddr, phase, oc)) break;
        if (valid) {
            float nn[3];
            canon_output(oc, fr, nn);
            float m[3];
            if (judged_normal(st, nn, tol, m))
                ++n_net;
            else
                ++n_myc;
            const float alpha = plic_alpha_banded(m[0], m[1], m[2], st[13], band);
            flux[fi] = face_flux(m, alpha, d, sv);
        }
    }
    n_net = __reduce_add_sync(0xffffffffu, n_net);
    n_myc = __reduce_add_sync(0xffffffffu, n_myc);
    if ((t & 31) == 0 && counters) {
        if (n_net) atomicAdd(&counters[0], (unsigned long long)n_net);
        if (n_myc) atomicAdd(&counters[1], (unsigned long long)n_myc);
    }
    mlp_cta_end(s, status);
}

void face_flux_learned(const float* cin, const float* ud, const Dims& g, int d, float sfac, float band,
                       const unsigned long long* list, long long cap, const int* off, int nseg, float* flux,
                       const MlpBlob* w, float tol, int* status, unsigned long long* counters, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_face_flux_learned, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpSmem));
        attr = true;
    }
    k_face_flux_learned<<<152 * 3, 128, sizeof(MlpSmem), st>>>(cin, ud, g, d, sfac, band, list, cap, off, nseg, flux,
                                                                w, tol, status, counters);
}

}  // namespace vof
