// FP32 instantiation of the split advection sweeps (mixed precision: float
// storage, normals and fluxes; the plane constant is refined in double for
// c < band or c > 1 - band).
#include "advect_impl.cuh"

namespace vof {
cudaError_t advect_set_fp32(const BoxSet<float, 1>& S, SweepArgs& a, int nsteps) { return advect_set(S, a, nsteps); }
cudaError_t advect_set_fp32(const BoxSet<float, kMaxBoxes>& S, SweepArgs& a, int nsteps) {
    return advect_set(S, a, nsteps);
}
int update_occupancy(bool fp64, int warps) {
    return fp64 ? update_occupancy_fp64(warps) : update_blocks_per_sm<float, kMaxBoxes>(warps);
}
cudaError_t advect_first_sweep_fp32(const BoxSet<float, kMaxBoxes>& S, SweepArgs& a) {
    return advect_first_sweep(S, a);
}
cudaError_t patch_list_fp32(const BoxSet<float, 1>& S, SweepArgs& a, int d, const uint32_t* bits, const int* labels,
                          const MoveTables& mt, const int* target) {
    return patch_list_set(S, a, d, bits, labels, mt, target);
}
}  // namespace vof
