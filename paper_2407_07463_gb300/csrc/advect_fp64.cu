// FP64 instantiation of the split advection sweeps.  Built with -fmad=false
// so that every product and sum rounds separately, as the plain FP64 method
// states them.
#include "advect_impl.cuh"

namespace vof {
cudaError_t advect_set_fp64(const BoxSet<double, 1>& S, SweepArgs& a, int nsteps) { return advect_set(S, a, nsteps); }
cudaError_t advect_set_fp64(const BoxSet<double, kMaxBoxes>& S, SweepArgs& a, int nsteps) {
    return advect_set(S, a, nsteps);
}
int update_occupancy_fp64(int warps) { return update_blocks_per_sm<double, kMaxBoxes>(warps); }
cudaError_t advect_first_sweep_fp64(const BoxSet<double, kMaxBoxes>& S, SweepArgs& a) {
    return advect_first_sweep(S, a);
}
cudaError_t patch_list_fp64(const BoxSet<double, 1>& S, SweepArgs& a, int d, const uint32_t* bits, const int* labels,
                          const MoveTables& mt, const int* target) {
    return patch_list_set(S, a, d, bits, labels, mt, target);
}
}  // namespace vof
