// FP64 instantiation of the split advection sweeps.  Built with -fmad=false
// so that every product and sum rounds separately, as the plain FP64 method
// states them.
#include "advect_impl.cuh"

namespace vof {
cudaError_t advect_steps_fp64(AdvectArgs& a, int nsteps) { return advect_steps_t<double>(a, nsteps); }
}  // namespace vof
