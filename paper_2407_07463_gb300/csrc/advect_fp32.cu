// FP32 instantiation of the split advection sweeps (mixed precision: float
// storage, normals and fluxes; the plane constant is refined in double for
// c < band or c > 1 - band).
#include "advect_impl.cuh"

namespace vof {
cudaError_t advect_steps_fp32(AdvectArgs& a, int nsteps) { return advect_steps_t<float>(a, nsteps); }
}  // namespace vof
