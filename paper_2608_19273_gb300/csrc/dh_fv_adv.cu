// Instantiation of the finite-volume stage kernels for the advection systems.
#include "dh_fv_stage.cuh"

namespace dh {

dh_status fv_launch_adv_flux(dh_plan* plan, const FvArgs& A, int wmode, cudaStream_t stream) {
  return fv_launch_pde<PdeAdvFlux>(plan, A, wmode, stream);
}

dh_status fv_launch_adv_ncp(dh_plan* plan, const FvArgs& A, int wmode, cudaStream_t stream) {
  return fv_launch_pde<PdeAdvNcp>(plan, A, wmode, stream);
}

}  // namespace dh
