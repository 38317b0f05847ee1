// Instantiation of the finite-volume stage kernels for 2D Euler.
#include "dh_fv_stage.cuh"

namespace dh {

dh_status fv_launch_euler2(dh_plan* plan, const FvArgs& A, int wmode, cudaStream_t stream) {
  return fv_launch_pde<PdeEuler2>(plan, A, wmode, stream);
}

}  // namespace dh
