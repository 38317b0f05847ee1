// Instantiation of the finite-volume stage kernels for SRHD.
#include "dh_fv_stage.cuh"

namespace dh {

dh_status fv_launch_srhd(dh_plan* plan, const FvArgs& A, int wmode, cudaStream_t stream) {
  return fv_launch_pde<PdeSRHD>(plan, A, wmode, stream);
}

}  // namespace dh
