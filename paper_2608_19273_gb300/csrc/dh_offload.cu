// Offload mode: the paper's batched kernel with host-resident patch data.
//
// The paper's generated code takes K patches in the AoAoS layout on the host,
// gathers them into one linear space, moves that to the GPU, runs the
// composed cell kernel, and scatters the outcome back (Sec. III-C Eq. 4 with
// the host-to-device memory-space pass of Sec. III-D; total versus compute
// time is what Sec. IV compares).  On GB300 the host's page-locked memory is
// directly addressable by the GPU over NVLink-C2C, so the gather prologue and
// the scatter epilogue here ARE the host<->device transfer: the AoAoS kernels
// read the caller's page-locked blocks in place and write the outcome back in
// place, with no staging copy.
//
//   dh_offload_bind: validates that each of the K block pointers is device
//     accessible (device, managed, or page-locked host memory) and keeps a
//     device copy of the pointer table in the plan.
//   dh_offload_run : gather (all nq quantities of every interior voxel) ->
//     n_steps Runge-Kutta steps on the device arena -> scatter of the first
//     nq_back quantities, all asynchronous on one stream.
#include <nvtx3/nvToolsExt.h>

#include "dh_internal.cuh"

using namespace dh;

extern "C" {

dh_status dh_offload_bind(dh_plan* plan, const double* const* blocks, int32_t nq, int32_t aos_halo) {
  if (!plan) { set_error("plan is NULL"); return DH_EINVAL; }
  if (!blocks) { set_error("dh_offload_bind: blocks is NULL"); return DH_EINVAL; }
  if (nq < 1 || nq > 256) { set_error("dh_offload_bind: nq = %d outside [1, 256]", nq); return DH_EINVAL; }
  if (nq < plan->nq + plan->nm) {
    set_error("dh_offload_bind: nq = %d is smaller than the PDE's N + M = %d", nq, plan->nq + plan->nm);
    return DH_EINVAL;
  }
  if (aos_halo < 0 || aos_halo > 8) { set_error("dh_offload_bind: aos_halo = %d outside [0, 8]", aos_halo); return DH_EINVAL; }
  for (int k = 0; k < plan->K; ++k) {
    const double* b = blocks[k];
    if (!b || ((uintptr_t)b & 7) != 0) { set_error("dh_offload_bind: block %d is NULL or not 8-byte aligned", k); return DH_EINVAL; }
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, b);
    if (e != cudaSuccess) { cudaGetLastError(); set_error("dh_offload_bind: block %d: pointer query failed", k); return DH_EINVAL; }
    const bool ok = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged ||
                    (at.type == cudaMemoryTypeHost && at.devicePointer == (const void*)b);
    if (!ok) {
      set_error("dh_offload_bind: block %d is not device accessible (pageable host memory? use page-locked memory)", k);
      return DH_EINVAL;
    }
  }
  if (!plan->d_offload) {
    cudaError_t e = cudaMalloc(&plan->d_offload, sizeof(double*) * plan->K);
    if (e != cudaSuccess) { plan->d_offload = nullptr; return cuda_error(e, "dh_offload_bind: cudaMalloc"); }
  }
  cudaError_t e = cudaMemcpy(plan->d_offload, blocks, sizeof(double*) * plan->K, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_error(e, "dh_offload_bind: table upload");
  plan->offload_nq = nq;
  plan->offload_halo = aos_halo;
  return DH_OK;
}

dh_status dh_offload_run(dh_plan* plan, int32_t scheme, int32_t rk, int32_t n_steps, double* arena, double* u1,
                         double* u2, double* acc, double* dt_dev, double* lam_dev, double cfl, double sigma_ko,
                         int32_t nq_back, void* stream) {
  if (!plan) { set_error("plan is NULL"); return DH_EINVAL; }
  if (!plan->d_offload) { set_error("dh_offload_run: no blocks bound (dh_offload_bind)"); return DH_EINVAL; }
  if (!arena || ((uintptr_t)arena & 7) != 0) { set_error("dh_offload_run: arena is NULL or misaligned"); return DH_EINVAL; }
  if (n_steps < 0 || n_steps > 1000000) { set_error("dh_offload_run: n_steps out of range"); return DH_EINVAL; }
  if (nq_back < 0 || nq_back > plan->offload_nq) { set_error("dh_offload_run: nq_back outside [0, nq]"); return DH_EINVAL; }
  if (cfl > 0 && !lam_dev) { set_error("dh_offload_run: cfl > 0 needs lam_dev"); return DH_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  const int nq = plan->offload_nq, h = plan->offload_halo;
  double* mat = plan->nm > 0 ? arena + (int64_t)plan->nq * plan->var_stride : nullptr;
  nvtxRangePushA("dh offload gather");
  dh_status st = aoas_move(plan, true, plan->d_offload, nq, 0, nq, h, arena, s);
  nvtxRangePop();
  if (st != DH_OK) return st;
  if (n_steps > 0 && cfl > 0 && plan->pde != DH_PDE_SRHD3D) {
    // the first step's dt needs the wave speed of the gathered state
    st = max_wave_speed(plan, arena, mat, lam_dev, stream);
    if (st != DH_OK) return st;
  }
  for (int i = 0; i < n_steps; ++i) {
    st = dh_rk_step(plan, scheme, rk, arena, u1, u2, acc, mat, dt_dev, lam_dev, cfl, sigma_ko, stream);
    if (st != DH_OK) return st;
  }
  nvtxRangePushA("dh offload scatter");
  if (nq_back > 0) st = aoas_move(plan, false, plan->d_offload, nq, 0, nq_back, h, arena, s);
  nvtxRangePop();
  return st;
}

}  // extern "C"
