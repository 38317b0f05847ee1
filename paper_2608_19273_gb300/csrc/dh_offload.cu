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
//   dh_offload_bind_staged: for page-locked host blocks that lie in one span of
//     host memory: the run copies that span to a device staging buffer with
//     one cudaMemcpyAsync (the copy engine, no SM time, so a second problem's
//     kernels can run meanwhile), gathers from the staged copy at HBM speed,
//     scatters into it and copies the span back with one cudaMemcpyAsync.
//   dh_offload_run : gather (all nq quantities of every interior voxel) ->
//     n_steps Runge-Kutta steps on the device arena -> scatter of the first
//     nq_back quantities, all asynchronous on one stream.
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <vector>

#include "dh_internal.cuh"

using namespace dh;

extern "C" {

dh_status dh_offload_bind(dh_plan* plan, const double* const* blocks, int32_t nq, int32_t aos_halo) {
  if (!plan) { set_error("plan is NULL"); return DH_EINVAL; }
  plan->offload_nq = 0;  // a failed bind leaves the plan unbound
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
  // (a copy from pageable memory may return before the device holds it: wait, a run may
  // follow on a non-blocking stream)
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e != cudaSuccess) return cuda_error(e, "dh_offload_bind: table upload");
  plan->offload_nq = nq;
  plan->offload_halo = aos_halo;
  plan->offload_staged = false;
  return DH_OK;
}

dh_status dh_offload_bind_staged(dh_plan* plan, const double* const* blocks, int32_t nq, int32_t aos_halo) {
  dh_status st = dh_offload_bind(plan, blocks, nq, aos_halo);  // validation and the in-place table
  if (st != DH_OK) return st;
  plan->offload_nq = 0;  // unbound until the staged table is in place (a failed bind leaves no binding)
  uintptr_t lo = UINTPTR_MAX, hi = 0;
  size_t total = 0;
  std::vector<double*> staged(plan->K);
  for (int k = 0; k < plan->K; ++k) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, blocks[k]) != cudaSuccess || at.type != cudaMemoryTypeHost) {
      cudaGetLastError();
      set_error("dh_offload_bind_staged: block %d is not page-locked host memory", k);
      return DH_EINVAL;
    }
    const int p = plan->h_patches[k].p, n = p + 2 * aos_halo;
    const size_t bytes = sizeof(double) * (size_t)nq * (size_t)n * (size_t)n * (size_t)(plan->dim == 3 ? n : 1);
    lo = std::min(lo, (uintptr_t)blocks[k]);
    hi = std::max(hi, (uintptr_t)blocks[k] + bytes);
    total += bytes;
  }
  const size_t span = hi - lo;
  if (span > 4 * total) {
    set_error("dh_offload_bind_staged: the blocks span %zu bytes for %zu bytes of blocks (more than 4x); "
              "use dh_offload_bind", span, total);
    return DH_EINVAL;
  }
  if (plan->stage_cap < span) {
    if (plan->d_stage) cudaFree(plan->d_stage);
    plan->d_stage = nullptr;
    plan->stage_cap = 0;
    cudaError_t e = cudaMalloc(&plan->d_stage, span);
    if (e != cudaSuccess) { plan->d_stage = nullptr; return cuda_error(e, "dh_offload_bind_staged: staging buffer"); }
    plan->stage_cap = span;
  }
  for (int k = 0; k < plan->K; ++k)
    staged[k] = reinterpret_cast<double*>(plan->d_stage + ((uintptr_t)blocks[k] - lo));
  cudaError_t e = cudaMemcpy(plan->d_offload, staged.data(), sizeof(double*) * plan->K, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e != cudaSuccess) return cuda_error(e, "dh_offload_bind_staged: table upload");
  plan->stage_host = reinterpret_cast<char*>(lo);
  plan->stage_bytes = span;
  plan->offload_staged = true;
  plan->offload_nq = nq;
  return DH_OK;
}

dh_status dh_offload_run(dh_plan* plan, int32_t scheme, int32_t rk, int32_t n_steps, double* arena, double* u1,
                         double* u2, double* acc, double* dt_dev, double* lam_dev, double cfl, double sigma_ko,
                         int32_t nq_back, void* stream) {
  if (!plan) { set_error("plan is NULL"); return DH_EINVAL; }
  if (!plan->d_offload || plan->offload_nq <= 0) {
    set_error("dh_offload_run: no blocks bound (dh_offload_bind or a successful dh_offload_bind_staged)");
    return DH_EINVAL;
  }
  if (!arena || ((uintptr_t)arena & 7) != 0) { set_error("dh_offload_run: arena is NULL or misaligned"); return DH_EINVAL; }
  if (n_steps < 0 || n_steps > 1000000) { set_error("dh_offload_run: n_steps out of range"); return DH_EINVAL; }
  if (nq_back < 0 || nq_back > plan->offload_nq) { set_error("dh_offload_run: nq_back outside [0, nq]"); return DH_EINVAL; }
  if (cfl > 0 && !lam_dev) { set_error("dh_offload_run: cfl > 0 needs lam_dev"); return DH_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  const int nq = plan->offload_nq, h = plan->offload_halo;
  double* mat = plan->nm > 0 ? arena + (int64_t)plan->nq * plan->var_stride : nullptr;
  nvtxRangePushA("dh offload gather");
  if (plan->offload_staged) {
    cudaError_t e = cudaMemcpyAsync(plan->d_stage, plan->stage_host, plan->stage_bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { nvtxRangePop(); return cuda_error(e, "dh_offload_run: staging copy in"); }
  }
  dh_status st = aoas_move(plan, true, plan->d_offload, nq, 0, nq, h, arena, s);
  nvtxRangePop();
  if (st != DH_OK) return st;
  if (n_steps > 0 && cfl > 0 && plan->pde != DH_PDE_SRHD3D) {
    // the first step's dt needs the wave speed of the gathered state
    st = max_wave_speed(plan, arena, mat, lam_dev, stream);
    if (st != DH_OK) return st;
  }
  // the steps as a captured graph would run them (derived quantities handed between stages)
  if (n_steps > 0) {
    st = rk_steps(plan, scheme, rk, n_steps, arena, u1, u2, acc, mat, dt_dev, lam_dev, cfl, sigma_ko, s);
    if (st != DH_OK) return st;
  }
  nvtxRangePushA("dh offload scatter");
  if (nq_back > 0) st = aoas_move(plan, false, plan->d_offload, nq, 0, nq_back, h, arena, s);
  if (st == DH_OK && plan->offload_staged && nq_back > 0)
    st = cuda_error(cudaMemcpyAsync(plan->stage_host, plan->d_stage, plan->stage_bytes, cudaMemcpyDeviceToHost, s),
                    "dh_offload_run: staging copy out");
  nvtxRangePop();
  return st;
}

}  // extern "C"
