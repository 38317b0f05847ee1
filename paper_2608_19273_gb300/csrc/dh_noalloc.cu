// patch_update_fv_noalloc: the finite-volume stage for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not
// wanted -- inside a host framework whose memory pool owns the whole device,
// in plugin hosts that forbid device allocations after start-up, or in
// real-time loops that must never block on the allocator.  Such callers
// cannot build a dh_plan, because a plan allocates its patch table, work list
// and reduction slots with cudaMalloc.
//
// What it does instead: the tables and the reduction slots live in one
// file-scope __device__ array (NA_SCRATCH_BYTES, below), which every GPU that
// loads this library holds until the process exits.  Each call validates the
// patch list like dh_plan_create (same-level neighbours only: coupled
// refinement levels are not supported here), copies it and the tile work list
// it builds into static host buffers, uploads both into the device array with
// cudaMemcpyAsync from those pageable buffers (staged by the driver before the
// call returns, so the caller's table is free again on return), clears the
// two reduction slots with cudaMemsetAsync, and launches the same stage
// kernel as patch_update_fv.  It calls no cudaMalloc, cudaFree or other
// allocating routine.
//
// Every call shares the one device array and overwrites what the previous
// call left there; calls that overlap on the GPU (different streams, or
// different host threads without ordering) race on it.  The first call on a
// device looks up the array's device address with cudaGetSymbolAddress while
// that device is current; make that first call before any stream capture.
#include <cstring>
#include <mutex>

#include "dh_internal.cuh"

namespace dh {
namespace {

constexpr int NA_MAX_PATCHES = 8192;
constexpr int NA_MAX_WORK = 16384;
constexpr size_t NA_RED_BYTES = 256;
constexpr size_t NA_PATCH_BYTES = sizeof(dh_patch) * NA_MAX_PATCHES;
constexpr size_t NA_WORK_BYTES = sizeof(Work) * NA_MAX_WORK;
constexpr size_t NA_SCRATCH_BYTES = NA_RED_BYTES + NA_PATCH_BYTES + NA_WORK_BYTES;
// the size the header states (72-byte patch records, 44-byte work items)
static_assert(sizeof(dh_patch) == 72 && sizeof(Work) == 44, "record sizes changed: update the stated size");
static_assert(NA_SCRATCH_BYTES == 1310976, "scratch size changed: update the header");
static_assert(dh_plan::NRED * sizeof(unsigned long long) <= NA_RED_BYTES, "reduction slots do not fit");

static __device__ __align__(256) unsigned char g_na_scratch[NA_SCRATCH_BYTES];

static std::mutex g_na_mutex;
// host staging of the patch table and the work list (static, not heap): every upload reads
// the library's own pageable copy, so the caller's array is free again when the call returns,
// even when it is page-locked (a copy from page-locked memory would still be in flight)
static dh_patch g_na_patches[NA_MAX_PATCHES];
static Work g_na_work[NA_MAX_WORK];
constexpr int NA_MAX_DEVICES = 64;
static unsigned char* g_na_addr[NA_MAX_DEVICES] = {nullptr};

// Same checks as dh_plan_create; returns the number of work items or a status < 0.
int na_build_work(int dim, const dh_patch* patches, int K, int halo, int64_t var_stride, bool* has_cls) {
  for (int k = 0; k < K; ++k) {
    const dh_patch& pt = patches[k];
    if (pt.p < 8 || pt.p % 8 != 0 || pt.p > 256) { set_error("patch %d: p = %d must be a multiple of 8 in [8, 256]", k, pt.p); return DH_EINVAL; }
    if (pt.p < halo) { set_error("patch %d: p smaller than the halo", k); return DH_EINVAL; }
    if (!(pt.dx > 0.0)) { set_error("patch %d: dx must be positive", k); return DH_EINVAL; }
    const int64_t n = dim == 3 ? (int64_t)pt.p * pt.p * pt.p : (int64_t)pt.p * pt.p;
    if (pt.offset < 0 || pt.offset % 16 != 0 || pt.offset + n > var_stride) { set_error("patch %d: bad offset", k); return DH_EINVAL; }
    for (int f = 0; f < 2 * dim; ++f) {
      const int nb = pt.nbr[f];
      if (nb < 0 || nb >= K || patches[nb].p != pt.p || patches[nb].dx != pt.dx) {
        set_error("patch %d: neighbour %d invalid or of different size", k, f);
        return DH_EINVAL;
      }
    }
  }
  // 16x16 columns first (largest work), then groups of four 8x8 columns of equal p.
  int nw = 0;
  has_cls[0] = has_cls[1] = false;
  for (int k = 0; k < K; ++k) {
    const int p = patches[k].p;
    if (p % 16 != 0) continue;
    for (int yy = 0; yy < p; yy += 16)
      for (int xx = 0; xx < p; xx += 16) {
        if (nw >= NA_MAX_WORK) { set_error("patch_update_fv_noalloc: more than %d work items", NA_MAX_WORK); return DH_EINVAL; }
        Work& w = g_na_work[nw++];
        w.cls = 0; w.pz = dim == 3 ? p : 1; w.z0 = 0;
        for (int i = 0; i < 4; ++i) { w.patch[i] = -1; w.x0[i] = 0; w.y0[i] = 0; }
        w.patch[0] = k; w.x0[0] = (int16_t)xx; w.y0[0] = (int16_t)yy;
        has_cls[0] = true;
      }
  }
  for (int p = 8; p <= 256; p += 16) {  // p % 16 == 8
    int slot = 4;
    for (int k = 0; k < K; ++k) {
      if (patches[k].p != p) continue;
      for (int yy = 0; yy < p; yy += 8)
        for (int xx = 0; xx < p; xx += 8) {
          if (slot == 4) {
            if (nw >= NA_MAX_WORK) { set_error("patch_update_fv_noalloc: more than %d work items", NA_MAX_WORK); return DH_EINVAL; }
            Work& w = g_na_work[nw++];
            w.cls = 1; w.pz = dim == 3 ? p : 1; w.z0 = 0;
            for (int i = 0; i < 4; ++i) { w.patch[i] = -1; w.x0[i] = 0; w.y0[i] = 0; }
            slot = 0;
            has_cls[1] = true;
          }
          Work& w = g_na_work[nw - 1];
          w.patch[slot] = k; w.x0[slot] = (int16_t)xx; w.y0[slot] = (int16_t)yy;
          ++slot;
        }
    }
  }
  return nw;
}

}  // namespace
}  // namespace dh

using namespace dh;

extern "C" dh_status patch_update_fv_noalloc(int32_t pde, int32_t dim, const dh_patch* patches, int32_t K,
                                             int64_t var_stride, const double* params, int32_t n_params,
                                             const double* qs, const double* q0, double* out, double* acc,
                                             const double* mat, const double* dt_dev, double a, double b,
                                             double g, double d, double* lam_out_dev, void* stream) {
  if (pde != DH_PDE_ADV_FLUX && pde != DH_PDE_ADV_NCP && pde != DH_PDE_EULER2D && pde != DH_PDE_EULER3D) {
    set_error("patch_update_fv_noalloc: PDE %d not supported", pde);
    return DH_EUNSUPPORTED;
  }
  if (dim != pde_dim(pde)) { set_error("patch_update_fv_noalloc: wrong dim for PDE"); return DH_EINVAL; }
  if (!patches || K <= 0) { set_error("patch_update_fv_noalloc: empty patch list"); return DH_EINVAL; }
  if (K > NA_MAX_PATCHES) {
    set_error("patch_update_fv_noalloc: K = %d exceeds the limit of %d patches", K, NA_MAX_PATCHES);
    return DH_EINVAL;
  }
  if (var_stride <= 0 || var_stride % 32 != 0) { set_error("patch_update_fv_noalloc: bad var_stride"); return DH_EINVAL; }
  if (n_params < 0 || (n_params > 0 && !params)) { set_error("patch_update_fv_noalloc: bad params"); return DH_EINVAL; }
  if (!qs || !dt_dev || (!out && !acc)) { set_error("patch_update_fv_noalloc: qs, dt_dev and an output are required"); return DH_EINVAL; }
  if (pde_nm(pde) > 0 && !mat) { set_error("patch_update_fv_noalloc: PDE needs the material arena"); return DH_EINVAL; }
  if (!q0 && a != 0.0) { set_error("patch_update_fv_noalloc: q0 is NULL but a != 0"); return DH_EINVAL; }
  if (out == qs || acc == qs || (out && out == acc)) { set_error("patch_update_fv_noalloc: out/acc alias"); return DH_EINVAL; }

  std::lock_guard<std::mutex> lock(g_na_mutex);
  // the whole table is validated and the work list built on the host before any CUDA call
  bool has_cls[2];
  const int nw = na_build_work(dim, patches, K, 1, var_stride, has_cls);
  if (nw < 0) return (dh_status)nw;
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (device < 0 || device >= NA_MAX_DEVICES) { set_error("patch_update_fv_noalloc: device id %d too large", device); return DH_EINVAL; }
  if (!g_na_addr[device]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_na_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(scratch)");
    g_na_addr[device] = static_cast<unsigned char*>(ptr);
  }

  unsigned char* base = g_na_addr[device];
  unsigned long long* red = reinterpret_cast<unsigned long long*>(base);
  dh_patch* d_patches = reinterpret_cast<dh_patch*>(base + NA_RED_BYTES);
  Work* d_work = reinterpret_cast<Work*>(base + NA_RED_BYTES + NA_PATCH_BYTES);
  cudaStream_t s = (cudaStream_t)stream;
  std::memcpy(g_na_patches, patches, sizeof(dh_patch) * K);
  e = cudaMemcpyAsync(d_patches, g_na_patches, sizeof(dh_patch) * K, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_work, g_na_work, sizeof(Work) * nw, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(red, 0, dh_plan::NRED * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return cuda_error(e, "patch_update_fv_noalloc: table upload");

  // A plan on the stack pointing into the static array: the stage launch path
  // is the one patch_update_fv uses; nothing is allocated or freed.
  dh_plan view;
  view.pde = pde; view.dim = dim; view.K = K; view.halo = 1; view.var_stride = var_stride;
  view.nq = pde_nq(pde); view.nm = pde_nm(pde); view.device = device;
  DevParams& P = view.params;
  P.gamma = 1.4; P.Gamma = 5.0 / 3.0; P.damp = 0.1; P.kappa = 0.1;
  std::memset(P.C, 0, sizeof(P.C));
  if (params && n_params > 0 && (pde == DH_PDE_EULER2D || pde == DH_PDE_EULER3D)) P.gamma = params[0];
  finish_params(P);
  view.d_patches = d_patches;
  view.d_wl[0] = d_work;
  view.n_wl[0] = nw;
  view.fv_var = 2;  // one CTA per tile, register cap for two CTAs per SM, tile set 0
  view.fv_zs = 0;
  view.wl_cls[0][0] = has_cls[0];
  view.wl_cls[0][1] = has_cls[1];
  view.d_red = red;
  return launch_fv_stage(&view, qs, q0, out, acc, mat, dt_dev, a, b, g, d, lam_out_dev, s);
}
