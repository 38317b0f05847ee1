// C-ABI entry points of libdh: plans, argument validation, small kernels
// (wave-speed maximum, CFL time step, primitive -> conserved) and dispatch to
// the stage kernels.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "dh_internal.cuh"
#include "dh_pde.cuh"

namespace dh {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

dh_status cuda_error(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return DH_OK;
  set_error("%s: %s", what, cudaGetErrorString(e));
  return DH_ECUDA;
}

int pde_nq(int pde) {
  static const int n[7] = {1, 1, 4, 5, 5, 5, 59};
  return (pde >= 0 && pde < 7) ? n[pde] : 0;
}
int pde_nm(int pde) {
  static const int m[7] = {3, 3, 0, 0, 1, 5, 0};
  return (pde >= 0 && pde < 7) ? m[pde] : 0;
}
int pde_dim(int pde) { return pde == DH_PDE_EULER2D ? 2 : 3; }

// ---------------------------------------------------------------- small kernels
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// One CTA per patch: lambda of every voxel, block max, atomicMax on the bit
// pattern, last CTA publishes and resets the scratch.
template <class PDE>
__global__ void __launch_bounds__(256) k_max_speed(const dh_patch* __restrict__ patches, int dim, int64_t vs,
                                                   const double* __restrict__ q, const double* __restrict__ mat,
                                                   DevParams P, double* lam_out, unsigned long long* red) {
  __shared__ double wmax[8];
  __shared__ bool last;
  const dh_patch pt = patches[blockIdx.x];
  const int n = dim == 3 ? pt.p * pt.p * pt.p : pt.p * pt.p;
  double lam = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double u[PDE::N + PDE::M], W[PDE::NW > 0 ? PDE::NW : 1];
    const int64_t e = pt.offset + i;
#pragma unroll
    for (int v = 0; v < PDE::N; ++v) u[v] = q[v * vs + e];
#pragma unroll
    for (int v = 0; v < PDE::M; ++v) u[PDE::N + v] = mat[v * vs + e];
    PDE::prims(u, P, W);
    lam = fmax(lam, max_speed_dirs<PDE>(u, W, P, dim));
  }
  lam = warp_max_d(lam);
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = lam;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, wmax[i]);
    atomicMax(red, (unsigned long long)__double_as_longlong(m));
    __threadfence();
    last = atomicAdd(red + 1, 1ull) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    *lam_out = __longlong_as_double((long long)atomicAdd(red, 0ull));
    red[0] = 0ull;
    red[1] = 0ull;
    __threadfence();
  }
}

// The same maximum from the derived quantities W of the state (systems whose
// speeds depend on W alone: Euler), e.g. those a stage kernel just wrote.
template <class PDE>
__global__ void __launch_bounds__(256) k_max_speed_w(const dh_patch* __restrict__ patches, int dim, int64_t vs,
                                                     const double* __restrict__ w, DevParams P, double* lam_out,
                                                     unsigned long long* red) {
  __shared__ double wmax[8];
  __shared__ bool last;
  const dh_patch pt = patches[blockIdx.x];
  const int n = dim == 3 ? pt.p * pt.p * pt.p : pt.p * pt.p;
  double lam = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double W[PDE::NW];
    const int64_t e = pt.offset + i;
#pragma unroll
    for (int v = 0; v < PDE::NW; ++v) W[v] = w[v * vs + e];
    lam = fmax(lam, max_speed_dirs<PDE>(nullptr, W, P, dim));
  }
  lam = warp_max_d(lam);
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = lam;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, wmax[i]);
    atomicMax(red, (unsigned long long)__double_as_longlong(m));
    __threadfence();
    last = atomicAdd(red + 1, 1ull) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    *lam_out = __longlong_as_double((long long)atomicAdd(red, 0ull));
    red[0] = 0ull;
    red[1] = 0ull;
    __threadfence();
  }
}

dh_status max_wave_speed_w(dh_plan* plan, const double* w, double* lam_out_dev, cudaStream_t s) {
  const dh_patch* P = plan->d_patches;
  switch (plan->pde) {
    case DH_PDE_EULER2D: k_max_speed_w<PdeEuler2><<<plan->K, 256, 0, s>>>(P, 2, plan->var_stride, w, plan->params, lam_out_dev, plan->d_red); break;
    case DH_PDE_EULER3D: k_max_speed_w<PdeEuler3><<<plan->K, 256, 0, s>>>(P, 3, plan->var_stride, w, plan->params, lam_out_dev, plan->d_red); break;
    default:
      set_error("max_wave_speed_w: PDE %d keeps no derived quantities", plan->pde);
      return DH_EUNSUPPORTED;
  }
  return cuda_error(cudaGetLastError(), "max_wave_speed_w launch");
}

__global__ void k_cfl_dt(const double* lam, double cfl, double dx_dim, double* dt) {
  // dt = cfl * dx / (dim * lambda); dx_dim = dx / dim
  *dt = cfl * dx_dim / lam[0];
}

template <int DIM>
__global__ void k_prim2con_euler(const dh_patch* __restrict__ patches, int64_t vs, const double* __restrict__ w,
                                 double* __restrict__ q, double gamma) {
  const dh_patch pt = patches[blockIdx.x];
  const int n = DIM == 3 ? pt.p * pt.p * pt.p : pt.p * pt.p;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int64_t e = pt.offset + i;
    const double rho = w[e], p = w[(DIM + 1) * vs + e];
    double kin = 0.0;
    q[e] = rho;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      const double u = w[(1 + k) * vs + e];
      const double m = rho * u;
      q[(1 + k) * vs + e] = m;
      kin = fma(m, u, kin);
    }
    q[(DIM + 1) * vs + e] = fma(0.5, kin, p / (gamma - 1.0));
  }
}

__global__ void k_prim2con_srhd(const dh_patch* __restrict__ patches, int64_t vs, const double* __restrict__ w,
                                double* __restrict__ q, double G) {
  const dh_patch pt = patches[blockIdx.x];
  const int n = pt.p * pt.p * pt.p;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int64_t e = pt.offset + i;
    const double rho = w[e], vx = w[vs + e], vy = w[2 * vs + e], vz = w[3 * vs + e], p = w[4 * vs + e];
    const double v2 = fma(vx, vx, fma(vy, vy, vz * vz));
    const double W2 = 1.0 / (1.0 - v2);
    const double W = sqrt(W2);
    const double rhoh = fma(G / (G - 1.0), p, rho);
    const double rhohW2 = rhoh * W2;
    const double D = rho * W;
    q[e] = D;
    q[vs + e] = rhohW2 * vx;
    q[2 * vs + e] = rhohW2 * vy;
    q[3 * vs + e] = rhohW2 * vz;
    q[4 * vs + e] = (rhohW2 - p) - D;
  }
}

// Eight independent FMA chains per thread (throughput, not latency, bound).
__global__ void __launch_bounds__(256) k_probe_dfma(double* out, int iters, double b, double c) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double a0 = 1.0 + 1e-3 * threadIdx.x, a1 = a0 + 0.1, a2 = a0 + 0.2, a3 = a0 + 0.3;
  double a4 = a0 + 0.4, a5 = a0 + 0.5, a6 = a0 + 0.6, a7 = a0 + 0.7;
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
    a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
  }
  out[t] = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
}

// recip_nr next to the IEEE division, for the accuracy test.
__global__ void k_check_recip(const double* x, double* y_nr, double* y_div, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    y_nr[i] = recip_nr(x[i]);
    y_div[i] = 1.0 / x[i];
  }
}

// sqrt_pos and rsqrt_pos, for the accuracy test.
__global__ void k_check_sqrt(const double* x, double* y_sqrt, double* y_rsqrt, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    y_sqrt[i] = sqrt_pos(x[i]);
    y_rsqrt[i] = rsqrt_pos(x[i]);
  }
}

static inline int pt_nbr(const dh_patch* patches, int k, int f) { return patches[k].nbr[f]; }

// Work list of the generic FV stage (k_fv_any; see dh_fv_any.cuh).  An item's shape: ng groups
// of bx x by x bz voxels; its limits: at most 256 voxels, 512 box cells with the face halo, 320
// line cells and 256 faces of one direction.
static bool any_fits(int bx, int by, int bz, int ng, int dim) {
  const int ez = dim == 3 ? 2 : 0;
  if (ng < 1 || ng > 8 || bx < 1 || by < 1 || bz < 1 || (dim == 2 && bz != 1)) return false;
  if (ng * bx * by * bz > 256 || ng * (bx + 2) * (by + 2) * (bz + ez) > 512) return false;
  for (int d = 0; d < dim; ++d) {
    const int lines = (bx + 2 * (d == 0)) * (by + 2 * (d == 1)) * (bz + 2 * (d == 2));
    const int faces = (bx + (d == 0)) * (by + (d == 1)) * (bz + (d == 2));
    if (ng * lines > 320 || ng * faces > 256) return false;
  }
  return true;
}

// Patches of equal p and dx packed whole, up to eight to an item, where that fits; 2x2x2 blocks of
// face-adjacent 3^3 patches as one 6^3 box; boxes of the larger patches otherwise, of the tile
// shape that needs the fewest boxes.  Largest work first.
static std::vector<AnyWork> any_work(const dh_patch* patches, int K, int dim) {
  std::vector<AnyWork> out;
  std::vector<int> order(K);
  for (int k = 0; k < K; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return patches[a].p != patches[b].p ? patches[a].p > patches[b].p : patches[a].dx < patches[b].dx;
  });
  auto blank = [] {
    AnyWork w{};
    for (int i = 0; i < 8; ++i) w.patch[i] = -1;
    return w;
  };
  // 3D patches of 3^3: 2x2x2 blocks of face-adjacent patches form one 6^3 box (216 voxels, 512
  // cells), so that the halos between the block's members are ordinary box cells
  std::vector<char> used(K, 0);
  if (dim == 3) {
    for (int a = 0; a < K; ++a) {
      if (used[a] || patches[a].p != 3) continue;
      const int b = patches[a].nbr[1], c = patches[a].nbr[3], e = patches[a].nbr[5];
      const int d = patches[c].nbr[1], f = patches[e].nbr[1], g = patches[e].nbr[3], h = patches[g].nbr[1];
      const int m[8] = {a, b, c, d, e, f, g, h};
      // every member distinct, unused, 3^3 at a's dx, and linked both ways to its three partners
      bool ok = true;
      for (int x = 0; x < 8 && ok; ++x) {
        ok = !used[m[x]] && patches[m[x]].p == 3 && patches[m[x]].dx == patches[a].dx;
        for (int y = 0; y < x && ok; ++y) ok = m[x] != m[y];
        for (int ax = 0; ax < 3 && ok; ++ax) ok = patches[m[x]].nbr[2 * ax + !((x >> ax) & 1)] == m[x ^ (1 << ax)];
      }
      if (!ok) continue;
      AnyWork w = blank();
      for (int x = 0; x < 8; ++x) { w.patch[x] = m[x]; used[m[x]] = 1; }
      w.bx = 6; w.by = 6; w.bz = 6; w.ng = 1; w.mp = 3;
      out.push_back(w);
    }
  }
  order.erase(std::remove_if(order.begin(), order.end(), [&](int k) { return used[k] != 0; }), order.end());
  static const int tiles3[][3] = {{6, 6, 6}, {8, 8, 3}, {7, 7, 4}, {8, 6, 4}, {6, 8, 4}};
  static const int tiles2[][3] = {{16, 15, 1}, {15, 16, 1}, {16, 8, 1}, {8, 16, 1}};
  size_t i = 0;
  while (i < order.size()) {
    const int k = order[i], p = patches[k].p;
    const int pz = dim == 3 ? p : 1;
    int G = 8;
    while (G >= 1 && !any_fits(p, p, pz, G, dim)) --G;
    if (G >= 1) {
      AnyWork w = blank();
      w.bx = (int8_t)p; w.by = (int8_t)p; w.bz = (int8_t)pz;
      int ng = 0;
      while (ng < G && i < order.size() && patches[order[i]].p == p && patches[order[i]].dx == patches[k].dx)
        w.patch[ng++] = order[i++];
      w.ng = (int8_t)ng;
      out.push_back(w);
      continue;
    }
    const int(*tl)[3] = dim == 3 ? tiles3 : tiles2;
    const int nt = dim == 3 ? 5 : 4;
    int best = 0;
    long best_n = -1;
    for (int t = 0; t < nt; ++t) {
      const long n = (long)((p + tl[t][0] - 1) / tl[t][0]) * ((p + tl[t][1] - 1) / tl[t][1]) *
                     ((pz + tl[t][2] - 1) / tl[t][2]);
      if (best_n < 0 || n < best_n) { best_n = n; best = t; }
    }
    const int tx = tl[best][0], ty = tl[best][1], tz = tl[best][2];
    for (int z0 = 0; z0 < pz; z0 += tz)
      for (int y0 = 0; y0 < p; y0 += ty)
        for (int x0 = 0; x0 < p; x0 += tx) {
          AnyWork w = blank();
          w.patch[0] = k;
          w.x0 = (int16_t)x0; w.y0 = (int16_t)y0; w.z0 = (int16_t)z0;
          w.bx = (int8_t)std::min(tx, p - x0);
          w.by = (int8_t)std::min(ty, p - y0);
          w.bz = (int8_t)std::min(tz, pz - z0);
          w.ng = 1;
          out.push_back(w);
        }
    ++i;
  }
  std::stable_sort(out.begin(), out.end(), [](const AnyWork& a, const AnyWork& b) {
    return a.ng * a.bx * a.by * a.bz > b.ng * b.bx * b.by * b.bz;
  });
  return out;
}

static dh_status check_plan(const dh_plan* plan) {
  if (!plan) {
    set_error("plan is NULL");
    return DH_EINVAL;
  }
  return DH_OK;
}

}  // namespace dh

using namespace dh;

extern "C" {

const char* dh_last_error(void) { return g_err; }

const char* dh_version(void) { return "libdh 0.1 (sm_103a)"; }

dh_status dh_plan_create(dh_plan** out, int32_t pde, int32_t dim, const dh_patch* patches, int32_t K,
                         int32_t halo, int64_t var_stride, const double* params, int32_t n_params) {
  if (!out) { set_error("dh_plan_create: out is NULL"); return DH_EINVAL; }
  *out = nullptr;
  if (pde < 0 || pde > 6) { set_error("dh_plan_create: unknown pde %d", pde); return DH_EINVAL; }
  if (dim != pde_dim(pde)) { set_error("dh_plan_create: pde %d needs dim %d, got %d", pde, pde_dim(pde), dim); return DH_EINVAL; }
  if (!patches || K <= 0) { set_error("dh_plan_create: empty patch list"); return DH_EINVAL; }
  if (halo < 1 || halo > 8) { set_error("dh_plan_create: halo %d out of range [1, 8]", halo); return DH_EINVAL; }
  if (var_stride <= 0 || var_stride % 32 != 0) { set_error("dh_plan_create: var_stride %lld must be a positive multiple of 32", (long long)var_stride); return DH_EINVAL; }
  if (n_params < 0 || (n_params > 0 && !params)) { set_error("dh_plan_create: bad params"); return DH_EINVAL; }
  bool generic = false;
  for (int k = 0; k < K; ++k) generic = generic || patches[k].p % 8 != 0;
  for (int k = 0; k < K; ++k) {
    const dh_patch& pt = patches[k];
    if (pt.p < 2 || pt.p > 256) { set_error("patch %d: p = %d must lie in [2, 256]", k, pt.p); return DH_EINVAL; }
    if (pt.p < halo) { set_error("patch %d: p = %d smaller than the halo %d", k, pt.p, halo); return DH_EINVAL; }
    if (!(pt.dx > 0.0)) { set_error("patch %d: dx must be positive", k); return DH_EINVAL; }
    const int64_t n = dim == 3 ? (int64_t)pt.p * pt.p * pt.p : (int64_t)pt.p * pt.p;
    if (pt.offset < 0 || pt.offset % 16 != 0 || pt.offset + n > var_stride) {
      set_error("patch %d: offset %lld not 16-aligned or block exceeds var_stride", k, (long long)pt.offset);
      return DH_EINVAL;
    }
    for (int f = 0; f < 2 * dim; ++f) {
      const int nb = pt.nbr[f];
      if (nb < 0 || nb >= K) { set_error("patch %d: neighbour %d = %d out of range", k, f, nb); return DH_EINVAL; }
      const bool same = patches[nb].p == pt.p && patches[nb].dx == pt.dx && patches[nb].level == pt.level;
      const bool coarser = patches[nb].p == pt.p && patches[nb].dx == 2.0 * pt.dx && patches[nb].level == pt.level - 1;
      if (coarser && generic) {
        set_error("patch %d: coupled refinement levels need patch sizes that are multiples of 8", k);
        return DH_EINVAL;
      }
      if (!same && !coarser) {
        set_error("patch %d: neighbour %d (patch %d) must have the same p, dx and level, or be one level coarser "
                  "with the same p and twice the dx", k, f, nb);
        return DH_EINVAL;
      }
    }
  }
  dh_plan* plan = new (std::nothrow) dh_plan();
  if (!plan) { set_error("dh_plan_create: out of host memory"); return DH_ENOMEM; }
  plan->pde = pde; plan->dim = dim; plan->K = K; plan->halo = halo; plan->var_stride = var_stride;
  plan->nq = pde_nq(pde); plan->nm = pde_nm(pde);
  plan->h_patches.assign(patches, patches + K);
  plan->dx_min = patches[0].dx;
  for (int k = 1; k < K; ++k) plan->dx_min = std::min(plan->dx_min, patches[k].dx);
  DevParams& P = plan->params;
  P.gamma = 1.4; P.Gamma = 5.0 / 3.0; P.damp = 0.1; P.kappa = 0.1;
  std::memset(P.C, 0, sizeof(P.C));
  if (params && n_params > 0) {
    if (pde == DH_PDE_EULER2D || pde == DH_PDE_EULER3D) P.gamma = params[0];
    if (pde == DH_PDE_SRHD3D) P.Gamma = params[0];
    if (pde == DH_PDE_WAVE3D) P.damp = params[0];
    if (pde == DH_PDE_GW59) {
      P.kappa = params[0];
      for (int i = 0; i < 121 && 1 + i < n_params; ++i) P.C[i] = params[1 + i];
    }
  }
  finish_params(P);
  // Tile work lists, largest work first (see dh_plan::d_wl): 16x16 columns for p % 16 == 0
  // (tile set 1: 32x8 columns for p % 32 == 0; tile set 2: none), groups of four 8x8
  // columns of equal p otherwise.  With zs = 1 columns of more than 16 planes march in
  // chunks of at most 16 planes (more, shorter CTAs), and a thin last wave (two CTAs
  // resident per SM) is filled by splitting the cheapest full columns into two
  // half-height chunks, which then come last.
  int n_sm = 152;
  {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, d) != cudaSuccess)
      n_sm = 152;
    cudaGetLastError();
  }
  std::vector<Work> lists[dh_plan::NWL];
  for (int li = 0; li < dh_plan::NWL && !generic; ++li) {
    const int tile = li / 2, zs = li % 2;
    std::vector<Work>& work = lists[li];
    std::vector<std::vector<std::pair<int, std::pair<int, int>>>> pending(257);
    for (int k = 0; k < K; ++k) {
      const int p = patches[k].p, pz = dim == 3 ? p : 1;
      const int cls = tile == 3 ? 3 : (tile == 1 && p % 32 == 0) ? 2 : (tile != 2 && p % 16 == 0) ? 0 : 1;
      if (cls == 1) {
        for (int yy = 0; yy < p; yy += 8)
          for (int xx = 0; xx < p; xx += 8) pending[p].push_back({k, {xx, yy}});
        continue;
      }
      const int tx = cls == 2 ? 32 : (cls == 3 ? 8 : 16), ty = cls == 2 ? 8 : (cls == 3 ? 8 : 16);
      const int chunk = (zs == 1 && pz > 16) ? 16 : pz;
      for (int zz = 0; zz < pz; zz += chunk)
        for (int yy = 0; yy < p; yy += ty)
          for (int xx = 0; xx < p; xx += tx) {
            Work w{};
            w.cls = cls; w.pz = std::min(chunk, pz - zz); w.z0 = zz;
            for (int i = 0; i < 4; ++i) { w.patch[i] = -1; w.x0[i] = 0; w.y0[i] = 0; }
            w.patch[0] = k; w.x0[0] = (int16_t)xx; w.y0[0] = (int16_t)yy;
            work.push_back(w);
          }
    }
    for (int p = 8; p <= 256; p += 8) {
      auto& v = pending[p];
      for (size_t i = 0; i < v.size(); i += 4) {
        Work w{};
        w.cls = 1; w.pz = dim == 3 ? p : 1; w.z0 = 0;
        for (int j = 0; j < 4; ++j) {
          if (i + j < v.size()) { w.patch[j] = v[i + j].first; w.x0[j] = (int16_t)v[i + j].second.first; w.y0[j] = (int16_t)v[i + j].second.second; }
          else { w.patch[j] = -1; w.x0[j] = 0; w.y0[j] = 0; }
        }
        work.push_back(w);
      }
    }
    auto cost = [](const Work& w) {
      int ng = 0;
      for (int j = 0; j < 4; ++j) ng += w.patch[j] >= 0;
      return (long long)(w.cls == 1 ? 64 * ng : (w.cls == 3 ? 64 : 256)) * w.pz;
    };
    std::stable_sort(work.begin(), work.end(), [&](const Work& a, const Work& b) { return cost(a) > cost(b); });
    if (zs == 1 && dim == 3) {
      const long long R = (tile == 3 ? 8LL : 2LL) * n_sm;  // resident CTAs per wave
      long long m = (R - (long long)work.size() % R) % R;
      std::vector<Work> halves;
      for (int i = (int)work.size() - 1; i >= 0 && m > 0; --i) {
        Work& w = work[i];
        if (w.cls == 1 || w.pz < 16) continue;  // (16-plane columns split into two chunks of 8)
        Work upper = w;
        w.pz = w.pz / 2;
        upper.pz = upper.pz - w.pz;
        upper.z0 = w.z0 + w.pz;
        halves.push_back(upper);
        --m;
      }
      work.insert(work.end(), halves.begin(), halves.end());
      std::stable_sort(work.begin(), work.end(), [&](const Work& a, const Work& b) { return cost(a) > cost(b); });
    }
    for (const Work& w : work) plan->wl_cls[li][w.cls] = true;
    plan->n_wl[li] = (int)work.size();
  }

  // FD tiles: 8x8x4 blocks (p is a multiple of 8)
  std::vector<FdWork> fdw;
  if (dim == 3 && !generic) {
    for (int k = 0; k < K; ++k) {
      const int p = patches[k].p;
      for (int zz = 0; zz < p; zz += 4)
        for (int yy = 0; yy < p; yy += 8)
          for (int xx = 0; xx < p; xx += 8) fdw.push_back(FdWork{k, (int16_t)xx, (int16_t)yy, (int16_t)zz, 0});
    }
  }
  plan->n_fdwork = (int)fdw.size();

  // Generic FV work (patch sizes not all multiples of 8): every item within the kernel's shared-
  // memory limits, checked here once more since the kernel indexes its arrays without checks.
  std::vector<AnyWork> anyw;
  plan->fv_generic = generic;
  if (generic) {
    anyw = any_work(patches, K, dim);
    for (const AnyWork& w : anyw)
      if (!any_fits(w.bx, w.by, w.bz, w.ng, dim)) {
        set_error("generic FV work item %dx%dx%d x %d exceeds the kernel's limits", w.bx, w.by, w.bz, w.ng);
        delete plan;
        return DH_EINVAL;
      }
  }
  plan->n_any = (int)anyw.size();

  // Levels for TMA staging (see dh_internal.cuh).
  std::vector<int2> lvl(K);
  {
    bool ok = dim == 3 && !generic;
    int nl = 0;
    for (int k = 0; k < K && ok;) {
      int e = k + 1;
      const int64_t step = (int64_t)patches[k].p * patches[k].p * patches[k].p;
      while (e < K && patches[e].p == patches[k].p && patches[e].offset == patches[e - 1].offset + step) ++e;
      if (nl >= 8) { ok = false; break; }
      plan->lvl_p[nl] = patches[k].p;
      plan->lvl_K[nl] = e - k;
      plan->lvl_off[nl] = patches[k].offset;
      for (int j = k; j < e; ++j) lvl[j] = make_int2(nl, j - k);
      ++nl;
      k = e;
    }
    for (int k = 0; k < K && ok; ++k)
      for (int f = 0; f < 6; ++f)
        if (lvl[pt_nbr(patches, k, f)].x != lvl[k].x) ok = false;
    plan->n_lvl = ok ? nl : 0;
    plan->tma_ok = ok;
  }

  cudaError_t e = cudaGetDevice(&plan->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&plan->num_sms, cudaDevAttrMultiProcessorCount, plan->device);
  if (e == cudaSuccess) e = cudaMalloc(&plan->d_patches, sizeof(dh_patch) * K);
  if (e == cudaSuccess) e = cudaMemcpy(plan->d_patches, patches, sizeof(dh_patch) * K, cudaMemcpyHostToDevice);
  for (int li = 0; li < dh_plan::NWL && e == cudaSuccess; ++li) {
    e = cudaMalloc(&plan->d_wl[li], sizeof(Work) * std::max<size_t>(1, lists[li].size()));
    if (e == cudaSuccess && !lists[li].empty())
      e = cudaMemcpy(plan->d_wl[li], lists[li].data(), sizeof(Work) * lists[li].size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess && !anyw.empty()) e = cudaMalloc(&plan->d_any, sizeof(AnyWork) * anyw.size());
  if (e == cudaSuccess && !anyw.empty())
    e = cudaMemcpy(plan->d_any, anyw.data(), sizeof(AnyWork) * anyw.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !fdw.empty()) e = cudaMalloc(&plan->d_fdwork, sizeof(FdWork) * fdw.size());
  if (e == cudaSuccess && !fdw.empty())
    e = cudaMemcpy(plan->d_fdwork, fdw.data(), sizeof(FdWork) * fdw.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&plan->d_red, dh_plan::NRED * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(plan->d_red, 0, dh_plan::NRED * sizeof(unsigned long long));
  if (e == cudaSuccess) {
    dh_status ast = amr_build(plan, patches, K, dim);
    if (ast != DH_OK) { dh_plan_destroy(plan); return ast; }
  }
  const std::vector<int2> aunits = aoas_units(patches, K, dim);
  plan->n_aunits = (int)aunits.size();
  if (e == cudaSuccess) e = cudaMalloc(&plan->d_aunits, sizeof(int2) * aunits.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(plan->d_aunits, aunits.data(), sizeof(int2) * aunits.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && plan->tma_ok) e = cudaMalloc(&plan->d_lvl, sizeof(int2) * K);
  if (e == cudaSuccess && plan->tma_ok) e = cudaMemcpy(plan->d_lvl, lvl.data(), sizeof(int2) * K, cudaMemcpyHostToDevice);
  // cudaMemset, and cudaMemcpy from pageable host memory, can return before the device
  // holds the data (they run on the legacy default stream); the first launch may come on
  // a non-blocking stream, so wait for them here
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e != cudaSuccess) {
    dh_status st = cuda_error(e, "dh_plan_create");
    dh_plan_destroy(plan);
    return e == cudaErrorMemoryAllocation ? DH_ENOMEM : st;
  }
  *out = plan;
  return DH_OK;
}

dh_status dh_plan_destroy(dh_plan* plan) {
  if (!plan) return DH_OK;
  if (plan->d_patches) cudaFree(plan->d_patches);
  for (int li = 0; li < dh_plan::NWL; ++li)
    if (plan->d_wl[li]) cudaFree(plan->d_wl[li]);
  if (plan->d_red) cudaFree(plan->d_red);
  if (plan->d_fdwork) cudaFree(plan->d_fdwork);
  if (plan->d_any) cudaFree(plan->d_any);
  if (plan->d_lvl) cudaFree(plan->d_lvl);
  if (plan->d_aunits) cudaFree(plan->d_aunits);
  if (plan->d_offload) cudaFree(plan->d_offload);
  if (plan->d_stage) cudaFree(plan->d_stage);
  if (plan->d_amr_oct) cudaFree(plan->d_amr_oct);
  if (plan->d_w) cudaFree(plan->d_w);
  if (plan->d_amr_reflux) cudaFree(plan->d_amr_reflux);
  if (plan->d_amr_restrict) cudaFree(plan->d_amr_restrict);
  if (plan->graph_exec) cudaGraphExecDestroy(plan->graph_exec);
  for (cudaEvent_t e : plan->ev_start) cudaEventDestroy(e);
  for (cudaEvent_t e : plan->ev_stop) cudaEventDestroy(e);
  delete plan;
  return DH_OK;
}

dh_status patch_update_fv(dh_plan* plan, const double* qs, const double* q0, double* out, double* acc,
                          const double* mat, const double* dt_dev, double a, double b, double g, double d,
                          double* lam_out_dev, void* stream) {
  dh_status st = check_plan(plan);
  if (st != DH_OK) return st;
  if (!qs || !dt_dev) { set_error("patch_update_fv: qs and dt_dev are required"); return DH_EINVAL; }
  if (!out && !acc) { set_error("patch_update_fv: nothing to write (out and acc are NULL)"); return DH_EINVAL; }
  if (plan->nm > 0 && !mat) { set_error("patch_update_fv: PDE needs the material arena"); return DH_EINVAL; }
  if (!q0 && a != 0.0) { set_error("patch_update_fv: q0 is NULL but a != 0"); return DH_EINVAL; }
  if (out == qs || acc == qs || (out && out == acc)) { set_error("patch_update_fv: out/acc must not alias qs or each other"); return DH_EINVAL; }
  if (plan->pde == DH_PDE_SRHD3D && lam_out_dev) { set_error("patch_update_fv: lam_out is not available for SRHD3D"); return DH_EUNSUPPORTED; }
  if (plan->pde == DH_PDE_WAVE3D || plan->pde == DH_PDE_GW59) {
    set_error("patch_update_fv: PDE %d is evolved with patch_update_fd_ko", plan->pde);
    return DH_EUNSUPPORTED;
  }
  if (!plan->coupled)
    return launch_fv_stage(plan, qs, q0, out, acc, mat, dt_dev, a, b, g, d, lam_out_dev, (cudaStream_t)stream);
  // coupled refinement levels: stage (prolongation inside), reflux, restriction, then the
  // wave speed of the coupled result
  if (plan->pde == DH_PDE_ADV_NCP) {
    set_error("patch_update_fv: coupled refinement levels need a conservative system (no B(Q).grad Q)");
    return DH_EUNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  st = launch_fv_stage(plan, qs, q0, out, acc, mat, dt_dev, a, b, g, d, nullptr, s);
  if (st == DH_OK) st = amr_couple(plan, qs, mat, out, acc, dt_dev, g, d, s);
  if (st == DH_OK && lam_out_dev) st = max_wave_speed(plan, out ? out : acc, mat, lam_out_dev, stream);
  return st;
}

dh_status patch_update_fd_ko(dh_plan* plan, const double* qs, const double* q0, double* out, double* acc,
                             const double* mat, const double* dt_dev, double a, double b, double g, double d,
                             double sigma_ko, double* lam_out_dev, void* stream) {
  dh_status st = check_plan(plan);
  if (st != DH_OK) return st;
  if (plan->fv_generic) { set_error("patch_update_fd_ko: needs patch sizes that are multiples of 8"); return DH_EUNSUPPORTED; }
  if (!qs || !dt_dev) { set_error("patch_update_fd_ko: qs and dt_dev are required"); return DH_EINVAL; }
  if (!out && !acc) { set_error("patch_update_fd_ko: nothing to write (out and acc are NULL)"); return DH_EINVAL; }
  if (plan->nm > 0 && !mat) { set_error("patch_update_fd_ko: PDE needs the material arena"); return DH_EINVAL; }
  if (!q0 && a != 0.0) { set_error("patch_update_fd_ko: q0 is NULL but a != 0"); return DH_EINVAL; }
  if (out == qs || acc == qs || (out && out == acc)) { set_error("patch_update_fd_ko: out/acc must not alias qs or each other"); return DH_EINVAL; }
  if (plan->halo < 3) { set_error("patch_update_fd_ko: the plan needs halo >= 3 (it has %d)", plan->halo); return DH_EINVAL; }
  if (plan->coupled) { set_error("patch_update_fd_ko: coupled refinement levels are supported by patch_update_fv only"); return DH_EUNSUPPORTED; }
  if (plan->dim != 3) { set_error("patch_update_fd_ko: 3D only"); return DH_EUNSUPPORTED; }
  if (!(sigma_ko >= 0.0)) { set_error("patch_update_fd_ko: sigma must be >= 0"); return DH_EINVAL; }
  return launch_fd_stage(plan, qs, q0, out, acc, mat, dt_dev, a, b, g, d, sigma_ko, lam_out_dev, (cudaStream_t)stream);
}

dh_status patch_update_fv_muscl(dh_plan* plan, const double* qs, const double* q0, double* out, double* acc,
                                const double* mat, const double* dt_dev, double a, double b, double g, double d,
                                double* lam_out_dev, void* stream) {
  dh_status st = check_plan(plan);
  if (st != DH_OK) return st;
  if (plan->fv_generic) { set_error("patch_update_fv_muscl: needs patch sizes that are multiples of 8"); return DH_EUNSUPPORTED; }
  if (!qs || !dt_dev) { set_error("patch_update_fv_muscl: qs and dt_dev are required"); return DH_EINVAL; }
  if (!out && !acc) { set_error("patch_update_fv_muscl: nothing to write (out and acc are NULL)"); return DH_EINVAL; }
  if (plan->nm > 0 && !mat) { set_error("patch_update_fv_muscl: PDE needs the material arena"); return DH_EINVAL; }
  if (!q0 && a != 0.0) { set_error("patch_update_fv_muscl: q0 is NULL but a != 0"); return DH_EINVAL; }
  if (out == qs || acc == qs || (out && out == acc)) { set_error("patch_update_fv_muscl: out/acc must not alias qs or each other"); return DH_EINVAL; }
  if (plan->halo < 2) { set_error("patch_update_fv_muscl: the plan needs halo >= 2 (it has %d)", plan->halo); return DH_EINVAL; }
  if (plan->coupled) { set_error("patch_update_fv_muscl: coupled refinement levels are supported by patch_update_fv only"); return DH_EUNSUPPORTED; }
  if (plan->dim != 3) { set_error("patch_update_fv_muscl: 3D only"); return DH_EUNSUPPORTED; }
  return launch_fv2_stage(plan, qs, q0, out, acc, mat, dt_dev, a, b, g, d, lam_out_dev, (cudaStream_t)stream);
}

dh_status max_wave_speed(dh_plan* plan, const double* q, const double* mat, double* lam_out_dev, void* stream) {
  dh_status st = check_plan(plan);
  if (st != DH_OK) return st;
  if (!q || !lam_out_dev) { set_error("max_wave_speed: q and lam_out_dev are required"); return DH_EINVAL; }
  if (plan->nm > 0 && !mat) { set_error("max_wave_speed: PDE needs the material arena"); return DH_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  const dh_patch* P = plan->d_patches;
  switch (plan->pde) {
    case DH_PDE_ADV_FLUX: k_max_speed<PdeAdvFlux><<<plan->K, 256, 0, s>>>(P, 3, plan->var_stride, q, mat, plan->params, lam_out_dev, plan->d_red); break;
    case DH_PDE_ADV_NCP: k_max_speed<PdeAdvNcp><<<plan->K, 256, 0, s>>>(P, 3, plan->var_stride, q, mat, plan->params, lam_out_dev, plan->d_red); break;
    case DH_PDE_EULER2D: k_max_speed<PdeEuler2><<<plan->K, 256, 0, s>>>(P, 2, plan->var_stride, q, mat, plan->params, lam_out_dev, plan->d_red); break;
    case DH_PDE_EULER3D: k_max_speed<PdeEuler3><<<plan->K, 256, 0, s>>>(P, 3, plan->var_stride, q, mat, plan->params, lam_out_dev, plan->d_red); break;
    case DH_PDE_SRHD3D: k_max_speed<PdeSRHD><<<plan->K, 256, 0, s>>>(P, 3, plan->var_stride, q, mat, plan->params, lam_out_dev, plan->d_red); break;
    case DH_PDE_WAVE3D: k_max_speed<PdeWave><<<plan->K, 256, 0, s>>>(P, 3, plan->var_stride, q, mat, plan->params, lam_out_dev, plan->d_red); break;
    case DH_PDE_GW59: k_max_speed<PdeGW59><<<plan->K, 256, 0, s>>>(P, 3, plan->var_stride, q, mat, plan->params, lam_out_dev, plan->d_red); break;
    default:
      set_error("max_wave_speed: PDE %d not supported yet", plan->pde);
      return DH_EUNSUPPORTED;
  }
  return cuda_error(cudaGetLastError(), "max_wave_speed launch");
}

dh_status dh_cfl_dt(dh_plan* plan, const double* lam_dev, double cfl, double* dt_dev, void* stream) {
  dh_status st = check_plan(plan);
  if (st != DH_OK) return st;
  if (!lam_dev || !dt_dev || !(cfl > 0.0)) { set_error("dh_cfl_dt: bad arguments"); return DH_EINVAL; }
  k_cfl_dt<<<1, 1, 0, (cudaStream_t)stream>>>(lam_dev, cfl, plan->dx_min / plan->dim, dt_dev);
  return cuda_error(cudaGetLastError(), "dh_cfl_dt launch");
}

dh_status dh_prim2con(dh_plan* plan, const double* prim, double* cons, void* stream) {
  dh_status st = check_plan(plan);
  if (st != DH_OK) return st;
  if (!prim || !cons || prim == cons) { set_error("dh_prim2con: bad buffers"); return DH_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  if (plan->pde == DH_PDE_EULER2D) k_prim2con_euler<2><<<plan->K, 256, 0, s>>>(plan->d_patches, plan->var_stride, prim, cons, plan->params.gamma);
  else if (plan->pde == DH_PDE_EULER3D) k_prim2con_euler<3><<<plan->K, 256, 0, s>>>(plan->d_patches, plan->var_stride, prim, cons, plan->params.gamma);
  else if (plan->pde == DH_PDE_SRHD3D) k_prim2con_srhd<<<plan->K, 256, 0, s>>>(plan->d_patches, plan->var_stride, prim, cons, plan->params.Gamma);
  else { set_error("dh_prim2con: PDE %d has no primitive form", plan->pde); return DH_EUNSUPPORTED; }
  return cuda_error(cudaGetLastError(), "dh_prim2con launch");
}

dh_status dh_plan_set_debug(dh_plan* plan, int32_t flags) {
  if (!plan) { set_error("plan is NULL"); return DH_EINVAL; }
  plan->debug_flags = flags;
  return DH_OK;
}

dh_status dh_plan_errors(dh_plan* plan, uint32_t* flags, int32_t clear) {
  if (!plan || !flags) { set_error("dh_plan_errors: bad arguments"); return DH_EINVAL; }
  unsigned long long v = 0;
  cudaError_t e = cudaMemcpy(&v, plan->d_red + 2, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error(e, "dh_plan_errors");
  *flags = (uint32_t)v;
  if (clear) {
    e = cudaMemset(plan->d_red + 2, 0, sizeof(v));
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);  // cleared before any later launch on any stream
    if (e != cudaSuccess) return cuda_error(e, "dh_plan_errors");
  }
  return DH_OK;
}

dh_status dh_check_recip(const double* x, double* y_nr, double* y_div, int64_t n, void* stream) {
  if (!x || !y_nr || !y_div || n <= 0 || n > (1ll << 40)) { set_error("dh_check_recip: bad arguments"); return DH_EINVAL; }
  k_check_recip<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, y_nr, y_div, n);
  return cuda_error(cudaGetLastError(), "dh_check_recip launch");
}

dh_status dh_generic_work_list(int32_t dim, const dh_patch* patches, int32_t K, int32_t* items, int32_t max_items,
                               int32_t* n_items) {
  if ((dim != 2 && dim != 3) || !patches || K <= 0 || !n_items || (items && max_items < 0)) {
    set_error("dh_generic_work_list: bad arguments");
    return DH_EINVAL;
  }
  for (int k = 0; k < K; ++k) {
    const dh_patch& pt = patches[k];
    if (pt.p < 2 || pt.p > 256) { set_error("dh_generic_work_list: patch %d: p = %d", k, pt.p); return DH_EINVAL; }
    for (int f = 0; f < 2 * dim; ++f)
      if (pt.nbr[f] < 0 || pt.nbr[f] >= K) { set_error("dh_generic_work_list: patch %d: bad neighbour", k); return DH_EINVAL; }
  }
  const std::vector<AnyWork> w = any_work(patches, K, dim);
  *n_items = (int32_t)w.size();
  if (!items) return DH_OK;
  if ((int64_t)w.size() > max_items) { set_error("dh_generic_work_list: %d items > max_items", (int)w.size()); return DH_EINVAL; }
  for (size_t i = 0; i < w.size(); ++i) {
    int32_t* o = items + 16 * i;
    for (int j = 0; j < 8; ++j) o[j] = w[i].patch[j];
    o[8] = w[i].x0; o[9] = w[i].y0; o[10] = w[i].z0;
    o[11] = w[i].bx; o[12] = w[i].by; o[13] = w[i].bz; o[14] = w[i].ng; o[15] = w[i].mp;
  }
  return DH_OK;
}

dh_status dh_check_sqrt(const double* x, double* y_sqrt, double* y_rsqrt, int64_t n, void* stream) {
  if (!x || !y_sqrt || !y_rsqrt || n <= 0 || n > (1ll << 40)) { set_error("dh_check_sqrt: bad arguments"); return DH_EINVAL; }
  k_check_sqrt<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, y_sqrt, y_rsqrt, n);
  return cuda_error(cudaGetLastError(), "dh_check_sqrt launch");
}

dh_status dh_probe_dfma(double* out_dev, int64_t n_threads, int32_t iters, void* stream) {
  if (!out_dev || n_threads <= 0 || n_threads % 256 != 0 || n_threads / 256 > (1ll << 30) || iters <= 0) {
    set_error("dh_probe_dfma: out_dev must be non-NULL, n_threads a positive multiple of 256, iters > 0");
    return DH_EINVAL;
  }
  k_probe_dfma<<<(unsigned)(n_threads / 256), 256, 0, (cudaStream_t)stream>>>(out_dev, iters, 0.999999, 1e-7);
  return cuda_error(cudaGetLastError(), "dh_probe_dfma launch");
}

}  // extern "C"
