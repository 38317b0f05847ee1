// Coarse-fine coupling of refinement levels for the first-order FV stage.
//
// The paper's meshes are Peano spacetrees (Sec. IV) whose cells carry the
// patches; it defines no coupling between levels.  Reading used here: ratio
// 2, a patch of level l+1 covers one octant of a patch of level l (its
// parent, still in the patch list), same p, half the voxel spacing; a face
// neighbour is either of the patch's own level or one level coarser.
//   * Prolongation (inside the stage kernel's halo gather): a halo voxel that
//     lies in a coarser neighbour takes the value of the coarse voxel that
//     contains it.
//   * Reflux (k_reflux, after the stage kernel): a coarse voxel next to the
//     finer level uses, on that face, the mean of the 2^(d-1) fine face
//     fluxes instead of its own coarse face flux:
//         out += g dt sgn (mean(F^_fine) - F^_coarse) / dx_coarse   (acc with d dt;
//         in the SSP-RK3 stage-sum form acc holds raw face-flux sums and takes
//         -2 sgn (mean(F^_fine) - F^_coarse) in stages 1 and 2),
//     sgn = -1 for the coarse voxel's +a face, +1 for its -a face.  Fine face
//     fluxes use the coarse voxel as the halo value, exactly as the fine
//     patch's own update did, so mass, momentum and energy are conserved
//     across levels.  Sums of 2^k values are balanced trees, so equal values
//     sum exactly (a constant state stays bitwise constant).
//   * Restriction (k_restrict, last): every coarse voxel covered by the finer
//     level becomes the mean of its 2^d fine voxels, finest level first.
// The plan builds, once: the octant bits of every patch, one reflux entry
// per (coarse voxel, face) grouped by face direction, and the list of (fine
// patch, parent) pairs by level.  A coarse voxel has at most one entry per
// direction; when it also has at most one entry overall (a convex refined
// region) all entries go in one launch, else one launch per direction, so no
// two threads of a launch write the same voxel.
#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>

#include "dh_internal.cuh"
#include "dh_pde.cuh"

namespace dh {
namespace {

struct CplArgs {
  const dh_patch* patches;
  const AmrReflux* reflux;
  const int2* restrict_list;  // (fine patch, parent)
  const int* oct;
  const double* qs;
  const double* mat;
  double* out;
  double* acc;
  const double* dt_dev;
  double g, d;
  int form;  // 0: general stage (acc += d dt L); 1-3: SSP-RK3 stage-sum form (acc = raw face-flux sums)
  double* w_out;  // derived quantities W of the result (NW-variable arena) to refresh, or NULL
  int64_t vs;
  int n, dim;
  DevParams P;
};

template <class PDE>
__device__ __forceinline__ void c_load(const CplArgs& A, int64_t e, double* q) {
#pragma unroll
  for (int v = 0; v < PDE::N; ++v) q[v] = A.qs[v * A.vs + e];
#pragma unroll
  for (int v = 0; v < PDE::M; ++v) q[PDE::N + v] = A.mat[v * A.vs + e];
}

// Flux F_a and speed lambda_a of one voxel state (N+M values).
template <class PDE>
__device__ __forceinline__ void c_flux(const DevParams& P, int a, const double* q, double* F, double& lam) {
  double W[PDE::NW > 0 ? PDE::NW : 1];
  PDE::prims(q, P, W);
  PDE::flux(a, q, W, P, F);
  lam = PDE::speed(a, q, W, P);
}

// Rusanov flux (F_L + F_R)/2 - max(lam_L, lam_R)/2 (Q_R - Q_L) from precomputed fluxes and speeds.
template <int N>
__device__ __forceinline__ void c_rusanov(const double* qL, const double* FL, double lL, const double* qR,
                                          const double* FR, double lR, double* fh) {
  const double hs = 0.5 * max_nn(lL, lR);
#pragma unroll
  for (int v = 0; v < N; ++v) fh[v] = 0.5 * (FL[v] + FR[v]) - hs * (qR[v] - qL[v]);
}

// One thread per reflux entry; the derived quantities, flux and speed of every
// voxel involved are computed once.
template <class PDE>
__global__ void __launch_bounds__(64) k_reflux(const __grid_constant__ CplArgs A) {
  constexpr int N = PDE::N, NV = PDE::N + PDE::M;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const AmrReflux R = A.reflux[i];
  const dh_patch& C = A.patches[R.C];
  const int64_t eC = C.offset + R.eC;
  const int a = R.axis;
  double qC[NV], qN[NV], qF[NV], FC[N], FN[N], FF[N], fc[N], ff[N], pair[N], fsum[N], lC, lN, lF;
  c_load<PDE>(A, eC, qC);
  c_load<PDE>(A, A.patches[R.N].offset + R.eN, qN);
  c_flux<PDE>(A.P, a, qC, FC, lC);
  c_flux<PDE>(A.P, a, qN, FN, lN);
  if (R.lo) c_rusanov<N>(qC, FC, lC, qN, FN, lN, fc);
  else c_rusanov<N>(qN, FN, lN, qC, FC, lC, fc);
  const int64_t f0 = A.patches[R.F].offset + R.eF;
  const int nk = A.dim == 3 ? 2 : 1;
  for (int sk = 0; sk < nk; ++sk) {
    for (int sj = 0; sj < 2; ++sj) {
      c_load<PDE>(A, f0 + sj * R.sb0 + sk * R.sb1, qF);
      c_flux<PDE>(A.P, a, qF, FF, lF);
      if (R.lo) c_rusanov<N>(qC, FC, lC, qF, FF, lF, ff);
      else c_rusanov<N>(qF, FF, lF, qC, FC, lC, ff);
#pragma unroll
      for (int v = 0; v < N; ++v) pair[v] = sj == 0 ? ff[v] : pair[v] + ff[v];
    }
#pragma unroll
    for (int v = 0; v < N; ++v) fsum[v] = sk == 0 ? pair[v] : fsum[v] + pair[v];
  }
  const double rn = A.dim == 3 ? 0.25 : 0.5;
  const double sgn = R.lo ? -1.0 : 1.0;
  const double dt = *A.dt_dev;
  const double gdt = A.g * dt, ddt = A.d * dt;
  double qn[NV];
#pragma unroll
  for (int v = 0; v < N; ++v) {
    const double dL = sgn * (fsum[v] * rn - fc[v]) / C.dx;
    const int64_t ev = v * A.vs + eC;
    if (A.out) {
      qn[v] = A.out[ev] + gdt * dL;
      A.out[ev] = qn[v];
    }
    if (A.acc && A.form == 0) A.acc[ev] = A.acc[ev] + ddt * dL;
    // stage-sum form: the raw sum (twice the face fluxes, L = -sum/(2 dx)) of stages 1 and 2
    if (A.acc && (A.form == 1 || A.form == 2)) A.acc[ev] = A.acc[ev] - 2.0 * sgn * (fsum[v] * rn - fc[v]);
  }
  // the derived quantities of the corrected voxel, for the next stage (multi-step graphs)
  if (A.w_out && A.out) {
#pragma unroll
    for (int v = N; v < NV; ++v) qn[v] = A.mat[(v - N) * A.vs + eC];
    double W[PDE::NW > 0 ? PDE::NW : 1];
    PDE::prims(qn, A.P, W);
#pragma unroll
    for (int i = 0; i < PDE::NW; ++i) A.w_out[i * A.vs + eC] = W[i];
  }
}

// Mean of the 2^d fine voxels under coarse voxel (x, y, z) of the covered block:
// pairs along x, then rows, then layers (balanced tree).
__device__ __forceinline__ double fine_mean(const double* a, int p, int dim, int x, int y, int z) {
  double layer[2];
  for (int sz = 0; sz < (dim == 3 ? 2 : 1); ++sz) {
    const int64_t r0 = ((int64_t)(dim == 3 ? 2 * z + sz : 0) * p + 2 * y) * p + 2 * x;
    const double row0 = a[r0] + a[r0 + 1];
    const double row1 = a[r0 + p] + a[r0 + p + 1];
    layer[sz] = row0 + row1;
  }
  const double sum = dim == 3 ? layer[0] + layer[1] : layer[0];
  return sum * (dim == 3 ? 0.125 : 0.25);
}

// As k_restrict, one thread per covered coarse voxel (all N variables), which
// then refreshes that voxel's derived quantities W in A.w_out.
template <class PDE>
__global__ void __launch_bounds__(256) k_restrict_w(const __grid_constant__ CplArgs A) {
  constexpr int N = PDE::N, NV = PDE::N + PDE::M;
  const int2 fp = A.restrict_list[blockIdx.x];
  const dh_patch& F = A.patches[fp.x];
  const dh_patch& Pp = A.patches[fp.y];
  const int p = F.p, h = p >> 1, o = A.oct[fp.x];
  const int hz = A.dim == 3 ? h : 1;
  const int nvox = h * h * hz;
  for (int r = threadIdx.x; r < nvox; r += blockDim.x) {
    const int x = r % h, y = (r / h) % h, z = r / (h * h);
    const int cx = (o & 1) * h + x, cy = ((o >> 1) & 1) * h + y, cz = A.dim == 3 ? ((o >> 2) & 1) * h + z : 0;
    const int64_t ec = Pp.offset + ((int64_t)cz * p + cy) * p + cx;
    double qn[NV];
#pragma unroll
    for (int v = 0; v < N; ++v) {
      qn[v] = fine_mean(A.out + (int64_t)v * A.vs + F.offset, p, A.dim, x, y, z);
      A.out[(int64_t)v * A.vs + ec] = qn[v];
      if (A.acc) A.acc[(int64_t)v * A.vs + ec] = fine_mean(A.acc + (int64_t)v * A.vs + F.offset, p, A.dim, x, y, z);
    }
#pragma unroll
    for (int v = N; v < NV; ++v) qn[v] = A.mat[(v - N) * A.vs + ec];
    double W[PDE::NW > 0 ? PDE::NW : 1];
    PDE::prims(qn, A.P, W);
#pragma unroll
    for (int i = 0; i < PDE::NW; ++i) A.w_out[i * A.vs + ec] = W[i];
  }
}

// One CTA per (fine patch, parent) pair: the (p/2)^d covered coarse voxels x N variables.
__global__ void __launch_bounds__(256) k_restrict(const __grid_constant__ CplArgs A, int nq) {
  const int2 fp = A.restrict_list[blockIdx.x];
  const dh_patch& F = A.patches[fp.x];
  const dh_patch& Pp = A.patches[fp.y];
  const int p = F.p, h = p >> 1, o = A.oct[fp.x];
  const int hz = A.dim == 3 ? h : 1;
  const int nvox = h * h * hz;
  for (int t = threadIdx.x; t < nvox * nq; t += blockDim.x) {
    const int v = t / nvox, r = t - v * nvox;
    const int x = r % h, y = (r / h) % h, z = r / (h * h);
    const int cx = (o & 1) * h + x, cy = ((o >> 1) & 1) * h + y, cz = A.dim == 3 ? ((o >> 2) & 1) * h + z : 0;
    const int64_t ec = Pp.offset + ((int64_t)cz * p + cy) * p + cx;
    for (int w = 0; w < 2; ++w) {
      double* arr = w == 0 ? A.out : A.acc;
      if (!arr) continue;
      arr[(int64_t)v * A.vs + ec] = fine_mean(arr + (int64_t)v * A.vs + F.offset, p, A.dim, x, y, z);
    }
  }
}

inline int lattice(const dh_patch& P, int a) { return (int)std::llround(P.x0[a] / (P.p * P.dx)); }

template <class PDE>
dh_status couple_pde(dh_plan* plan, CplArgs A, cudaStream_t s) {
  // one launch for all entries when no coarse voxel has entries in two directions,
  // else one launch per direction
  const int groups = plan->amr_reflux_single ? 1 : 6;
  for (int f = 0; f < groups; ++f) {
    const int lo = plan->amr_reflux_off[f], hi = plan->amr_reflux_single ? plan->amr_reflux_off[6] : plan->amr_reflux_off[f + 1];
    const int n = hi - lo;
    if (n == 0) continue;
    A.reflux = plan->d_amr_reflux + lo;
    A.n = n;
    k_reflux<PDE><<<(n + 63) / 64, 64, 0, s>>>(A);
    dh_status st = cuda_error(cudaGetLastError(), "k_reflux launch");
    if (st != DH_OK) return st;
  }
  for (size_t l = 0; l + 1 < plan->amr_restrict_off.size(); ++l) {
    const int n = plan->amr_restrict_off[l + 1] - plan->amr_restrict_off[l];
    if (n == 0) continue;
    A.restrict_list = plan->d_amr_restrict + plan->amr_restrict_off[l];
    // the raw sums of the stage-sum form are never read for covered coarse voxels
    if (A.form != 0) A.acc = nullptr;
    if (A.w_out && A.out) k_restrict_w<PDE><<<n, 256, 0, s>>>(A);
    else k_restrict<<<n, 256, 0, s>>>(A, plan->nq);
    dh_status st = cuda_error(cudaGetLastError(), "k_restrict launch");
    if (st != DH_OK) return st;
  }
  return DH_OK;
}

}  // namespace

// Host-side analysis of the patch table: coupled faces, octants, parents,
// reflux entries and restriction pairs.  Returns DH_EINVAL on an unsupported
// coupling (the message names the patch).
dh_status amr_build(dh_plan* plan, const dh_patch* patches, int K, int dim) {
  bool coupled = false;
  for (int k = 0; k < K && !coupled; ++k)
    for (int f = 0; f < 2 * dim; ++f)
      if (patches[patches[k].nbr[f]].level != patches[k].level) coupled = true;
  plan->coupled = coupled;
  if (!coupled) return DH_OK;
  for (int k = 0; k < K; ++k)
    for (int f = 0; f < 2 * dim; ++f) {
      const dh_patch& n = patches[patches[k].nbr[f]];
      if (n.level == patches[k].level) continue;
      if (n.level != patches[k].level - 1 || n.p != patches[k].p || n.dx != 2.0 * patches[k].dx) {
        set_error("patch %d: neighbour %d must have the same level, or be one level coarser with the same p and "
                  "twice the dx", k, f);
        return DH_EINVAL;
      }
    }
  std::map<std::tuple<int, int, int, int>, int> at;
  std::vector<int> oct(K, 0);
  for (int k = 0; k < K; ++k) {
    int c[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
      c[a] = lattice(patches[k], a);
      oct[k] |= (c[a] & 1) << a;
    }
    at[std::make_tuple(patches[k].level, c[0], c[1], c[2])] = k;
  }
  // parents of every patch above the coarsest level present
  int lmin = patches[0].level, lmax = patches[0].level;
  for (int k = 1; k < K; ++k) { lmin = std::min(lmin, patches[k].level); lmax = std::max(lmax, patches[k].level); }
  std::vector<int> par(K, -1);
  std::vector<std::vector<int2>> by_level(lmax - lmin + 1);
  for (int k = 0; k < K; ++k) {
    if (patches[k].level == lmin) continue;
    const int c0 = lattice(patches[k], 0) / 2, c1 = lattice(patches[k], 1) / 2, c2 = dim == 3 ? lattice(patches[k], 2) / 2 : 0;
    auto it = at.find(std::make_tuple(patches[k].level - 1, c0, c1, c2));
    if (it == at.end() || patches[it->second].p != patches[k].p || patches[it->second].dx != 2.0 * patches[k].dx) {
      set_error("patch %d (level %d): no covering patch one level coarser (needed for restriction)", k,
                patches[k].level);
      return DH_EINVAL;
    }
    par[k] = it->second;
    by_level[patches[k].level - lmin].push_back(make_int2(k, par[k]));
  }
  plan->amr_restrict_off.assign(1, 0);
  std::vector<int2> rl;
  for (int l = lmax - lmin; l >= 1; --l) {  // finest level first
    rl.insert(rl.end(), by_level[l].begin(), by_level[l].end());
    plan->amr_restrict_off.push_back((int)rl.size());
  }
  // reflux entries by face direction of the fine patch
  std::vector<AmrReflux> ent[6];
  for (int k = 0; k < K; ++k) {
    const dh_patch& F = patches[k];
    const int p = F.p, h = p / 2;
    for (int f = 0; f < 2 * dim; ++f) {
      const int C = F.nbr[f];
      if (patches[C].level >= F.level) continue;
      const int a = f / 2, lo = f % 2 == 0;
      const int b0 = (a + 1) % dim, b1 = dim == 3 ? (a + 2) % dim : -1;
      const int stride[3] = {1, p, p * p};
      for (int kk = 0; kk < (dim == 3 ? h : 1); ++kk)
        for (int jj = 0; jj < h; ++jj) {
          int cc[3] = {0, 0, 0}, cn[3] = {0, 0, 0}, cf[3] = {0, 0, 0};
          cc[a] = lo ? p - 1 : 0;
          cn[a] = ((oct[k] >> a) & 1) * h + (lo ? 0 : h - 1);
          cf[a] = lo ? 0 : p - 1;
          cc[b0] = cn[b0] = ((oct[k] >> b0) & 1) * h + jj;
          cf[b0] = 2 * jj;
          if (b1 >= 0) { cc[b1] = cn[b1] = ((oct[k] >> b1) & 1) * h + kk; cf[b1] = 2 * kk; }
          AmrReflux R;
          R.C = C; R.N = par[k]; R.F = k;
          R.eC = (cc[2] * p + cc[1]) * p + cc[0];
          R.eN = (cn[2] * p + cn[1]) * p + cn[0];
          R.eF = (cf[2] * p + cf[1]) * p + cf[0];
          R.sb0 = stride[b0];
          R.sb1 = b1 >= 0 ? stride[b1] : 0;
          R.axis = a;
          R.lo = lo;
          ent[f].push_back(R);
        }
    }
  }
  std::vector<AmrReflux> all;
  plan->amr_reflux_off[0] = 0;
  for (int f = 0; f < 6; ++f) {
    all.insert(all.end(), ent[f].begin(), ent[f].end());
    plan->amr_reflux_off[f + 1] = (int)all.size();
  }
  {
    std::vector<std::pair<int, int>> keys;
    keys.reserve(all.size());
    for (const AmrReflux& R : all) keys.push_back(std::make_pair(R.C, R.eC));
    std::sort(keys.begin(), keys.end());
    plan->amr_reflux_single = std::adjacent_find(keys.begin(), keys.end()) == keys.end();
  }
  cudaError_t e = cudaMalloc(&plan->d_amr_oct, sizeof(int) * K);
  if (e == cudaSuccess) e = cudaMemcpy(plan->d_amr_oct, oct.data(), sizeof(int) * K, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !all.empty()) e = cudaMalloc(&plan->d_amr_reflux, sizeof(AmrReflux) * all.size());
  if (e == cudaSuccess && !all.empty())
    e = cudaMemcpy(plan->d_amr_reflux, all.data(), sizeof(AmrReflux) * all.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !rl.empty()) e = cudaMalloc(&plan->d_amr_restrict, sizeof(int2) * rl.size());
  if (e == cudaSuccess && !rl.empty())
    e = cudaMemcpy(plan->d_amr_restrict, rl.data(), sizeof(int2) * rl.size(), cudaMemcpyHostToDevice);
  return cuda_error(e, "amr_build");
}

// Reflux and restriction after a first-order FV stage on a coupled plan.
dh_status amr_couple(dh_plan* plan, const double* qs, const double* mat, double* out, double* acc,
                     const double* dt_dev, double g, double d, cudaStream_t s, int form, double* w_out) {
  CplArgs A{};
  A.w_out = w_out;
  A.patches = plan->d_patches;
  A.oct = plan->d_amr_oct;
  A.qs = qs; A.mat = mat; A.out = out; A.acc = acc; A.dt_dev = dt_dev;
  A.g = g; A.d = d;
  A.form = form;
  A.vs = plan->var_stride;
  A.dim = plan->dim;
  A.P = plan->params;
  switch (plan->pde) {
    case DH_PDE_ADV_FLUX: return couple_pde<PdeAdvFlux>(plan, A, s);
    case DH_PDE_EULER2D: return couple_pde<PdeEuler2>(plan, A, s);
    case DH_PDE_EULER3D: return couple_pde<PdeEuler3>(plan, A, s);
    case DH_PDE_SRHD3D: return couple_pde<PdeSRHD>(plan, A, s);
    default:
      set_error("coupled refinement levels: PDE %d not supported (conservative systems only)", plan->pde);
      return DH_EUNSUPPORTED;
  }
}

}  // namespace dh
