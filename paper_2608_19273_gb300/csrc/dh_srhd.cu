// Conservative -> primitive recovery for special-relativistic hydrodynamics:
// per voxel, FP64 Newton iteration on the pressure, seeded either by the
// previous pressure (plain) or by the FP32 MLP guess, with the plain seed as
// fallback.  (The paper has no SRHD; definitions are the textbook ones.)
//
//   E = tau + D, S^2 = |S|^2, bracket p > p_lo = max(0, |S| - E)
//   f(p)  = ((G-1)/G) [ (E+p) - S^2/(E+p) - D sqrt(1 - S^2/(E+p)^2) ] - p
//   f'(p) = ((G-1)/G) [ 1 + S^2/(E+p)^2 - D S^2 / ((E+p)^3 sqrt(1 - S^2/(E+p)^2)) ] - 1
//   p <- p - f/f'; a step that leaves the bracket is replaced by the midpoint
//   between the current iterate and p_lo and never counts as convergence;
//   converged when |p_new - p| <= tol p_new; at most max_iter steps.
//   Seeds: MLP (if weights given) -> p_prev (if given) -> cold seed
//   max((1 + 1e-8) p_lo + 1e-300, (G-1) tau); the first seed is tried, the
//   second only if the first fails.  With seed_refine = k > 0 the first seed is
//   first refined by up to k FP32 Newton steps (refine_seed_f32); the second seed
//   (plain Newton from the previous pressure) never is.  status: 0 first seed converged, 1 second
//   seed converged, 2 both failed (p = p_prev or the cold seed, counted in
//   fail_count).  Recovery: v = S/(E+p), W = 1/sqrt(1 - v^2), rho = D/W.
// Failures never trap: they are reported through status and the counter.
#include "dh_internal.cuh"
#include "dh_mlp.cuh"
#include "dh_pde.cuh"

namespace dh {

// Returns iterations used (> 0) on convergence, -iterations on failure.
// The Newton step is evaluated in an equivalent algebraic form that needs one
// reciprocal and one reciprocal square root per iteration.  With y = E + p and
// q = sqrt(y^2 - S^2) = y sqrt(1 - S^2/y^2) (the square-root term of f is D q / y):
//   y f  = gf q (q - D) - p y          (gf = (G-1)/G)
//   y^2 f' = gf S^2 (q - D)/q + (gf - 1) y^2
//   p_new = p - (y^2 f) / (y^2 f') = p - y (gf q (q - D) - p y) / (gf S^2 (q - D)/q + (gf - 1) y^2)
// The root and the iterates agree with the textbook form to rounding (the
// stopping test still compares successive iterates).  Adds and products are
// issued as FMAs with the run-time constants one/mone/zero (GB300 runs DFMA
// faster than DADD/DMUL; results are bitwise the same); the reciprocal is a
// refined hardware estimate (recip_nr, one third-order step, <= 1 ulp from the
// IEEE quotient), and so is the reciprocal square root (rsqrt_pos, one third-order
// step, within two ulps).  A state whose y^2 - S^2 is not positive gives NaN (failure).
__device__ int srhd_newton_dev(double gf, double D, double S2, double E, double p_lo, double p0, double tol,
                               int max_iter, double one, double mone, double zero, double* p_out) {
  const double gfS2 = fma(gf, S2, zero), gm1 = fma(gf, one, mone);
  double p = p0;
  for (int it = 1; it <= max_iter; ++it) {
    const double y = fma(E, one, p);
    const double d = fma(y, y, -S2);                      // q^2
    const double iq = rsqrt_pos(d);                       // 1/q
    const double q = fma(d, iq, zero);
    const double qmD = fma(D, mone, q);                   // q - D
    const double num = fma(fma(-p, y, fma(fma(gf, q, zero), qmD, zero)), y, zero);   // y^2 f
    const double den = fma(fma(gm1, y, zero), y, fma(fma(gfS2, qmD, zero), iq, zero)); // y^2 f'
    double pn = fma(-num, recip_nr(den), p);
    // The three tests below compare bit patterns on the integer pipe: p_lo,
    // |pn - p| and tol pn are non-negative, and a non-negative double orders
    // like its bits read as a signed 64-bit integer (a negative pn reads as a
    // negative integer, so it still compares below p_lo).
    const long long ipn = __double_as_longlong(pn);
    if ((ipn & 0x7fffffffffffffffll) > 0x7ff0000000000000ll) { *p_out = pn; return -it; }  // NaN
    if (ipn <= __double_as_longlong(p_lo)) {
      pn = fma(0.5, p, 0.5 * p_lo);
    } else if (__double_as_longlong(fabs(fma(pn, one, -p))) <= __double_as_longlong(fma(tol, pn, zero))) {
      *p_out = pn;
      return it;
    }
    p = pn;
  }
  *p_out = p;
  return -max_iter;
}

// FP32 refinement of the first seed: up to k Newton steps on the pressure in single
// precision.  The terms of the textbook f cancel in FP32 for fast flows (1 - S^2/(E+p)^2 is
// 0.01 at W = 10) and for cold gas (the rest mass D against rho h W), which leaves seeds a few
// 1e-5 off; the step is therefore formed from two invariants taken once in FP64 with fused
// multiply-adds, A = E^2 - S^2 and B = tau (tau + 2 D) - S^2 = A - D^2, in which nothing
// cancels during the iteration: with y = E + p and t = p (E + y) = y^2 - E^2,
//   q = sqrt(y^2 - S^2) = sqrt(A + t),  q - D = (q^2 - D^2)/(q + D) = (B + t)/(q + D),
//   y f = gf q (q - D) - p y,  y^2 f' = gf S^2 (q - D)/q + (gf - 1) y^2  (the FP64 step's form),
//   p <- p - y (y f)/(y^2 f').
// Every FP32 operation is IEEE-rounded with no fused multiply-add (the __f*_rn intrinsics) on
// float copies of A, B, E, D and S^2; a step whose result is not finite or not above the
// bracket's lower end (in float) stops the refinement and keeps the value before it.  The same
// operations in the same order as the oracle's reference, so the refined seed is bitwise the
// oracle's; the seeds land within about 1e-6 of the root, from which two FP64 Newton steps meet
// the 1e-12 rule.  FP32 runs far faster than FP64 on this GPU: the steps cost little next to
// one FP64 Newton iteration.
__device__ __forceinline__ double refine_seed_f32(const double* q, double E, double S2, double p_lo, double seed,
                                                  int k, float gf) {
  const double A = __fma_rn(E, E, -S2), B = __fma_rn(q[4], __fma_rn(2.0, q[0], q[4]), -S2);
  // the conversions run on the integer pipes (f32_rn: the hardware's rounding, bit for bit)
  const float Af = f32_rn(A), Bf = f32_rn(B), Ef = f32_rn(E);
  const float Df = f32_rn(q[0]), S2f = f32_rn(S2);
  const float lo = __double_as_longlong(p_lo) == 0 ? 0.0f : f32_rn(p_lo);
  const float gm = __fsub_rn(gf, 1.0f);
  float p = f32_rn(seed);
  for (int i = 0; i < k; ++i) {
    const float y = __fadd_rn(Ef, p);
    const float t = __fmul_rn(p, __fadd_rn(Ef, y));
    const float qq = __fsqrt_rn(__fadd_rn(Af, t));
    const float qmD = __fdiv_rn(__fadd_rn(Bf, t), __fadd_rn(qq, Df));
    const float yf = __fsub_rn(__fmul_rn(__fmul_rn(gf, qq), qmD), __fmul_rn(p, y));
    const float den = __fadd_rn(__fdiv_rn(__fmul_rn(__fmul_rn(gf, S2f), qmD), qq), __fmul_rn(__fmul_rn(gm, y), y));
    const float pn = __fsub_rn(p, __fdiv_rn(__fmul_rn(y, yf), den));
    if (!(pn > lo && pn < __int_as_float(0x7f800000))) break;
    p = pn;
  }
  return f64_of_f32(p);
}

struct C2PArgs {
  const double* cons;
  double* prim;
  const double* p_prev;
  const float* mlp;
  double tol;
  int max_iter;
  int refine;              // FP32 Newton steps applied to the first seed (0: none)
  float gf32;              // (G - 1)/G rounded to float (the refinement's constant)
  uint8_t* status;
  int32_t* iters;
  int32_t* fail_count;
  int64_t vs;
  double G;
  double gf;               // (G - 1)/G
  double one, mone, zero;  // 1, -1, 0 for the FMA forms of adds and products
};

__device__ __forceinline__ int c2p_voxel(const C2PArgs& A, const float* w, int64_t e) {
  const int64_t vs = A.vs;
  double q[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) q[v] = A.cons[v * vs + e];
  const double G = A.G;
  const double D = q[0], E = q[4] + q[0];
  const double S2 = fma(q[1], q[1], fma(q[2], q[2], q[3] * q[3]));
  // p_lo = max(0, |S| - E) (+0, never -0).  For E > 0 and |S|^2 < E^2 (1 - 2^-50) the
  // correctly rounded |S| lies below E whatever the roundings of that bound, so p_lo = 0
  // without the square root (the usual case: physical states have |S| < E); the learned
  // seed needs |S| itself.
  double S = 0.0, p_lo = 0.0;
  const bool ref = A.refine > 0;
  if ((w && !ref) || !(E > 0.0 && S2 < E * E * (1.0 - 0x1p-50))) {
    S = sqrt(S2);
    p_lo = S > E ? S - E : 0.0;
  }
  // the cold seed is formed only where it is used
  auto cold = [&]() { return fmax(fma(1.0 + 1e-8, p_lo, 1e-300), (G - 1.0) * q[4]); };
  const bool have_prev = A.p_prev != nullptr;
  double s1;
  bool have2;
  if (w) {
    float x[3], h1[32], h2[32];
    // with the FP32 refinement the seed's |S| and exp are FP32 too (the refinement is)
    mlp_inputs_f32(w, D, E, ref ? f64_of_f32(__fsqrt_rn(f32_rn(S2))) : S, x);
    const float y = mlp_forward(w, x, h1, h2);
    const double ps = ref ? f64_of_f32(__fmul_rn(f32_rn(E), expf(y))) : E * exp((double)y);
    const double lo = p_lo * (1.0 + 1e-12);
    s1 = ps > lo ? ps : cold();
    have2 = true;
  } else {
    s1 = have_prev ? A.p_prev[e] : cold();
    have2 = have_prev;
  }
  if (ref) s1 = refine_seed_f32(q, E, S2, p_lo, s1, A.refine, A.gf32);
  double p;
  int it1 = srhd_newton_dev(A.gf, D, S2, E, p_lo, s1, A.tol, A.max_iter, A.one, A.mone, A.zero, &p);
  int total = it1 > 0 ? it1 : -it1;
  uint8_t st = 0;
  if (it1 <= 0) {
    int it2 = 0;
    if (have2) {
      // second seed: the previous pressure after the learned one, else the cold seed
      const double s2 = (w && have_prev) ? A.p_prev[e] : cold();
      it2 = srhd_newton_dev(A.gf, D, S2, E, p_lo, s2, A.tol, A.max_iter, A.one, A.mone, A.zero, &p);
      total += it2 > 0 ? it2 : -it2;
    }
    if (have2 && it2 > 0) st = 1;
    else { st = 2; p = have_prev ? A.p_prev[e] : cold(); }
  }
  const double rEp = recip_nr(E + p);
  const double vx = q[1] * rEp, vy = q[2] * rEp, vz = q[3] * rEp;
  const double v2 = fma(vx, vx, fma(vy, vy, vz * vz));
  // rho = D / W = D sqrt(1 - v^2)
  A.prim[e] = D * sqrt_pos(1.0 - v2);
  A.prim[vs + e] = vx;
  A.prim[2 * vs + e] = vy;
  A.prim[3 * vs + e] = vz;
  A.prim[4 * vs + e] = p;
  if (A.status) A.status[e] = st;
  if (A.iters) A.iters[e] = total;
  return st == 2 ? 1 : 0;
}

__device__ __forceinline__ void load_mlp_smem(const float* src, float* dst) {
  for (int i = threadIdx.x; i < MLP_LEN; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

__device__ __forceinline__ void count_failures(int nfail, int32_t* fail_count) {
  // warp-aggregated counter update (order-independent integer sum)
  const unsigned m = __ballot_sync(0xffffffffu, nfail != 0);
  if (fail_count && (threadIdx.x & 31) == 0 && m) atomicAdd(fail_count, __popc(m));
}

// One CTA per patch.
__global__ void __launch_bounds__(256) k_con2prim_patches(const dh_patch* __restrict__ patches, int dim,
                                                          const __grid_constant__ C2PArgs A) {
  __shared__ __align__(16) float w[MLP_LEN];
  if (A.mlp) load_mlp_smem(A.mlp, w);
  const dh_patch pt = patches[blockIdx.x];
  const int n = dim == 3 ? pt.p * pt.p * pt.p : pt.p * pt.p;
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    int f = 0;
    if (i < n) f = c2p_voxel(A, A.mlp ? w : nullptr, pt.offset + i);
    count_failures(f, A.fail_count);
  }
}

// Flat array of n voxels (element i of variable v at v * stride + i).
__global__ void __launch_bounds__(256) k_con2prim_flat(int64_t n, const __grid_constant__ C2PArgs A) {
  __shared__ __align__(16) float w[MLP_LEN];
  if (A.mlp) load_mlp_smem(A.mlp, w);
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    int f = 0;
    if (i < n) f = c2p_voxel(A, A.mlp ? w : nullptr, i);
    count_failures(f, A.fail_count);
  }
}

// Diagnostic of the integer-pipe conversions against the hardware's.
__global__ void k_check_convert(const double* x, float* f_int, float* f_hw, const float* g, double* d_int,
                                double* d_hw, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  f_int[i] = f32_rn(x[i]);
  f_hw[i] = __double2float_rn(x[i]);
  d_int[i] = f64_of_f32(g[i]);
  d_hw[i] = (double)g[i];
}

static dh_status c2p_check(const double* cons, double* prim, double tol, int32_t max_iter, int32_t seed_refine) {
  if (!cons || !prim || cons == prim) { set_error("con2prim: cons and prim are required and distinct"); return DH_EINVAL; }
  if (!(tol > 0.0) || max_iter < 1 || max_iter > 1000) { set_error("con2prim: tol > 0 and 1 <= max_iter <= 1000 required"); return DH_EINVAL; }
  if (seed_refine < 0 || seed_refine > 8) { set_error("con2prim: seed_refine must lie in [0, 8]"); return DH_EINVAL; }
  return DH_OK;
}

}  // namespace dh

using namespace dh;

extern "C" {

dh_status con2prim(dh_plan* plan, const double* cons, double* prim, const double* p_prev, const float* mlp_w,
                   double tol, int32_t max_iter, int32_t seed_refine, uint8_t* status, int32_t* iters,
                   int32_t* fail_count_dev, void* stream) {
  if (!plan) { set_error("plan is NULL"); return DH_EINVAL; }
  if (plan->pde != DH_PDE_SRHD3D) { set_error("con2prim: the plan's PDE is not SRHD3D"); return DH_EUNSUPPORTED; }
  dh_status st = c2p_check(cons, prim, tol, max_iter, seed_refine);
  if (st != DH_OK) return st;
  const double G = plan->params.Gamma;
  C2PArgs A{cons, prim, p_prev, mlp_w, tol, max_iter, seed_refine, (float)((G - 1.0) / G), status, iters,
            fail_count_dev, plan->var_stride, G, (G - 1.0) / G, 1.0, -1.0, 0.0};
  k_con2prim_patches<<<plan->K, 256, 0, (cudaStream_t)stream>>>(plan->d_patches, plan->dim, A);
  return cuda_error(cudaGetLastError(), "con2prim launch");
}

dh_status con2prim_flat(const double* cons, double* prim, int64_t n, int64_t stride, const double* p_prev,
                        const float* mlp_w, double Gamma, double tol, int32_t max_iter, int32_t seed_refine,
                        uint8_t* status, int32_t* iters, int32_t* fail_count_dev, void* stream) {
  dh_status st = c2p_check(cons, prim, tol, max_iter, seed_refine);
  if (st != DH_OK) return st;
  if (n <= 0 || stride < n) { set_error("con2prim_flat: need 0 < n <= stride"); return DH_EINVAL; }
  if (!(Gamma > 1.0)) { set_error("con2prim_flat: Gamma must exceed 1"); return DH_EINVAL; }
  C2PArgs A{cons, prim, p_prev, mlp_w, tol, max_iter, seed_refine, (float)((Gamma - 1.0) / Gamma), status, iters,
            fail_count_dev, stride, Gamma, (Gamma - 1.0) / Gamma, 1.0, -1.0, 0.0};
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n + 255) / 256;
  const int grid = (int)std::min<int64_t>(want, (int64_t)sms * 8);
  k_con2prim_flat<<<grid, 256, 0, (cudaStream_t)stream>>>(n, A);
  return cuda_error(cudaGetLastError(), "con2prim_flat launch");
}

dh_status dh_check_convert(const double* x, float* f_int, float* f_hw, const float* g, double* d_int, double* d_hw,
                           int64_t n, void* stream) {
  if (!x || !f_int || !f_hw || !g || !d_int || !d_hw || n <= 0 || n > (1ll << 40)) {
    set_error("dh_check_convert: bad arguments");
    return DH_EINVAL;
  }
  k_check_convert<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, f_int, f_hw, g, d_int, d_hw, n);
  return cuda_error(cudaGetLastError(), "dh_check_convert launch");
}

}  // extern "C"
