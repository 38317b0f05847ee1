// PDE terms of Eq. 1 (dQ/dt + div F(Q) + B(Q).grad Q = S(Q)) as device functors.
//
// Each system provides, per voxel, the derived quantities W (computed once per
// voxel and shared by all directions), the flux F_d, the largest
// characteristic speed lambda_d, the non-conservative product B_d(Qb).dQ and
// the source S.  The direction d may be a run-time value: it is only used in
// selects, never to index a register array, so the same code serves interior
// voxels (d unrolled) and halo voxels of either direction without divergence.
#pragma once

#include <type_traits>

#include "dh_internal.cuh"

namespace dh {

__device__ __forceinline__ double sel3(int d, double a, double b, double c) {
  return d == 0 ? a : (d == 1 ? b : c);
}

// GB300 issues FP64 fused multiply-adds with register operands at 2.0 per
// clock per SM, but DADD, DMUL and FP64 instructions with a constant-bank
// operand (a kernel parameter or a literal) at 1.68 (measured).  The FV stage
// therefore writes its adds, subtractions and products as FMAs whose extra
// operand is 1, -1 or 0 from its parameters (values the compiler cannot see,
// so it cannot turn them back into DADD/DMUL), and its kernels copy those
// parameters into registers once per thread (a shuffle hides them from the
// compiler, which would fold them into constant-bank operands).  The FD stage
// keeps plain operations (the FMA form measured 7% slower there with
// constant-bank operands, and no faster with register operands).  The results are bitwise those of a + b, a - b and a * b (a
// product that is -0 comes out as +0).
__device__ __forceinline__ double ADD(const DevParams& P, double a, double b) { return fma(a, P.one, b); }
__device__ __forceinline__ double SUB(const DevParams& P, double a, double b) { return fma(b, P.mone, a); }
__device__ __forceinline__ double MUL(const DevParams& P, double a, double b) { return fma(a, b, P.zero); }

// 1/a for a normal, finite, positive or negative a: the hardware reciprocal
// estimate y (PTX rcp.approx.ftz.f64, relative error below 2^-19.9 over 2^28
// sampled mantissas and exponents on GB300) refined by one step of the
// third-order (Householder, order 2) iteration for f(y) = 1/y - a:
// with e = 1 - a y, 1/a = y / (1 - e) = y (1 + e + e^2 + e^3 + ...), and
// y (1 + e + e^2) leaves a relative error of e^3 < 2^-59.  Three FMAs instead of
// a full IEEE division (about 5.7 FMA times); the result is within one unit
// in the last place of the correctly rounded reciprocal (checked against 1.0/a
// by the GPU tests).
__device__ __forceinline__ double recip_nr(double a) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
  const double e = fma(-a, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

// 1/sqrt(x) for normal, finite x > 0: the hardware estimate y (PTX
// rsqrt.approx.ftz.f64, relative error below 1e-6 over 2^22 samples spanning the
// normal range on GB300) refined by one third-order step of the binomial series
// (1 - e)^(-1/2) = 1 + e/2 + 3e^2/8 + 5e^3/16 + ...  with e = 1 - x y^2 (formed by an
// FMA): y (1 + e/2 + 3e^2/8) leaves a relative error of about 5e^3/16 < 1e-18, so
// the result is within two units in the last place of the correctly rounded value
// (checked by the GPU tests).  Five FP64 operations.
__device__ __forceinline__ double rsqrt_nr(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x * y, y, 1.0);
  return fma(y * e, fma(0.375, e, 0.5), y);
}

// 1/sqrt(x): rsqrt_nr for normal, finite x > 0; zero, subnormal, negative, infinite and NaN
// arguments take rsqrt itself (bit tests on the integer pipe).
__device__ __forceinline__ double rsqrt_pos(double x) {
  const long long b = __double_as_longlong(x);
  return (b >= 0x0010000000000000ll && b < 0x7ff0000000000000ll) ? rsqrt_nr(x) : rsqrt(x);
}

// sqrt(x) for finite x > 0 from the same estimate: with s = x y and e = 1 - s y,
// sqrt(x) = s (1 - e)^(-1/2) = s (1 + e/2 + 3e^2/8 + ...), the same third-order step
// (five FP64 operations; within two units in the last place of the correctly rounded
// square root, checked by the GPU tests).  Zero, subnormal, negative, infinite and NaN
// arguments take sqrt itself.  The bit tests run on the integer pipe.
__device__ __forceinline__ double sqrt_pos(double x) {
  const long long b = __double_as_longlong(x);
  if (b >= 0x0010000000000000ll && b < 0x7ff0000000000000ll) {
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double s = x * y;
    const double e = fma(-s, y, 1.0);
    return fma(s * e, fma(0.375, e, 0.5), s);
  }
  return sqrt(x);
}

// max(a, b) for a, b >= +0 (characteristic speeds): non-negative doubles order
// like their bit patterns read as signed 64-bit integers, so the comparison
// runs on the integer pipe instead of the FP64 pipe.
__device__ __forceinline__ double max_nn(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  return __longlong_as_double(ia > ib ? ia : ib);
}

// ---------------------------------------------------------------- advection
// dq/dt + div(a q) = 0 with material velocity a (M = 3).  F_d = a_d q, lambda_d = |a_d|.
struct PdeAdvFlux {
  static constexpr int N = 1, M = 3, NW = 1, DIM = 3;
  static constexpr bool FLUX = true, NCP = false, SRC = false, SYM = false;
  __device__ static void prims(const double*, const DevParams&, double*) {}
  __device__ static void flux(int d, const double* q, const double*, const DevParams& P, double* F) {
    F[0] = MUL(P, sel3(d, q[1], q[2], q[3]), q[0]);
  }
  __device__ static double speed(int d, const double* q, const double*, const DevParams&) {
    return fabs(sel3(d, q[1], q[2], q[3]));
  }
  __device__ static void ncp(int, const double*, const double*, const DevParams&, double*) {}
  __device__ static void source(const double*, const double*, const DevParams&, double*) {}
};

// dq/dt + a . grad q = 0 (non-conservative form, F = 0): B_d = a_d.
struct PdeAdvNcp {
  static constexpr int N = 1, M = 3, NW = 1, DIM = 3;
  static constexpr bool FLUX = false, NCP = true, SRC = false, SYM = false;
  __device__ static constexpr bool needs_grad(int, int v) { return v == 0; }
  __device__ static void prims(const double*, const DevParams&, double*) {}
  __device__ static void flux(int, const double*, const double*, const DevParams&, double*) {}
  __device__ static double speed(int d, const double* q, const double*, const DevParams&) {
    return fabs(sel3(d, q[1], q[2], q[3]));
  }
  // qb holds N + M midpoint values (evolved then material).
  __device__ static void ncp(int d, const double* qb, const double* dq, const DevParams& P, double* D) {
    D[0] = MUL(P, sel3(d, qb[1], qb[2], qb[3]), dq[0]);
  }
  __device__ static void source(const double*, const double*, const DevParams&, double*) {}
};

// ---------------------------------------------------------------- Euler
// Ideal-gas Euler equations in DIM dimensions: Q = (rho, rho u_k, E).
// W = (u_0 .. u_{DIM-1}, p, c, H = E + p): one reciprocal and one square root per voxel.
template <int D_>
struct PdeEuler {
  static constexpr int DIM = D_, N = D_ + 2, M = 0, NW = D_ + 3;
  static constexpr bool FLUX = true, NCP = false, SRC = false, SYM = true;
  __device__ static void prims(const double* q, const DevParams& P, double* w) {
    const double r = recip_nr(q[0]);
    w[0] = MUL(P, q[1], r);
    double kin = MUL(P, q[1], w[0]);
#pragma unroll
    for (int k = 1; k < DIM; ++k) {
      w[k] = MUL(P, q[1 + k], r);
      kin = fma(q[1 + k], w[k], kin);
    }
    const double p = MUL(P, P.gm1, fma(-0.5, kin, q[DIM + 1]));
    w[DIM] = p;
    w[DIM + 1] = sqrt_pos(MUL(P, MUL(P, P.gamma, p), r));
    w[DIM + 2] = ADD(P, q[DIM + 1], p);
  }
  // The momentum flux rho u_k u_d is symmetric in (k, d); every direction forms
  // it as m_min(k,d) u_max(k,d), so the x, y and z fluxes of one voxel share
  // their off-diagonal products bit for bit (flux_xy).
  __device__ static void flux(int d, const double* q, const double* w, const DevParams& P, double* F) {
    const double u = (DIM == 3) ? sel3(d, w[0], w[1], w[DIM == 3 ? 2 : 0]) : (d == 0 ? w[0] : w[1]);
    const double p = w[DIM];
    F[0] = (DIM == 3) ? sel3(d, q[1], q[2], q[DIM == 3 ? 3 : 1]) : (d == 0 ? q[1] : q[2]);
#pragma unroll
    for (int k = 0; k < DIM; ++k)
      F[1 + k] = fma(k < d ? q[1 + k] : F[0], k < d ? u : w[k], d == k ? p : P.zero);
    F[DIM + 1] = MUL(P, w[DIM + 2], u);
  }
  // F_x and F_y of a voxel whose F_z (3D) is already formed: the same values as
  // flux(0) and flux(1), with the products m_x u_y, m_x u_z, m_y u_z formed once.
  __device__ static void flux_xy(const double* q, const double* w, const double* Fz, const DevParams& P, double* Fx,
                                 double* Fy) {
    const double p = w[DIM], cxy = MUL(P, q[1], w[1]);
    Fx[0] = q[1];
    Fx[1] = fma(q[1], w[0], p);
    Fx[2] = cxy;
    Fy[0] = q[2];
    Fy[1] = cxy;
    Fy[2] = fma(q[2], w[1], p);
    if (DIM == 3) {
      Fx[DIM == 3 ? 3 : 0] = Fz[1];
      Fy[DIM == 3 ? 3 : 0] = Fz[2];
    }
    Fx[DIM + 1] = MUL(P, w[DIM + 2], w[0]);
    Fy[DIM + 1] = MUL(P, w[DIM + 2], w[1]);
  }
  __device__ static double speed(int d, const double*, const double* w, const DevParams& P) {
    const double u = (DIM == 3) ? sel3(d, w[0], w[1], w[DIM == 3 ? 2 : 0]) : (d == 0 ? w[0] : w[1]);
    return ADD(P, fabs(u), w[DIM + 1]);
  }
  __device__ static void ncp(int, const double*, const double*, const DevParams&, double*) {}
  __device__ static void source(const double*, const double*, const DevParams&, double*) {}
};

using PdeEuler2 = PdeEuler<2>;
using PdeEuler3 = PdeEuler<3>;

// ---------------------------------------------------------------- SRHD
// Special-relativistic hydrodynamics, Q = (D, S_x, S_y, S_z, tau), ideal gas Gamma.
// The material slots carry the primitives (rho, v_x, v_y, v_z, p) recovered by
// con2prim.  W = (v_x, v_y, v_z, p, 1 - cs^2, cs^2 (1 - v^2), 1 - v^2 cs^2,
// 1/(1 - v^2 cs^2)): the direction-independent factors of the speeds.
//   F_d = (D v_d, S v_d + p e_d, S_d - D v_d)
//   lambda_pm = [v_d (1 - cs^2) +- cs sqrt((1 - v^2)(1 - v^2 cs^2 - v_d^2 (1 - cs^2)))] / (1 - v^2 cs^2)
//   max(|lambda_+|, |lambda_-|) = (|v_d| (1 - cs^2) + sqrt(cs^2 (1 - v^2)(...))) / (1 - v^2 cs^2)
// (cs is folded under the square root: one square root per direction, none per voxel).
struct PdeSRHD {
  static constexpr int N = 5, M = 5, NW = 8, DIM = 3;
  static constexpr bool FLUX = true, NCP = false, SRC = false, SYM = true;
  __device__ static void prims(const double* q, const DevParams& P, double* w) {
    const double rho = q[5], vx = q[6], vy = q[7], vz = q[8], p = q[9];
    const double v2 = fma(vx, vx, fma(vy, vy, MUL(P, vz, vz)));
    const double rhoh = fma(P.Gq, p, rho);
    const double cs2 = MUL(P, MUL(P, P.Gamma, p), recip_nr(rhoh));
    const double c0 = fma(-v2, cs2, P.one);
    w[0] = vx; w[1] = vy; w[2] = vz; w[3] = p;
    w[4] = SUB(P, P.one, cs2);
    w[5] = MUL(P, cs2, SUB(P, P.one, v2));
    w[6] = c0;
    w[7] = recip_nr(c0);
  }
  // S_k v_d = rho h W^2 v_k v_d is symmetric in (k, d); every direction forms
  // it as S_min(k,d) v_max(k,d) (shared products, flux_xy).
  __device__ static void flux(int d, const double* q, const double* w, const DevParams& P, double* F) {
    const double v = sel3(d, w[0], w[1], w[2]), p = w[3], Sd = sel3(d, q[1], q[2], q[3]);
    F[0] = MUL(P, q[0], v);
#pragma unroll
    for (int k = 0; k < 3; ++k) F[1 + k] = fma(k < d ? q[1 + k] : Sd, k < d ? v : w[k], d == k ? p : P.zero);
    F[4] = fma(-q[0], v, Sd);
  }
  __device__ static void flux_xy(const double* q, const double* w, const double* Fz, const DevParams& P, double* Fx,
                                 double* Fy) {
    const double p = w[3], cxy = MUL(P, q[1], w[1]);
    Fx[0] = MUL(P, q[0], w[0]);
    Fx[1] = fma(q[1], w[0], p);
    Fx[2] = cxy;
    Fx[3] = Fz[1];
    Fx[4] = fma(-q[0], w[0], q[1]);
    Fy[0] = MUL(P, q[0], w[1]);
    Fy[1] = cxy;
    Fy[2] = fma(q[2], w[1], p);
    Fy[3] = Fz[2];
    Fy[4] = fma(-q[0], w[1], q[2]);
  }
  __device__ static double speed(int d, const double*, const double* w, const DevParams& P) {
    const double v = sel3(d, w[0], w[1], w[2]), omc = w[4];
    const double disc = MUL(P, w[5], fma(-MUL(P, v, v), omc, w[6]));
    return MUL(P, fma(fabs(v), omc, sqrt_pos(disc)), w[7]);
  }
  // The largest speed over the three directions.  For |v_d| < 1 (and cs^2 < 1) the speed
  // increases with |v_d|:
  // with a = 1 - cs^2, b = cs^2 (1 - v^2), c = 1 - v^2 cs^2 = a + b, d lambda / d|v_d| has the sign
  // of sqrt(c - v_d^2 a) - |v_d| sqrt(b), i.e. of c (1 - v_d^2) > 0.  So the maximum is the speed
  // of the direction of the largest |v_d|: one square root instead of three, and the value is
  // that direction's speed bit for bit (the max over separately rounded speeds can differ from
  // it only between directions whose |v_d| agree to a few units in the last place).
  __device__ static double max_speed(const double* w, const DevParams& P) {
    const double u = max_nn(max_nn(fabs(w[0]), fabs(w[1])), fabs(w[2]));
    const double omc = w[4];
    const double disc = MUL(P, w[5], fma(-MUL(P, u, u), omc, w[6]));
    return MUL(P, fma(u, omc, sqrt_pos(disc)), w[7]);
  }
  __device__ static void ncp(int, const double*, const double*, const DevParams&, double*) {}
  __device__ static void source(const double*, const double*, const DevParams&, double*) {}
};

// ---------------------------------------------------------------- wave system
// First-order reduction of the damped scalar wave equation with speed c(x):
//   d_t phi = Pi,  d_t Pi = c^2 div psi - gamma Pi,  d_t psi_i = d_i Pi
// as Eq. 1: F = 0; B_d has (row Pi, col psi_d) = -c^2 and (row psi_d, col Pi) = -1;
// S = (Pi, -gamma Pi, 0, 0, 0).  Material: c (M = 1).  lambda_d = c.
struct PdeWave {
  static constexpr int N = 5, M = 1, NW = 1, DIM = 3;
  static constexpr bool FLUX = false, NCP = true, SRC = true, SYM = false;
  __device__ static constexpr bool needs_grad(int d, int v) { return v == 1 || v == 2 + d; }
  __device__ static void prims(const double*, const DevParams&, double*) {}
  __device__ static void flux(int, const double*, const double*, const DevParams&, double*) {}
  __device__ static double speed(int, const double* q, const double*, const DevParams&) { return q[5]; }
  __device__ static void ncp(int d, const double* qb, const double* dq, const DevParams& P, double* D) {
    const double c2 = MUL(P, qb[5], qb[5]);
    D[0] = 0.0;
    D[1] = MUL(P, -c2, sel3(d, dq[2], dq[3], dq[4]));
    D[2] = d == 0 ? -dq[1] : 0.0;
    D[3] = d == 1 ? -dq[1] : 0.0;
    D[4] = d == 2 ? -dq[1] : 0.0;
  }
  __device__ static void source(const double* q, const double*, const DevParams& P, double* S) {
    S[0] = q[1];
    S[1] = MUL(P, -P.damp, q[1]);
    S[2] = 0.0; S[3] = 0.0; S[4] = 0.0;
  }
};

// ---------------------------------------------------------------- GW59 stand-in
// 11 first-order scalar waves (phi_a, Pi_a, psi_a,xyz) coupled to a lapse alpha
// and shift beta (59 unknowns):
//   d_t phi_a   = alpha Pi_a + beta^k psi_a,k
//   d_t Pi_a    = alpha d_k psi_a,k + beta^k d_k Pi_a + alpha sum_b C_ab phi_b Pi_b
//   d_t psi_a,i = alpha d_i Pi_a + Pi_a d_i alpha + beta^k d_k psi_a,i
//   d_t alpha   = -kappa alpha^2 sum_a Pi_a^2
//   d_t beta^i  = 3/4 sum_a psi_a,i Pi_a
// F = 0; every gradient term is part of B(Q).grad Q.  Layout: field a at 5a..5a+4,
// alpha at 55, beta at 56..58.  lambda_d = alpha + |beta^d|.
struct PdeGW59 {
  static constexpr int N = 59, M = 0, NW = 1, DIM = 3;
  static constexpr bool FLUX = false, NCP = true, SRC = true, SYM = false;
  __device__ static void prims(const double*, const DevParams&, double*) {}
  __device__ static double speed(int d, const double* q, const double*, const DevParams&) {
    return q[55] + fabs(sel3(d, q[56], q[57], q[58]));
  }
};

// The largest characteristic speed of a voxel over its dim directions (SRHD: the speed of the
// direction of the largest |v_d|, which is the largest).
template <class PDE>
__device__ __forceinline__ double max_speed_dirs(const double* u, const double* W, const DevParams& P, int dim) {
  if constexpr (std::is_same<PDE, PdeSRHD>::value) {
    return PdeSRHD::max_speed(W, P);
  } else {
    double l = fmax(PDE::speed(0, u, W, P), PDE::speed(1, u, W, P));
    if (dim == 3) l = fmax(l, PDE::speed(2, u, W, P));
    return l;
  }
}

}  // namespace dh
