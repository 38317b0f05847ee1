// Finite-difference Runge-Kutta stage: 4th-order centred first derivatives and
// 6th-difference Kreiss-Oliger dissipation (paper Sec. I and Sec. IV: FD4
// with KO dissipation; KO normalisation sigma/(64 dx) is the r = 3 form):
//   L(Q) = -sum_d B_d(Q) dQ/dx_d + S(Q) + sigma/(64 dx) sum_d delta6_d Q
//   dQ/dx  = [(Q_-2 - Q_+2) + 8 (Q_+1 - Q_-1)] / (12 dx)
//   delta6 = Q_-3 - 6 Q_-2 + 15 Q_-1 - 20 Q_0 + 15 Q_+1 - 6 Q_+2 + Q_+3
//   out = a q0 + b qs + g dt L ; acc += d dt L
// The three directional sixth differences are summed grouped by distance r
// (T_r = sum_d (Q_-r + Q_+r) - 6 Q_0, with 6 Q_0 formed by the same additions),
// which is exactly zero on constant data, so constant states stay bitwise
// constant.
//
// Kernel design: a CTA owns an 8x8x4 tile of one patch (one voxel per
// thread).  The variables are staged in groups of at most five into shared
// memory together with the tile's three-voxel face halos (edges and corners
// are never read by the axis-aligned stencils and are not loaded); halo
// voxels outside the patch come from the face neighbours.  Two staging
// variants exist (the autotuner picks one):
//   * plain loads: every thread copies voxels into a padded 14x14x10 box;
//   * TMA: one thread issues seven 5-D tensor copies per group (interior box
//     and six face slabs, from this patch or its neighbours) that complete on
//     an mbarrier; groups are double buffered, so the next field group of
//     GW59 streams in while the current one is computed.
// Every derivative is taken only for the variables that a column of B_d
// reads.  GW59 is processed field by field (lapse/shift first, then the 11
// scalar-wave fields), keeping per voxel only the coupling quantities (alpha,
// beta, grad alpha, phi_b Pi_b, source sums) in registers.
#include <cuda.h>

#include <cstring>
#include <type_traits>

#include "dh_internal.cuh"
#include "dh_pde.cuh"

namespace dh {

// Tensor-map descriptor as a kernel parameter (opaque 128 bytes).
struct alignas(64) TmaDesc {
  unsigned long long v[16];
};

constexpr int FD_MAX_LEVELS = 8;
enum { TMA_INT = 0, TMA_XS = 1, TMA_YS = 2, TMA_ZS = 3 };

struct FdArgs {
  TmaDesc maps[FD_MAX_LEVELS][4];  // per level: interior, x-slab, y-slab, z-slab boxes of qs
  const dh_patch* patches;
  const FdWork* work;
  const int2* lvl;                 // per patch: (level, index within the level)
  const double* qs;
  const double* q0;
  double* out;
  double* acc;
  const double* mat;
  const double* dt_dev;
  double a, b, g, d;
  double sigma;
  double* lam_out;
  unsigned long long* red;
  unsigned int* err;               // error flags (bit 0: a TMA wait gave up)
  int debug_no_issue;              // test hook: arm the barrier but issue no copy
  int64_t vs;
  DevParams P;
};

// Plain FP64 adds, subtractions and products.  (Issuing them as FMAs with
// run-time 1/-1/0 operands, as the FV stage does, measured 7% slower here.)
__device__ __forceinline__ double PADD(const DevParams&, double a, double b) { return a + b; }
__device__ __forceinline__ double PSUB(const DevParams&, double a, double b) { return a - b; }
__device__ __forceinline__ double PMUL(const DevParams&, double a, double b) { return a * b; }

constexpr int FTX = 8, FTY = 8, FTZ = 4, FH = 3;
constexpr int FBX = FTX + 2 * FH, FBY = FTY + 2 * FH, FBZ = FTZ + 2 * FH;
constexpr int FBOX = FBX * FBY * FBZ;                                               // 1960
constexpr int FNSLOT = FTX * FTY * FTZ + 2 * FH * (FTY * FTZ + FTX * FTZ + FTX * FTY);  // 1024
constexpr int FNT = FTX * FTY * FTZ;                                                // 256 threads
constexpr int GV = 5;                                                               // variables per group

// TMA staging buffer of one group (doubles): dense boxes, each 128-byte aligned.
//   interior [5][4][8][8], x-slabs [5][4][8][4] (x rounded out to 16-byte
//   alignment: the slab starts one voxel further out), y-slabs [5][4][3][8],
//   z-slabs [5][3][8][8].
constexpr int TI = 0;
constexpr int TXM = TI + GV * 4 * 8 * 8;   // 1280
constexpr int TXP = TXM + GV * 4 * 8 * 4;  // 1920
constexpr int TYM = TXP + GV * 4 * 8 * 4;  // 2560
constexpr int TYP = TYM + GV * 4 * 3 * 8;  // 3040
constexpr int TZM = TYP + GV * 4 * 3 * 8;  // 3520
constexpr int TZP = TZM + GV * 3 * 8 * 8;  // 4480
constexpr int TBUF = TZP + GV * 3 * 8 * 8;  // 5440 doubles = 43,520 bytes
constexpr unsigned TBYTES = TBUF * 8;
static_assert((TXM * 8) % 128 == 0 && (TXP * 8) % 128 == 0 && (TYM * 8) % 128 == 0 && (TYP * 8) % 128 == 0 &&
                  (TZM * 8) % 128 == 0 && (TZP * 8) % 128 == 0 && (TBUF * 8) % 128 == 0,
              "TMA destinations must be 128-byte aligned");

__device__ __forceinline__ int64_t fd_vox_index(const dh_patch* __restrict__ P, int k, int p, int x, int y, int z) {
  if (x < 0) { k = P[k].nbr[0]; x += p; }
  else if (x >= p) { k = P[k].nbr[1]; x -= p; }
  else if (y < 0) { k = P[k].nbr[2]; y += p; }
  else if (y >= p) { k = P[k].nbr[3]; y -= p; }
  else if (z < 0) { k = P[k].nbr[4]; z += p; }
  else if (z >= p) { k = P[k].nbr[5]; z -= p; }
  return P[k].offset + ((int64_t)z * p + y) * p + x;
}

// Slot s of the tile-plus-face-halo set -> tile-relative (x, y, z).
__device__ __forceinline__ void fd_slot(int s, int& x, int& y, int& z) {
  if (s < FNT) { x = s % FTX; y = (s / FTX) % FTY; z = s / (FTX * FTY); return; }
  int r = s - FNT;
  if (r < 2 * FH * FTY * FTZ) {  // x slabs
    const int side = r / (FH * FTY * FTZ), rr = r % (FH * FTY * FTZ);
    const int h = rr % FH;
    y = (rr / FH) % FTY; z = rr / (FH * FTY);
    x = side == 0 ? -FH + h : FTX + h;
    return;
  }
  r -= 2 * FH * FTY * FTZ;
  if (r < 2 * FH * FTX * FTZ) {  // y slabs
    const int side = r / (FH * FTX * FTZ), rr = r % (FH * FTX * FTZ);
    x = rr % FTX; const int h = (rr / FTX) % FH; z = rr / (FTX * FH);
    y = side == 0 ? -FH + h : FTY + h;
    return;
  }
  r -= 2 * FH * FTX * FTZ;  // z slabs
  const int side = r / (FH * FTX * FTY), rr = r % (FH * FTX * FTY);
  x = rr % FTX; y = (rr / FTX) % FTY; const int h = rr / (FTX * FTY);
  z = side == 0 ? -FH + h : FTZ + h;
}

__device__ __forceinline__ int fd_box(int x, int y, int z) { return ((z + FH) * FBY + (y + FH)) * FBX + (x + FH); }

// ------------------------------------------------------------- stencils
// 4th-order centred derivative (times 1/(12 dx)) from the values at -2, -1, +1, +2.
__device__ __forceinline__ double st_d1(const DevParams& P, double m2, double m1, double p1, double p2, double r12) {
  return PMUL(P, fma(8.0, PSUB(P, p1, m1), PSUB(P, m2, p2)), r12);
}
// Read access to one staged group: the padded box ...
struct BoxAcc {
  const double* box;
  int c;
  __device__ double val(int v) const { return box[v * FBOX + c]; }
  template <int D>
  __device__ double nb(int v, int o) const {
    constexpr int st = D == 0 ? 1 : (D == 1 ? FBX : FBX * FBY);
    return box[v * FBOX + c + o * st];
  }
};

// ... or the TMA staging buffer (dense interior box plus face slabs).
struct TmaAcc {
  const double* b;
  int lx, ly, lz;
  __device__ double val(int v) const { return b[TI + ((v * 4 + lz) * 8 + ly) * 8 + lx]; }
  template <int D>
  __device__ double nb(int v, int o) const {
    if (D == 0) {
      const int x = lx + o;
      if (x < 0) return b[TXM + ((v * 4 + lz) * 8 + ly) * 4 + (x + 4)];
      if (x >= 8) return b[TXP + ((v * 4 + lz) * 8 + ly) * 4 + (x - 8)];
      return b[TI + ((v * 4 + lz) * 8 + ly) * 8 + x];
    } else if (D == 1) {
      const int y = ly + o;
      if (y < 0) return b[TYM + ((v * 4 + lz) * 3 + (y + 3)) * 8 + lx];
      if (y >= 8) return b[TYP + ((v * 4 + lz) * 3 + (y - 8)) * 8 + lx];
      return b[TI + ((v * 4 + lz) * 8 + y) * 8 + lx];
    } else {
      const int z = lz + o;
      if (z < 0) return b[TZM + ((v * 3 + (z + 3)) * 8 + ly) * 8 + lx];
      if (z >= 4) return b[TZP + ((v * 3 + (z - 4)) * 8 + ly) * 8 + lx];
      return b[TI + ((v * 4 + z) * 8 + ly) * 8 + lx];
    }
  }
};

template <int D, class Acc>
__device__ __forceinline__ double acc_d1(const DevParams& P, const Acc& S, int v, double r12) {
  return st_d1(P, S.template nb<D>(v, -2), S.template nb<D>(v, -1), S.template nb<D>(v, 1), S.template nb<D>(v, 2), r12);
}
// Sum over the three directions of the sixth differences, grouped by distance:
//   sum_d delta6_d = T3 - 6 T2 + 15 T1,   T_r = S_r - 6c,
//   S_r = ((Q_-r + Q_+r)_x + (Q_-r + Q_+r)_y) + (Q_-r + Q_+r)_z,
// with 6c formed as ((2c + 2c) + 2c) -- the very additions S_r performs on
// constant data -- so every T_r is exactly 0 on constants (23 FP64 operations
// per variable instead of 27 for three bracketed directional differences).
template <class Acc>
__device__ __forceinline__ double acc_ko3(const DevParams& P, const Acc& S, int v) {
  const double c = S.val(v);
  const double two = PMUL(P, 2.0, c);
  const double six = PADD(P, PADD(P, two, two), two);
  double T[3];
#pragma unroll
  for (int r = 1; r <= 3; ++r) {
    const double sx = PADD(P, S.template nb<0>(v, -r), S.template nb<0>(v, r));
    const double sy = PADD(P, S.template nb<1>(v, -r), S.template nb<1>(v, r));
    const double sz = PADD(P, S.template nb<2>(v, -r), S.template nb<2>(v, r));
    T[r - 1] = PSUB(P, PADD(P, PADD(P, sx, sy), sz), six);
  }
  return fma(15.0, T[0], fma(-6.0, T[1], T[2]));
}

// ------------------------------------------------------------- staging
// Plain loads into the padded box (single buffer; the caller synchronises).
__device__ __forceinline__ void fd_stage_vars(const FdArgs& A, double* box, const FdWork& w, int p, int v0, int nv) {
  for (int s = threadIdx.x; s < FNSLOT; s += FNT) {
    int x, y, z;
    fd_slot(s, x, y, z);
    const int64_t e = fd_vox_index(A.patches, w.patch, p, w.x0 + x, w.y0 + y, w.z0 + z);
    const int c = fd_box(x, y, z);
    for (int v = 0; v < nv; ++v) box[v * FBOX + c] = __ldg(A.qs + (int64_t)(v0 + v) * A.vs + e);
  }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// One TMA tensor copy (5-D tile) into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load5(void* dst, const TmaDesc* map, int c0, int c1, int c2, int c3, int c4,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::
          "r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
      "r"(smem_u32(bar))
      : "memory");
}

// Bounded wait for phase `parity` of `bar`: gives up after ~2^27 SM clocks
// (about 65 ms) and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > (1ll << 27)) return false;
  }
}

// Issue the seven copies of group v0 (variables v0..v0+4) of tile w into buffer `buf`.
__device__ void tma_issue(const FdArgs& A, const FdWork& w, int p, double* buf, uint64_t* bar, int v0) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(TBYTES) : "memory");
  if (A.debug_no_issue) return;
  const int2 me = A.lvl[w.patch];
  const TmaDesc* M = A.maps[me.x];
  const dh_patch& pt = A.patches[w.patch];
  const int x0 = w.x0, y0 = w.y0, z0 = w.z0, kl = me.y;
  tma_load5(buf + TI, &M[TMA_INT], x0, y0, z0, kl, v0, bar);
  // x slabs (4 wide, 16-byte aligned start), from this patch or the x neighbours
  if (x0 > 0) tma_load5(buf + TXM, &M[TMA_XS], x0 - 4, y0, z0, kl, v0, bar);
  else tma_load5(buf + TXM, &M[TMA_XS], p - 4, y0, z0, A.lvl[pt.nbr[0]].y, v0, bar);
  if (x0 + 8 < p) tma_load5(buf + TXP, &M[TMA_XS], x0 + 8, y0, z0, kl, v0, bar);
  else tma_load5(buf + TXP, &M[TMA_XS], 0, y0, z0, A.lvl[pt.nbr[1]].y, v0, bar);
  if (y0 > 0) tma_load5(buf + TYM, &M[TMA_YS], x0, y0 - 3, z0, kl, v0, bar);
  else tma_load5(buf + TYM, &M[TMA_YS], x0, p - 3, z0, A.lvl[pt.nbr[2]].y, v0, bar);
  if (y0 + 8 < p) tma_load5(buf + TYP, &M[TMA_YS], x0, y0 + 8, z0, kl, v0, bar);
  else tma_load5(buf + TYP, &M[TMA_YS], x0, 0, z0, A.lvl[pt.nbr[3]].y, v0, bar);
  if (z0 > 0) tma_load5(buf + TZM, &M[TMA_ZS], x0, y0, z0 - 3, kl, v0, bar);
  else tma_load5(buf + TZM, &M[TMA_ZS], x0, y0, p - 3, A.lvl[pt.nbr[4]].y, v0, bar);
  if (z0 + 4 < p) tma_load5(buf + TZP, &M[TMA_ZS], x0, y0, z0 + 4, kl, v0, bar);
  else tma_load5(buf + TZP, &M[TMA_ZS], x0, y0, 0, A.lvl[pt.nbr[5]].y, v0, bar);
}

// CTA-uniform wait; on a timeout every thread records it, waits once more
// (bounded) for copies still in flight, and the caller abandons the tile.
__device__ bool tma_wait_all(const FdArgs& A, uint64_t* bar, uint32_t parity) {
  const bool ok = mbar_wait(bar, parity);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) atomicOr(A.err, 1u);
    mbar_wait(bar, parity);
    return false;
  }
  return true;
}

// out / acc update of one variable; returns the new value of the result.
__device__ __forceinline__ double fd_combine(const FdArgs& A, int64_t ev, double qsv, double L, double gdt,
                                             double ddt) {
  double res = 0.0;
  if (A.out) {
    double base = A.b == 1.0 ? qsv : PMUL(A.P, A.b, qsv);
    if (A.q0) base = fma(A.a, __ldg(A.q0 + ev), base);
    res = fma(gdt, L, base);
  }
  if (A.acc) {
    const double r = fma(ddt, L, A.acc[ev]);
    A.acc[ev] = r;
    if (!A.out) res = r;
  }
  if (A.out) A.out[ev] = res;
  return res;
}

// ------------------------------------------------------------- generic (N <= 5)
template <class PDE, class Acc>
__device__ void fd_voxel_generic(const FdArgs& A, const Acc& S, int64_t e, double dx, double& lam_thread) {
  constexpr int N = PDE::N, NV = PDE::N + PDE::M;
  const double r12 = 1.0 / (12.0 * dx);
  const double ko = A.sigma / (64.0 * dx);
  const double dt = *A.dt_dev;
  const double gdt = A.g * dt, ddt = A.d * dt;
  double q[NV], L[N], W[1];
#pragma unroll
  for (int v = 0; v < N; ++v) q[v] = S.val(v);
#pragma unroll
  for (int v = 0; v < PDE::M; ++v) q[N + v] = __ldg(A.mat + (int64_t)v * A.vs + e);
  if (PDE::SRC) PDE::source(q, W, A.P, L);
  else {
#pragma unroll
    for (int v = 0; v < N; ++v) L[v] = 0.0;
  }
  double dq[N], D[N];
#pragma unroll
  for (int v = 0; v < N; ++v) dq[v] = PDE::needs_grad(0, v) ? acc_d1<0>(A.P, S, v, r12) : 0.0;
  PDE::ncp(0, q, dq, A.P, D);
#pragma unroll
  for (int v = 0; v < N; ++v) L[v] = PSUB(A.P, L[v], D[v]);
#pragma unroll
  for (int v = 0; v < N; ++v) dq[v] = PDE::needs_grad(1, v) ? acc_d1<1>(A.P, S, v, r12) : 0.0;
  PDE::ncp(1, q, dq, A.P, D);
#pragma unroll
  for (int v = 0; v < N; ++v) L[v] = PSUB(A.P, L[v], D[v]);
#pragma unroll
  for (int v = 0; v < N; ++v) dq[v] = PDE::needs_grad(2, v) ? acc_d1<2>(A.P, S, v, r12) : 0.0;
  PDE::ncp(2, q, dq, A.P, D);
#pragma unroll
  for (int v = 0; v < N; ++v) L[v] = PSUB(A.P, L[v], D[v]);
  double res[NV];
#pragma unroll
  for (int v = 0; v < N; ++v) {
    const double Lv = fma(ko, acc_ko3(A.P, S, v), L[v]);
    res[v] = fd_combine(A, (int64_t)v * A.vs + e, q[v], Lv, gdt, ddt);
  }
  if (A.lam_out) {
#pragma unroll
    for (int v = N; v < NV; ++v) res[v] = q[v];
    double l = fmax(fmax(PDE::speed(0, res, W, A.P), PDE::speed(1, res, W, A.P)), PDE::speed(2, res, W, A.P));
    lam_thread = fmax(lam_thread, l);
  }
}

// The wave system written out (same operator as the generic path with
// PdeWave's B and S): the 1/(12 dx) of the derivatives is folded into the
// FMAs that consume them.
//   L_phi   = Pi + KO,   L_Pi = c^2 r12 (Dx psi_x + Dy psi_y + Dz psi_z) - damp Pi + KO,
//   L_psi_d = r12 Dd Pi + KO,   Dd q = (q_-2 - q_+2) + 8 (q_+1 - q_-1) along d.
template <int D, class Acc>
__device__ __forceinline__ double acc_raw(const DevParams& P, const Acc& S, int v) {
  return fma(8.0, PSUB(P, S.template nb<D>(v, 1), S.template nb<D>(v, -1)),
             PSUB(P, S.template nb<D>(v, -2), S.template nb<D>(v, 2)));
}

template <class Acc>
__device__ void fd_voxel_wave(const FdArgs& A, const Acc& S, int64_t e, double dx, double& lam_thread) {
  const DevParams& P = A.P;
  const double r12 = 1.0 / (12.0 * dx);
  const double ko = A.sigma / (64.0 * dx);
  const double dt = *A.dt_dev;
  const double gdt = A.g * dt, ddt = A.d * dt;
  const double q[5] = {S.val(0), S.val(1), S.val(2), S.val(3), S.val(4)};
  const double c = __ldg(A.mat + e);
  const double div = PADD(P, PADD(P, acc_raw<0>(P, S, 2), acc_raw<1>(P, S, 3)), acc_raw<2>(P, S, 4));
  double L[5];
  L[0] = fma(ko, acc_ko3(P, S, 0), q[1]);
  L[1] = fma(ko, acc_ko3(P, S, 1), fma(PMUL(P, PMUL(P, c, c), r12), div, PMUL(P, -P.damp, q[1])));
  L[2] = fma(ko, acc_ko3(P, S, 2), PMUL(P, r12, acc_raw<0>(P, S, 1)));
  L[3] = fma(ko, acc_ko3(P, S, 3), PMUL(P, r12, acc_raw<1>(P, S, 1)));
  L[4] = fma(ko, acc_ko3(P, S, 4), PMUL(P, r12, acc_raw<2>(P, S, 1)));
#pragma unroll
  for (int v = 0; v < 5; ++v) fd_combine(A, (int64_t)v * A.vs + e, q[v], L[v], gdt, ddt);
  if (A.lam_out) lam_thread = fmax(lam_thread, c);
}

template <class PDE, bool TMA>
__device__ void fd_tile_generic(const FdArgs& A, const FdWork& w, double* smem, uint64_t* bars, double& lam_thread) {
  static_assert(PDE::N <= GV, "generic FD path stages one group of at most five variables");
  const dh_patch& pt = A.patches[w.patch];
  const int p = pt.p;
  const int t = threadIdx.x;
  const int lx = t % FTX, ly = (t / FTX) % FTY, lz = t / (FTX * FTY);
  const int64_t e = pt.offset + ((int64_t)(w.z0 + lz) * p + (w.y0 + ly)) * p + (w.x0 + lx);
  if (TMA) {
    if (t == 0) tma_issue(A, w, p, smem, &bars[0], 0);
    if (!tma_wait_all(A, &bars[0], 0)) return;
    if constexpr (std::is_same<PDE, PdeWave>::value) fd_voxel_wave(A, TmaAcc{smem, lx, ly, lz}, e, pt.dx, lam_thread);
    else fd_voxel_generic<PDE>(A, TmaAcc{smem, lx, ly, lz}, e, pt.dx, lam_thread);
  } else {
    fd_stage_vars(A, smem, w, p, 0, PDE::N);
    __syncthreads();
    if constexpr (std::is_same<PDE, PdeWave>::value) fd_voxel_wave(A, BoxAcc{smem, fd_box(lx, ly, lz)}, e, pt.dx, lam_thread);
    else fd_voxel_generic<PDE>(A, BoxAcc{smem, fd_box(lx, ly, lz)}, e, pt.dx, lam_thread);
  }
}

// ------------------------------------------------------------- GW59
struct Gw59State {
  double al, bx, by, bz, dal0, dal1, dal2, ko_ab[4], u[11], sumPi2, bs0, bs1, bs2;
  double alr, bxr, byr, bzr;  // alpha and beta times 1/(12 dx): the field derivatives stay unscaled
};

template <class Acc>
__device__ __forceinline__ void gw59_lapse_shift(const FdArgs& A, const Acc& S, int64_t e, double r12, double ko,
                                                 Gw59State& G) {
  const DevParams& P = A.P;
  G.al = S.val(0); G.bx = S.val(1); G.by = S.val(2); G.bz = S.val(3);
  G.alr = PMUL(P, G.al, r12); G.bxr = PMUL(P, G.bx, r12); G.byr = PMUL(P, G.by, r12); G.bzr = PMUL(P, G.bz, r12);
  G.dal0 = acc_d1<0>(P, S, 0, r12);
  G.dal1 = acc_d1<1>(P, S, 0, r12);
  G.dal2 = acc_d1<2>(P, S, 0, r12);
#pragma unroll
  for (int v = 0; v < 4; ++v) G.ko_ab[v] = PMUL(P, ko, acc_ko3(P, S, v));
  // phi_b Pi_b at this voxel for the source coupling
#pragma unroll
  for (int bb = 0; bb < 11; ++bb)
    G.u[bb] = PMUL(P, __ldg(A.qs + (int64_t)(5 * bb) * A.vs + e), __ldg(A.qs + (int64_t)(5 * bb + 1) * A.vs + e));
  G.sumPi2 = 0.0; G.bs0 = 0.0; G.bs1 = 0.0; G.bs2 = 0.0;
}

template <class Acc>
__device__ __forceinline__ void gw59_field(const FdArgs& A, const Acc& S, int a, int64_t e, double r12, double ko,
                                           double gdt, double ddt, Gw59State& G) {
  const DevParams& P = A.P;
  const int64_t vs = A.vs;
  const double al = G.al, bx = G.bx, by = G.by, bz = G.bz;
  const double phi = S.val(0), Pi = S.val(1), px = S.val(2), py = S.val(3), pz = S.val(4);
  // unscaled derivatives (the 1/(12 dx) sits in alr, bxr, byr, bzr)
  const double dPi0 = acc_raw<0>(P, S, 1), dPi1 = acc_raw<1>(P, S, 1), dPi2 = acc_raw<2>(P, S, 1);
  // coupling sum_b C_ab phi_b Pi_b
  double cs = PMUL(P, P.C[11 * a], G.u[0]);
#pragma unroll
  for (int bb = 1; bb < 11; ++bb) cs = fma(P.C[11 * a + bb], G.u[bb], cs);
  // phi: alpha Pi + beta . psi
  const double Lphi = fma(al, Pi, fma(bx, px, fma(by, py, PMUL(P, bz, pz))));
  // Pi: alpha div psi + beta . grad Pi + alpha cs
  const double dpx0 = acc_raw<0>(P, S, 2), dpx1 = acc_raw<1>(P, S, 2), dpx2 = acc_raw<2>(P, S, 2);
  const double dpy0 = acc_raw<0>(P, S, 3), dpy1 = acc_raw<1>(P, S, 3), dpy2 = acc_raw<2>(P, S, 3);
  const double dpz0 = acc_raw<0>(P, S, 4), dpz1 = acc_raw<1>(P, S, 4), dpz2 = acc_raw<2>(P, S, 4);
  const double alr = G.alr, bxr = G.bxr, byr = G.byr, bzr = G.bzr;
  const double LPi = fma(alr, PADD(P, PADD(P, dpx0, dpy1), dpz2), fma(bxr, dPi0, fma(byr, dPi1, fma(bzr, dPi2, PMUL(P, al, cs)))));
  // psi_i: alpha d_i Pi + Pi d_i alpha + beta . grad psi_i
  const double Lpx = fma(alr, dPi0, fma(Pi, G.dal0, fma(bxr, dpx0, fma(byr, dpx1, PMUL(P, bzr, dpx2)))));
  const double Lpy = fma(alr, dPi1, fma(Pi, G.dal1, fma(bxr, dpy0, fma(byr, dpy1, PMUL(P, bzr, dpy2)))));
  const double Lpz = fma(alr, dPi2, fma(Pi, G.dal2, fma(bxr, dpz0, fma(byr, dpz1, PMUL(P, bzr, dpz2)))));
  G.sumPi2 = fma(Pi, Pi, G.sumPi2);
  G.bs0 = fma(px, Pi, G.bs0);
  G.bs1 = fma(py, Pi, G.bs1);
  G.bs2 = fma(pz, Pi, G.bs2);
  const int64_t eb = (int64_t)(5 * a) * vs + e;
  fd_combine(A, eb, phi, fma(ko, acc_ko3(P, S, 0), Lphi), gdt, ddt);
  fd_combine(A, eb + vs, Pi, fma(ko, acc_ko3(P, S, 1), LPi), gdt, ddt);
  fd_combine(A, eb + 2 * vs, px, fma(ko, acc_ko3(P, S, 2), Lpx), gdt, ddt);
  fd_combine(A, eb + 3 * vs, py, fma(ko, acc_ko3(P, S, 3), Lpy), gdt, ddt);
  fd_combine(A, eb + 4 * vs, pz, fma(ko, acc_ko3(P, S, 4), Lpz), gdt, ddt);
}

__device__ __forceinline__ void gw59_finish(const FdArgs& A, int64_t e, double gdt, double ddt, const Gw59State& G,
                                            double& lam_thread) {
  const DevParams& P = A.P;
  const int64_t vs = A.vs;
  const double Lal = fma(PMUL(P, -P.kappa, PMUL(P, G.al, G.al)), G.sumPi2, G.ko_ab[0]);
  const double ra = fd_combine(A, 55 * vs + e, G.al, Lal, gdt, ddt);
  const double r0 = fd_combine(A, 56 * vs + e, G.bx, fma(0.75, G.bs0, G.ko_ab[1]), gdt, ddt);
  const double r1 = fd_combine(A, 57 * vs + e, G.by, fma(0.75, G.bs1, G.ko_ab[2]), gdt, ddt);
  const double r2 = fd_combine(A, 58 * vs + e, G.bz, fma(0.75, G.bs2, G.ko_ab[3]), gdt, ddt);
  if (A.lam_out) lam_thread = fmax(lam_thread, PADD(P, ra, fmax(fmax(fabs(r0), fabs(r1)), fabs(r2))));
}

template <bool TMA>
__device__ void fd_tile_gw59(const FdArgs& A, const FdWork& w, double* smem, uint64_t* bars, double& lam_thread) {
  const dh_patch& pt = A.patches[w.patch];
  const int p = pt.p;
  const int t = threadIdx.x;
  const int lx = t % FTX, ly = (t / FTX) % FTY, lz = t / (FTX * FTY);
  const int64_t e = pt.offset + ((int64_t)(w.z0 + lz) * p + (w.y0 + ly)) * p + (w.x0 + lx);
  const double dx = pt.dx;
  const double r12 = 1.0 / (12.0 * dx);
  const double ko = A.sigma / (64.0 * dx);
  const double dt = *A.dt_dev;
  const double gdt = A.g * dt, ddt = A.d * dt;
  Gw59State G;
  if (TMA) {
    // groups: 0 = lapse/shift (variables 55..59, 59 out of range reads as 0), 1..11 = fields 0..10
    if (t == 0) tma_issue(A, w, p, smem, &bars[0], 55);
#pragma unroll 1
    for (int gi = 0; gi < 12; ++gi) {
      const int b = gi & 1;
      if (gi + 1 < 12 && t == 0) tma_issue(A, w, p, smem + (b ^ 1) * TBUF, &bars[b ^ 1], 5 * gi);
      if (!tma_wait_all(A, &bars[b], (gi >> 1) & 1)) {
        // abandon the tile; the copy issued into the other buffer may still be in flight
        if (gi + 1 < 12) mbar_wait(&bars[b ^ 1], ((gi + 1) >> 1) & 1);
        return;
      }
      const TmaAcc S{smem + b * TBUF, lx, ly, lz};
      if (gi == 0) gw59_lapse_shift(A, S, e, r12, ko, G);
      else gw59_field(A, S, gi - 1, e, r12, ko, gdt, ddt, G);
      __syncthreads();  // buffer b is free for the copy issued in the next iteration
    }
  } else {
    const BoxAcc S{smem, fd_box(lx, ly, lz)};
    fd_stage_vars(A, smem, w, p, 55, 4);
    __syncthreads();
    gw59_lapse_shift(A, S, e, r12, ko, G);
#pragma unroll 1
    for (int a = 0; a < 11; ++a) {
      __syncthreads();  // previous group's box reads are done
      fd_stage_vars(A, smem, w, p, 5 * a, 5);
      __syncthreads();
      gw59_field(A, S, a, e, r12, ko, gdt, ddt, G);
    }
  }
  gw59_finish(A, e, gdt, ddt, G, lam_thread);
}

__device__ __forceinline__ double fd_warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ void fd_publish_lambda(double lam, double* lam_out, unsigned long long* red) {
  __shared__ double wmax[FNT / 32];
  __shared__ bool last;
  lam = fd_warp_max(lam);
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = lam;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < FNT / 32; ++i) m = fmax(m, wmax[i]);
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

// Kernel variants (chosen per plan by the autotuner):
//   VAR bit 1: at most 128 registers so that two CTAs fit on an SM;
//   VAR bit 2: TMA staging (double-buffered groups) instead of plain loads;
//   VAR bit 3 / bit 4: register caps for three / four CTAs per SM (80 / 64
//              registers; with TMA staging the single group buffer of the
//              generic path, 43.6 KB, lets that many CTAs share an SM).
template <int VAR>
constexpr int fd_min_blocks() {
  return (VAR & 16) ? 4 : (VAR & 8) ? 3 : (VAR & 2) ? 2 : 1;
}

template <class PDE, int VAR>
__global__ void __launch_bounds__(FNT, fd_min_blocks<VAR>()) k_fd_stage(const __grid_constant__ FdArgs A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[2];
  constexpr bool TMA = (VAR & 4) != 0;
  // TMA destinations start on a 128-byte boundary (the launch adds 128 bytes of slack)
  double* smem = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
  if (TMA) {
    if (threadIdx.x == 0) {
      mbar_init(&bars[0], 1);
      mbar_init(&bars[1], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
  }
  const FdWork w = A.work[blockIdx.x];
  double lam = 0.0;
  if constexpr (PDE::N == 59) fd_tile_gw59<TMA>(A, w, smem, bars, lam);
  else fd_tile_generic<PDE, TMA>(A, w, smem, bars, lam);
  if (A.lam_out) fd_publish_lambda(lam, A.lam_out, A.red);
}

template <class PDE, int VAR>
static dh_status fd_launch_var(dh_plan* plan, const FdArgs& A, cudaStream_t stream) {
  constexpr bool TMA = (VAR & 4) != 0;
  constexpr int NB = PDE::N == 59 ? 5 : PDE::N;
  // TMA: GW59 double-buffers its field groups, the generic path stages one group
  const size_t smem = (TMA ? (PDE::N == 59 ? 2 : 1) * (size_t)TBYTES : sizeof(double) * NB * FBOX) + 128;
  static int configured_device = -1;
  if (configured_device != plan->device) {
    cudaError_t e = cudaFuncSetAttribute(k_fd_stage<PDE, VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(k_fd_stage)");
    configured_device = plan->device;
  }
  k_fd_stage<PDE, VAR><<<plan->n_fdwork, FNT, smem, stream>>>(A);
  return cuda_error(cudaGetLastError(), "k_fd_stage launch");
}

template <class PDE>
static dh_status fd_launch(dh_plan* plan, const FdArgs& A, cudaStream_t stream) {
  if constexpr (PDE::N != 59) {
    if (plan->fd_var == 12) return fd_launch_var<PDE, 12>(plan, A, stream);
    if (plan->fd_var == 20) return fd_launch_var<PDE, 20>(plan, A, stream);
  }
  switch (plan->fd_var & 6) {
    case 0: return fd_launch_var<PDE, 0>(plan, A, stream);
    case 2: return fd_launch_var<PDE, 2>(plan, A, stream);
    case 4: return fd_launch_var<PDE, 4>(plan, A, stream);
    default: return fd_launch_var<PDE, 6>(plan, A, stream);
  }
}

// ------------------------------------------------------------- tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// 5-D maps over qs for every level: (x, y, z, patch, variable), four box shapes.
static dh_status encode_maps(dh_plan* plan, const double* qs, FdArgs& A) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) { set_error("patch_update_fd_ko: cuTensorMapEncodeTiled is unavailable"); return DH_EUNSUPPORTED; }
  static const cuuint32_t boxes[4][5] = {{8, 8, 4, 1, GV}, {4, 8, 4, 1, GV}, {8, 3, 4, 1, GV}, {8, 8, 3, 1, GV}};
  for (int l = 0; l < plan->n_lvl; ++l) {
    const uint64_t p = (uint64_t)plan->lvl_p[l];
    const cuuint64_t dims[5] = {p, p, p, (cuuint64_t)plan->lvl_K[l], (cuuint64_t)plan->nq};
    const cuuint64_t strides[4] = {p * 8, p * p * 8, p * p * p * 8, (cuuint64_t)plan->var_stride * 8};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    void* base = (void*)(qs + plan->lvl_off[l]);
    for (int bt = 0; bt < 4; ++bt) {
      CUtensorMap m;
      CUresult r = fn(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, base, dims, strides, boxes[bt], estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) {
        set_error("patch_update_fd_ko: cuTensorMapEncodeTiled failed (%d) for level %d", (int)r, l);
        return DH_ECUDA;
      }
      static_assert(sizeof(TmaDesc) == sizeof(CUtensorMap), "tensor map size");
      std::memcpy(&A.maps[l][bt], &m, sizeof(CUtensorMap));
    }
  }
  return DH_OK;
}

dh_status launch_fd_stage(dh_plan* plan, const double* qs, const double* q0, double* out, double* acc,
                          const double* mat, const double* dt_dev, double a, double b, double g, double d,
                          double sigma, double* lam_out, cudaStream_t stream) {
  FdArgs A;
  std::memset(&A.maps, 0, sizeof(A.maps));
  A.patches = plan->d_patches;
  A.work = plan->d_fdwork;
  A.lvl = plan->d_lvl;
  A.qs = qs; A.q0 = q0; A.out = out; A.acc = acc; A.mat = mat; A.dt_dev = dt_dev;
  A.a = a; A.b = b; A.g = g; A.d = d; A.sigma = sigma;
  A.lam_out = lam_out;
  A.red = plan->d_red;
  A.err = reinterpret_cast<unsigned int*>(plan->d_red + 2);
  A.debug_no_issue = plan->debug_flags & 1;
  A.vs = plan->var_stride;
  A.P = plan->params;
  if (plan->fd_var & 4) {
    if (!plan->tma_ok) { set_error("patch_update_fd_ko: the TMA variant needs contiguous levels (see dh_plan_create)"); return DH_EUNSUPPORTED; }
    dh_status st = encode_maps(plan, qs, A);
    if (st != DH_OK) return st;
  }
  switch (plan->pde) {
    case DH_PDE_ADV_NCP: return fd_launch<PdeAdvNcp>(plan, A, stream);
    case DH_PDE_WAVE3D: return fd_launch<PdeWave>(plan, A, stream);
    case DH_PDE_GW59: return fd_launch<PdeGW59>(plan, A, stream);
    default:
      set_error("patch_update_fd_ko: PDE %d not supported by the FD stage", plan->pde);
      return DH_EUNSUPPORTED;
  }
}

}  // namespace dh
