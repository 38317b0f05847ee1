// The finite-volume stage kernel: templates shared by the per-PDE translation units
// (dh_fv_<pde>.cu instantiate them; dh_fv.cu dispatches on the plan's PDE).
//
// Finite-volume Runge-Kutta stage over all patches in one launch.
//
// Scheme (paper Sec. II-A Eq. 3; Rusanov flux and midpoint path-conservative
// product as the readings of the unspecified face flux):
//   L(Q)_i = -(1/dx) sum_d [F^_{i+1/2} - F^_{i-1/2} + (D_{i+1/2} + D_{i-1/2})/2] + S(Q_i)
//   out = a q0 + b qs + g dt L ; acc += d dt L
// or, for the three stages of SSP-RK3 (Shu-Osher) written in its Butcher form
// u1 = u0 + dt L0, u2 = u0 + dt/4 (L0 + L1), u3 = u0 + dt/6 (L0 + L1) + 2 dt/3 L2
// (the same scheme; "stage-sum form"), with acc holding the raw face-flux sum R
// of the earlier stages (R = s0, then s0 + s1; L = -s/(2 dx) for the systems
// without a source term):
//   stage 1: out = qs + g dt L,             R  = s
//   stage 2: out = q0 + g dt (-(R + s)/(2 dx)), R = R + s      (g = 1/4)
//   stage 3: out = q0 + d dt (-R/(2 dx)) + g dt L              (d = 1/6, g = 2/3)
// i.e. one or two FP64 operations per quantity and stage instead of up to three.
//
// Kernel design (GB300: the FP64 pipe, ~2 FMA/clk/SM, is the bottleneck, so
// every FP64 operation is done once and only by full warps):
//   * A CTA owns a (TX x TY) column of one patch -- 16x16 or 32x8 -- (or four 8x8
//     columns of up to four patches) and marches it through the z-planes of the
//     patch; in the persistent form a CTA takes tile after tile from a queue.
//   * Per voxel, the derived quantities W (one reciprocal, one square root for
//     Euler), the three directional fluxes F_d and speeds lambda_d are computed
//     exactly once.  x/y neighbours exchange them through shared memory; the
//     z neighbour is the same thread one plane later (registers).
//   * The ring of halo voxels around the column (neighbour patches or the
//     rest of the same patch) is computed by the first 2(TX+TY)G threads;
//     ring voxels only need the one direction that crosses into the column.
//   * Every face flux is computed once: each voxel thread computes its -x and
//     -y faces, the +x/+y boundary faces are computed by ring threads; the
//     factor 1/2 of the Rusanov average is folded into the final -1/(2dx).
//   * The maximum characteristic speed of the result is reduced with warp
//     shuffles, then one atomicMax per CTA on the bit pattern (valid for
//     non-negative doubles), and the last CTA publishes it (no spin waits).
#pragma once

#include <algorithm>
#include <type_traits>

#include "dh_internal.cuh"
#include "dh_pde.cuh"
#include "dh_tma.cuh"

namespace dh {

struct FvArgs {
  const dh_patch* patches;
  const Work* work;
  const double* qs;
  const double* q0;
  double* out;
  double* acc;
  const double* mat;
  const double* dt_dev;
  double a, b, g, d;
  double* lam_out;
  // with lam_out: the last CTA also writes the next time step's dt = cfl dx_dim / lambda
  // (the CFL rule, same expression as dh_cfl_dt), NULL otherwise
  double* dt_next;
  double cfl, dx_dim;
  unsigned long long* red;
  unsigned int* queue;  // persistent launch: tile queue head and exit count (two words), else NULL
  int n_work;           // tiles in the work list
  const int* oct;  // octant bits per patch on coupled plans, else NULL
  const double* w_in;  // derived quantities W of qs (NW-variable arena) when the stage reads them
  double* w_out;       // W of the result, written by a stage that computes it for lambda
  int form;        // 0: the general stage above; 1-3: SSP-RK3 stage 1-3 in stage-sum form (acc = R)
  int64_t vs;      // var stride
  // TMA staging (kernel variant bit 6): level of every patch (level, index within it), the
  // error word (bit 0: a bounded wait for a copy gave up) and a test hook (no copy issued)
  const int2* lvl;
  unsigned int* err;
  int debug_no_issue;
  DevParams P;
};

// The stage's arithmetic constants as register values.  On GB300 an FP64 FMA whose operands
// are all registers issues at 2.0 per clock per SM, while DADD, DMUL and any FP64 instruction
// with a constant-bank operand (a kernel parameter or a literal) issue at 1.68 (measured), so
// the constants that the adds, subtractions and products written as FMAs use (1, -1, 0, 1/2)
// and the gas constants are copied into registers once per thread: a shuffle hides their
// values from the compiler, which would otherwise fold them back into constant-bank operands.
__device__ __forceinline__ double opaque_reg(double v) { return __shfl_sync(0xffffffffu, v, 0); }
__device__ __forceinline__ FvArgs with_reg_params(const FvArgs& A) {
  FvArgs L = A;
  L.P.one = opaque_reg(A.P.one);
  L.P.mone = opaque_reg(A.P.mone);
  L.P.zero = opaque_reg(A.P.zero);
  L.P.half = opaque_reg(A.P.half);
  L.P.gamma = opaque_reg(A.P.gamma);
  L.P.gm1 = opaque_reg(A.P.gm1);
  L.P.Gamma = opaque_reg(A.P.Gamma);
  L.P.Gq = opaque_reg(A.P.Gq);
  return L;
}

// Tensor maps of the TMA-staged variant, per arena level of back-to-back patches: boxes of
// one z-plane of a 16x16 or 32x8 column and of its four ring strips (x strips two voxels
// wide, so that every copy starts on a 16-byte boundary).  Other variants get an empty struct.
enum { FVB_INT16 = 0, FVB_XS16 = 1, FVB_YS16 = 2, FVB_INT32 = 3, FVB_XS8 = 4, FVB_YS32 = 5, FVB_N = 6 };
constexpr int FV_TMA_LEVELS = 8;
template <bool TMA>
struct FvMaps {
  int unused;
};
template <>
struct FvMaps<true> {
  fvtma::Map m[FV_TMA_LEVELS][FVB_N];
};

// Arena index of voxel (x, y, z) of patch k; at most one coordinate may lie
// outside [0, p): it is then taken from the face neighbour (periodic wrap is
// encoded in the neighbour table).  On coupled plans (oct != NULL) a
// neighbour one level coarser supplies the coarse voxel that contains the
// position (piecewise-constant prolongation): along the face axis the coarse
// index is p + floor(c/2) below the patch and floor((c - p)/2) above it,
// across it the patch's octant half plus floor(c/2).
static __device__ __forceinline__ int64_t vox_index(const dh_patch* __restrict__ P, const int* __restrict__ oct, int k,
                                             int p, int x, int y, int z) {
  int f = -1;
  if (x < 0) f = 0;
  else if (x >= p) f = 1;
  else if (y < 0) f = 2;
  else if (y >= p) f = 3;
  else if (z < 0) f = 4;
  else if (z >= p) f = 5;
  if (f < 0) return P[k].offset + ((int64_t)z * p + y) * p + x;
  const int n = P[k].nbr[f];
  if (oct && P[n].level < P[k].level) {
    const int o = oct[k], h = p >> 1, a = f >> 1;
    int c[3] = {x, y, z};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (b == a) c[b] = c[b] < 0 ? p + (c[b] >> 1) : (c[b] - p) >> 1;
      else c[b] = ((o >> b) & 1) * h + (c[b] >> 1);
    }
    return P[n].offset + ((int64_t)c[2] * p + c[1]) * p + c[0];
  }
  if (f == 0) x += p;
  else if (f == 1) x -= p;
  else if (f == 2) y += p;
  else if (f == 3) y -= p;
  else if (f == 4) z += p;
  else z -= p;
  return P[n].offset + ((int64_t)z * p + y) * p + x;
}

static __device__ __forceinline__ void prefetch_l2(const double* a) { asm volatile("prefetch.global.L2 [%0];" ::"l"(a)); }

template <class PDE>
__device__ __forceinline__ void load_q(const FvArgs& A, int64_t e, double* q) {
#pragma unroll
  for (int v = 0; v < PDE::N; ++v) q[v] = __ldg(A.qs + v * A.vs + e);
#pragma unroll
  for (int v = 0; v < PDE::M; ++v) q[PDE::N + v] = __ldg(A.mat + v * A.vs + e);
}

// Derived quantities W of the voxel at arena index e: read from the W arena the
// previous step's last stage wrote (WM bit 0) or computed from q.  Both give
// the same bits: the stored W was computed by PDE::prims from the same values.
template <class PDE, int WM>
__device__ __forceinline__ void derive(const FvArgs& A, int64_t e, const double* q, double* W) {
  if (WM & 1) {
#pragma unroll
    for (int i = 0; i < PDE::NW; ++i) W[i] = __ldg(A.w_in + i * A.vs + e);
  } else {
    PDE::prims(q, A.P, W);
  }
}

// F_x and F_y of one voxel (F_z already formed in 3D): systems with a symmetric
// flux share its off-diagonal products between directions.
template <class PDE>
__device__ __forceinline__ void flux_xy(const double* q, const double* W, const double* Fz, const DevParams& P,
                                        double* Fx, double* Fy) {
  if constexpr (PDE::SYM) {
    PDE::flux_xy(q, W, Fz, P, Fx, Fy);
  } else {
    PDE::flux(0, q, W, P, Fx);
    PDE::flux(1, q, W, P, Fy);
  }
}

// Systems whose derived quantities are many (SRHD: eight) form all three
// speeds of a voxel where its z flux is formed, so that only the two in-plane
// speeds, not the speed factors, stay live across the plane's barrier.
template <class PDE>
constexpr bool speeds_with_z() { return PDE::NW >= 8; }

template <class PDE, int TX, int TY, int G, bool EARLY, int WM, bool TMA = false>
struct FvTile {
  static constexpr int N = PDE::N, NV = PDE::N + PDE::M, NW = PDE::NW, DIM = PDE::DIM;
  static constexpr int NT = TX * TY * G;
  static constexpr int RG = TX + TY;           // ring voxels per group and half
  static constexpr int HALF = G * RG;          // face-computing ring voxels (+x, +y)
  static constexpr int NR = 2 * HALF;
  static constexpr int NS = NT + 2 * NR;        // interior slots + two ring buffers (plane parity)
  static constexpr int FXG = (TX + 1) * TY, FYG = TX * (TY + 1);
  static constexpr int FX = G * FXG, FY = G * FYG;
  static constexpr int NF = PDE::NCP ? 2 : 1;
  // first thread of the +x/+y boundary faces: with one column per CTA the halo
  // ring occupies warps 0 and 1, so the faces go to warp 2 (another SM
  // sub-partition: the extra FP64 work of a plane is spread over three of them)
  static constexpr int FT0 = (NR <= 64 && NT >= 96) ? 64 : 0;
  static constexpr size_t SMEM_BASE = sizeof(double) * ((size_t)NV * NS + 2 * (size_t)N * NS + 2 * NS +
                                                        (size_t)NF * N * (FX + FY));
  // TMA staging (one column, 3D, no material): two plane buffers, each holding the interior
  // [N][TY][TX] and the ring strips -x, +x [N][TY][2] and -y, +y [N][TX] of one z-plane
  static constexpr int ST_INT = N * TX * TY, ST_XS = N * TY * 2, ST_YS = N * TX;
  static constexpr int ST_XM = ST_INT, ST_XP = ST_XM + ST_XS, ST_YM = ST_XP + ST_XS, ST_YP = ST_YM + ST_YS;
  static constexpr int ST_PLANE = ST_YP + ST_YS;  // doubles per plane buffer
  static constexpr uint32_t ST_BYTES = 8u * ST_PLANE, ST_INT_BYTES = 8u * ST_INT;
  static_assert(!TMA || (G == 1 && DIM == 3 && PDE::M == 0), "TMA staging: one column, 3D, no material");
  static_assert(!TMA || ((8 * ST_INT) % 128 == 0 && (8 * ST_XS) % 128 == 0 && (8 * ST_YS) % 128 == 0),
                "TMA destinations must stay 128-byte aligned");
  static constexpr size_t SMEM = SMEM_BASE + (TMA ? 2 * (size_t)ST_BYTES + 128 : 0);
  static_assert(NT == 256 || NT == 64, "tile classes use 256 threads, or 64 (one 8x8 column)");

  struct Smem {
    double *Q, *Fx, *Fy, *Lx, *Ly, *Hx, *Hy, *Dx, *Dy;
    double* st[2];  // TMA plane buffers (128-byte aligned)
  };
  __device__ static Smem carve(double* s) {
    Smem S;
    S.Q = s; s += NV * NS;
    S.Fx = s; s += N * NS;
    S.Fy = s; s += N * NS;
    S.Lx = s; s += NS;
    S.Ly = s; s += NS;
    S.Hx = s; s += N * FX;
    S.Hy = s; s += N * FY;
    S.Dx = s; if (PDE::NCP) s += N * FX;
    S.Dy = s; if (PDE::NCP) s += N * FY;
    if (TMA) {
      double* a = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(s) + 127) & ~(uintptr_t)127);
      S.st[0] = a;
      S.st[1] = a + ST_PLANE;
    } else {
      S.st[0] = S.st[1] = nullptr;
    }
    return S;
  }

  // Thread 0: the copies of z-plane z (0 <= z <= p; z = p is the first plane of the +z
  // neighbour) of the column into plane buffer `buf`, completing on `bar`: the interior, and
  // with `ring` the four strips around it (from this patch or its x/y neighbours, which lie
  // in the same level).
  __device__ static void tma_issue(const FvArgs& A, const FvMaps<true>& M, const Work& w, int p, int z, bool ring,
                                   double* buf, uint64_t* bar) {
    fvtma::bar_expect(bar, ring ? ST_BYTES : ST_INT_BYTES);
    if (A.debug_no_issue) return;
    const int k = w.patch[0];
    const int2 me = A.lvl[k];
    const dh_patch& pt = A.patches[k];
    const fvtma::Map* L = M.m[me.x];
    constexpr int BI = TX == 16 ? FVB_INT16 : FVB_INT32, BX = TX == 16 ? FVB_XS16 : FVB_XS8;
    constexpr int BY = TX == 16 ? FVB_YS16 : FVB_YS32;
    const int x0 = w.x0[0], y0 = w.y0[0];
    if (z >= p) {
      fvtma::load5(buf, &L[BI], x0, y0, z - p, A.lvl[pt.nbr[5]].y, 0, bar);
      return;
    }
    const int kl = me.y;
    fvtma::load5(buf, &L[BI], x0, y0, z, kl, 0, bar);
    if (!ring) return;
    if (x0 > 0) fvtma::load5(buf + ST_XM, &L[BX], x0 - 2, y0, z, kl, 0, bar);
    else fvtma::load5(buf + ST_XM, &L[BX], p - 2, y0, z, A.lvl[pt.nbr[0]].y, 0, bar);
    if (x0 + TX < p) fvtma::load5(buf + ST_XP, &L[BX], x0 + TX, y0, z, kl, 0, bar);
    else fvtma::load5(buf + ST_XP, &L[BX], 0, y0, z, A.lvl[pt.nbr[1]].y, 0, bar);
    if (y0 > 0) fvtma::load5(buf + ST_YM, &L[BY], x0, y0 - 1, z, kl, 0, bar);
    else fvtma::load5(buf + ST_YM, &L[BY], x0, p - 1, z, A.lvl[pt.nbr[2]].y, 0, bar);
    if (y0 + TY < p) fvtma::load5(buf + ST_YP, &L[BY], x0, y0 + TY, z, kl, 0, bar);
    else fvtma::load5(buf + ST_YP, &L[BY], x0, 0, z, A.lvl[pt.nbr[3]].y, 0, bar);
  }

  // Face value F^' = (FL + FR) - s (QR - QL)  (twice the Rusanov flux) and,
  // for non-conservative systems, D = B_d((QL+QR)/2)(QR - QL).
  __device__ static void face(const Smem& S, const DevParams& P, int d, int Ls, int Rs, double* H, double* D,
                              int fidx, int fstride) {
    const double* F = d == 0 ? S.Fx : S.Fy;
    const double* L = d == 0 ? S.Lx : S.Ly;
    const double s = max_nn(L[Ls], L[Rs]);
    double dq[N];
#pragma unroll
    for (int v = 0; v < N; ++v) {
      const double qL = S.Q[v * NS + Ls], qR = S.Q[v * NS + Rs];
      dq[v] = SUB(P, qR, qL);
      double h;
      if (PDE::FLUX) h = fma(-s, dq[v], ADD(P, F[v * NS + Ls], F[v * NS + Rs]));
      else h = MUL(P, -s, dq[v]);
      H[v * fstride + fidx] = h;
    }
    if (PDE::NCP) {
      double qb[NV], Dv[N];
#pragma unroll
      for (int v = 0; v < NV; ++v) qb[v] = MUL(P, 0.5, ADD(P, S.Q[v * NS + Ls], S.Q[v * NS + Rs]));
      PDE::ncp(d, qb, dq, P, Dv);
#pragma unroll
      for (int v = 0; v < N; ++v) D[v * fstride + fidx] = Dv[v];
    }
  }

  // Ring voxel r of plane z (into ring buffer buf): load, derive, flux and speed
  // in its one direction.
  __device__ static void ring_voxel(const FvArgs& A, const Smem& S, const Work& w, int r, int p, int z, int buf,
                                    const double* stb = nullptr) {
    const int h = r < HALF ? 0 : 1;
    const int rr = r - h * HALF;
    const int g = rr / RG, j = rr % RG;
    const int k = w.patch[g];
    if (k < 0) return;
    const int x0 = w.x0[g], y0 = w.y0[g];
    int x, y, d;
    if (j < TY) { d = 0; y = y0 + j; x = h == 0 ? x0 + TX : x0 - 1; }
    else { d = 1; x = x0 + (j - TY); y = h == 0 ? y0 + TY : y0 - 1; }
    const int64_t e = vox_index(A.patches, A.oct, k, p, x, y, z);
    double q[NV], W[NW > 0 ? NW : 1], F[N];
    if (TMA && stb) {
      // the staged strips of this plane: x strips start one voxel before the -x ring voxel
      // and at the +x ring voxel (two wide), y strips hold the ring rows
      const double* src = j < TY ? (h == 0 ? stb + ST_XP + 2 * j : stb + ST_XM + 2 * j + 1)
                                 : (h == 0 ? stb + ST_YP + (j - TY) : stb + ST_YM + (j - TY));
      const int vstep = j < TY ? 2 * TY : TX;
#pragma unroll
      for (int v = 0; v < NV; ++v) q[v] = src[v * vstep];
    } else {
      load_q<PDE>(A, e, q);
    }
    derive<PDE, WM>(A, e, q, W);
    const int s = NT + buf * NR + r;
#pragma unroll
    for (int v = 0; v < NV; ++v) S.Q[v * NS + s] = q[v];
    double* Fd = d == 0 ? S.Fx : S.Fy;
    double* Ld = d == 0 ? S.Lx : S.Ly;
    if (PDE::FLUX) {
      PDE::flux(d, q, W, A.P, F);
#pragma unroll
      for (int v = 0; v < N; ++v) Fd[v * NS + s] = F[v];
    }
    Ld[s] = PDE::speed(d, q, W, A.P);
  }

  // maps, bars, abort: TMA staging only (the maps of every level, two mbarriers, the CTA's
  // flag that a wait gave up)
  __device__ static void run(const FvArgs& A, const Work& w, double* smem, double& lam_thread,
                             const FvMaps<TMA>* maps = nullptr, uint64_t* bars = nullptr, int* abort = nullptr) {
    const Smem S = carve(smem);
    const int tid = threadIdx.x;
    const int g = tid / (TX * TY), lxy = tid % (TX * TY), lx = lxy % TX, ly = lxy / TX;
    const int k = w.patch[g];
    const bool act = k >= 0;
    const int pz = w.pz, z0 = w.z0;
    // the patch size of every group in this CTA is the same (pz in 3D; 2D: from the table)
    const int kk = act ? k : w.patch[0];
    const int p = A.patches[kk].p;
    const double dxk = A.patches[kk].dx;
    const int x = (act ? w.x0[g] : 0) + lx, y = (act ? w.y0[g] : 0) + ly;
    const int64_t off = act ? A.patches[k].offset : 0;
    const double dt = *A.dt_dev;
    const double gdt = A.g * dt, ddt = A.d * dt;
    // TMA bookkeeping of thread 0: a buffer whose copies no wait has yet seen complete, and
    // the parity of that buffer's current phase
    bool pend[2] = {false, false};
    uint32_t ph[2] = {0u, 0u};
    if constexpr (TMA) {
      // planes z0+1 and z0+2 (with their ring strips where they are marched) stream in while
      // the prologue loads planes z0 and z0-1
      if (tid == 0) {
        tma_issue(A, *maps, w, p, z0 + 1, 1 < pz, S.st[0], &bars[0]);
        pend[0] = true;
        if (2 <= pz) {
          tma_issue(A, *maps, w, p, z0 + 2, 2 < pz, S.st[1], &bars[1]);
          pend[1] = true;
        }
      }
    }
    const double cL = -0.5 / dxk;  // -1/(2 dx): faces hold twice the flux
    const double cS = gdt * cL, cA = ddt * cL;  // stage scalars folded with -1/(2 dx)
    const bool b1 = A.b == 1.0;
    const bool ring = tid < NR;

    // smem slots of this voxel and of its -x / -y neighbours
    const int me = tid;
    const int xm0 = lx > 0 ? me - 1 : NT + HALF + g * RG + ly;       // ring buffer 0
    const int ym0 = ly > 0 ? me - TX : NT + HALF + g * RG + TY + lx;
    const int xm1 = lx > 0 ? me - 1 : xm0 + NR;                         // ring buffer 1
    const int ym1 = ly > 0 ? me - TX : ym0 + NR;
    // face indices
    const int fxl = g * FXG + ly * (TX + 1) + lx, fxr = fxl + 1;
    const int fyl = g * FYG + ly * TX + lx, fyu = fyl + TX;

    double Qk[NV];                 // this voxel, current plane
    double Fzk[N > 0 ? N : 1];     // its z flux (3D)
    double Lzk = 0.0;              // its z speed
    double Hzlo[N], Dzlo[N];       // face below the current plane
#pragma unroll
    for (int v = 0; v < N; ++v) { Hzlo[v] = 0.0; Dzlo[v] = 0.0; Fzk[v] = 0.0; }

    // ---- prologue: plane 0 (and plane -1 for the first z face)
    if (act) {
      double Wk[NW > 0 ? NW : 1], F[N];
      load_q<PDE>(A, off + ((int64_t)z0 * p + y) * p + x, Qk);
      derive<PDE, WM>(A, off + ((int64_t)z0 * p + y) * p + x, Qk, Wk);
      if (DIM == 3 && PDE::FLUX) PDE::flux(2, Qk, Wk, A.P, Fzk);
      if (PDE::FLUX) {
        double F2[N];
        flux_xy<PDE>(Qk, Wk, Fzk, A.P, F, F2);
#pragma unroll
        for (int v = 0; v < N; ++v) { S.Fx[v * NS + me] = F[v]; S.Fy[v * NS + me] = F2[v]; }
      }
      S.Lx[me] = PDE::speed(0, Qk, Wk, A.P);
      S.Ly[me] = PDE::speed(1, Qk, Wk, A.P);
#pragma unroll
      for (int v = 0; v < NV; ++v) S.Q[v * NS + me] = Qk[v];
      if (DIM == 3) {
        Lzk = PDE::speed(2, Qk, Wk, A.P);
        // plane -1 from the -z neighbour
        double Qm[NV], Wm[NW > 0 ? NW : 1], Fzm[N];
        const int64_t em = vox_index(A.patches, A.oct, k, p, x, y, z0 - 1);
        load_q<PDE>(A, em, Qm);
        derive<PDE, WM>(A, em, Qm, Wm);
        if (PDE::FLUX) PDE::flux(2, Qm, Wm, A.P, Fzm);
        const double s = max_nn(PDE::speed(2, Qm, Wm, A.P), Lzk);
        double dq[N];
#pragma unroll
        for (int v = 0; v < N; ++v) {
          dq[v] = SUB(A.P, Qk[v], Qm[v]);
          Hzlo[v] = PDE::FLUX ? fma(-s, dq[v], ADD(A.P, Fzm[v], Fzk[v])) : MUL(A.P, -s, dq[v]);
        }
        if (PDE::NCP) {
          double qb[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) qb[v] = MUL(A.P, 0.5, ADD(A.P, Qm[v], Qk[v]));
          PDE::ncp(2, qb, dq, A.P, Dzlo);
        }
      }
    }
    if (ring) ring_voxel(A, S, w, tid, p, z0, 0);
    __syncthreads();

    for (int kz = 0; kz < pz; ++kz) {
      const int buf = kz & 1;
      const int zg = z0 + kz;  // plane index within the patch
      // the update of the next plane reads its q0 (and, in the stage-sum form, its
      // raw sums R) straight from memory: bring those lines into L2 a plane ahead
      if (act && kz + 1 < pz && (A.q0 || A.form >= 2)) {
        const int64_t e1 = off + ((int64_t)(zg + 1) * p + y) * p + x;
#pragma unroll
        for (int v = 0; v < N; ++v) {
          if (A.q0) prefetch_l2(A.q0 + v * A.vs + e1);
          if (A.form >= 2) prefetch_l2(A.acc + v * A.vs + e1);
        }
      }
      // the state (and stored derived quantities) of the plane after next, which the
      // next iteration loads for its own voxel (z <= p: at most the +z neighbour's
      // first plane)
      if (DIM == 3 && act && kz + 1 < pz) {
        const int64_t e2 = vox_index(A.patches, A.oct, k, p, x, y, zg + 2);
        if (!TMA) {
#pragma unroll
          for (int v = 0; v < N; ++v) prefetch_l2(A.qs + v * A.vs + e2);
        }
#pragma unroll
        for (int v = 0; v < PDE::M; ++v) prefetch_l2(A.mat + v * A.vs + e2);
        if (WM & 1) {
#pragma unroll
          for (int i = 0; i < NW; ++i) prefetch_l2(A.w_in + i * A.vs + e2);
        }
      }
      // ---- faces of plane kz inside the plane
      if (act) {
        face(S, A.P, 0, buf ? xm1 : xm0, me, S.Hx, S.Dx, fxl, FX);
        face(S, A.P, 1, buf ? ym1 : ym0, me, S.Hy, S.Dy, fyl, FY);
      }
      if (tid >= FT0 && tid < FT0 + HALF) {
        // +x and +y boundary faces of the column: one call with a run-time
        // direction so that a warp holding both kinds does not diverge
        const int ft = tid - FT0, gg = ft / RG, j = ft % RG;
        if (w.patch[gg] >= 0) {
          const bool isx = j < TY;
          const int Ls = isx ? gg * TX * TY + j * TX + (TX - 1) : gg * TX * TY + (TY - 1) * TX + (j - TY);
          const int fidx = isx ? gg * FXG + j * (TX + 1) + TX : gg * FYG + TY * TX + (j - TY);
          face(S, A.P, isx ? 0 : 1, Ls, NT + buf * NR + ft, isx ? S.Hx : S.Hy, isx ? S.Dx : S.Dy, fidx,
               isx ? FX : FY);
        }
      }
      // ---- next plane's own voxel (3D): derived quantities, z flux, z face
      double Qn[NV], Wn[NW > 0 ? NW : 1], Fzn[N], Lzn = 0.0, Lxn = 0.0, Lyn = 0.0, Hzhi[N], Dzhi[N];
#pragma unroll
      for (int v = 0; v < N; ++v) { Hzhi[v] = 0.0; Dzhi[v] = 0.0; Fzn[v] = 0.0; }
      // TMA: plane zg+1 in buffer kz & 1 (its (kz >> 1)-th use).  A wait that gives up raises
      // the error flag and stops this CTA's later waits (the tile's results are then invalid);
      // the buffer is re-armed only by a thread 0 that saw its phase complete, since a second
      // arrival on an unfinished phase is not allowed.
      bool staged = true;
      if constexpr (TMA) {
        staged = fvtma::bar_wait(&bars[kz & 1], (kz >> 1) & 1, abort);
        if (staged) {
          pend[kz & 1] = false;
          ph[kz & 1] ^= 1u;
        } else {
          if (!*(volatile int*)abort) atomicOr(A.err, 1u);
          *(volatile int*)abort = 1;
        }
      }
      if (DIM == 3 && act) {
        const int64_t en = vox_index(A.patches, A.oct, k, p, x, y, zg + 1);
        if constexpr (TMA) {
          const double* b = S.st[kz & 1];
#pragma unroll
          for (int v = 0; v < NV; ++v) Qn[v] = b[v * TX * TY + ly * TX + lx];
        } else {
          load_q<PDE>(A, en, Qn);
        }
        derive<PDE, WM>(A, en, Qn, Wn);
        if (PDE::FLUX) PDE::flux(2, Qn, Wn, A.P, Fzn);
        Lzn = PDE::speed(2, Qn, Wn, A.P);
        if (speeds_with_z<PDE>()) {
          Lxn = PDE::speed(0, Qn, Wn, A.P);
          Lyn = PDE::speed(1, Qn, Wn, A.P);
        }
        const double s = max_nn(Lzk, Lzn);
        double dq[N];
#pragma unroll
        for (int v = 0; v < N; ++v) {
          dq[v] = SUB(A.P, Qn[v], Qk[v]);
          Hzhi[v] = PDE::FLUX ? fma(-s, dq[v], ADD(A.P, Fzk[v], Fzn[v])) : MUL(A.P, -s, dq[v]);
        }
        if (PDE::NCP) {
          double qb[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) qb[v] = MUL(A.P, 0.5, ADD(A.P, Qk[v], Qn[v]));
          PDE::ncp(2, qb, dq, A.P, Dzhi);
        }
      }
      // EARLY variant: the ring of plane kz+1 (other ring buffer) overlaps this phase
      if (EARLY && DIM == 3 && kz + 1 < pz && ring) ring_voxel(A, S, w, tid, p, zg + 1, buf ^ 1, S.st[kz & 1]);
      __syncthreads();
      // ---- update of plane kz
      if (act) {
        double Sv[N];
        if (PDE::SRC) {
          double Wk[NW > 0 ? NW : 1];
          PDE::prims(Qk, A.P, Wk);
          PDE::source(Qk, Wk, A.P, Sv);
        }
        const int64_t e = off + ((int64_t)zg * p + y) * p + x;
        double res[NV];
#pragma unroll
        for (int v = 0; v < N; ++v) {
          const DevParams& P = A.P;
          double sum = ADD(P, SUB(P, S.Hx[v * FX + fxr], S.Hx[v * FX + fxl]),
                           SUB(P, S.Hy[v * FY + fyu], S.Hy[v * FY + fyl]));
          if (DIM == 3) sum = ADD(P, sum, SUB(P, Hzhi[v], Hzlo[v]));
          if (PDE::NCP) {
            double dsum = ADD(P, ADD(P, S.Dx[v * FX + fxr], S.Dx[v * FX + fxl]),
                              ADD(P, S.Dy[v * FY + fyu], S.Dy[v * FY + fyl]));
            if (DIM == 3) dsum = ADD(P, dsum, ADD(P, Dzhi[v], Dzlo[v]));
            sum = ADD(P, sum, dsum);
          }
          const int64_t ev = v * A.vs + e;
          if (!PDE::SRC && A.form != 0) {
            double o;
            if (A.form == 1) {
              o = fma(cS, sum, Qk[v]);
              A.acc[ev] = sum;
            } else if (A.form == 2) {
              const double t = ADD(P, A.acc[ev], sum);
              o = fma(cS, t, __ldg(A.q0 + ev));
              A.acc[ev] = t;
            } else {
              o = fma(cS, sum, fma(cA, A.acc[ev], __ldg(A.q0 + ev)));
            }
            res[v] = o;
            A.out[ev] = o;
            continue;
          }
          if (A.out) {
            double base = b1 ? Qk[v] : MUL(P, A.b, Qk[v]);
            if (A.q0) base = fma(A.a, __ldg(A.q0 + ev), base);
            res[v] = PDE::SRC ? fma(gdt, fma(cL, sum, Sv[v]), base) : fma(cS, sum, base);
          }
          if (A.acc) {
            const double r = PDE::SRC ? fma(ddt, fma(cL, sum, Sv[v]), A.acc[ev]) : fma(cA, sum, A.acc[ev]);
            A.acc[ev] = r;
            if (!A.out) res[v] = r;
          }
          if (A.out) A.out[ev] = res[v];
        }
        if (A.lam_out || (WM & 2)) {
#pragma unroll
          for (int v = N; v < NV; ++v) res[v] = Qk[v];
          double Wr[NW > 0 ? NW : 1];
          PDE::prims(res, A.P, Wr);
          if (WM & 2) {
#pragma unroll
            for (int i = 0; i < NW; ++i) A.w_out[i * A.vs + e] = Wr[i];
          }
          if (A.lam_out) {
            double l = max_nn(PDE::speed(0, res, Wr, A.P), PDE::speed(1, res, Wr, A.P));
            if (DIM == 3) l = max_nn(l, PDE::speed(2, res, Wr, A.P));
            lam_thread = max_nn(lam_thread, l);
          }
        }
      }
      // ---- publish plane kz+1 (3D)
      if (DIM == 3 && kz + 1 < pz) {
        if (act) {
          if (PDE::FLUX) {
            double F[N], F2[N];
            flux_xy<PDE>(Qn, Wn, Fzn, A.P, F, F2);
#pragma unroll
            for (int v = 0; v < N; ++v) { S.Fx[v * NS + me] = F[v]; S.Fy[v * NS + me] = F2[v]; }
          }
          S.Lx[me] = speeds_with_z<PDE>() ? Lxn : PDE::speed(0, Qn, Wn, A.P);
          S.Ly[me] = speeds_with_z<PDE>() ? Lyn : PDE::speed(1, Qn, Wn, A.P);
#pragma unroll
          for (int v = 0; v < NV; ++v) { S.Q[v * NS + me] = Qn[v]; Qk[v] = Qn[v]; }
#pragma unroll
          for (int v = 0; v < N; ++v) { Fzk[v] = Fzn[v]; Hzlo[v] = Hzhi[v]; Dzlo[v] = Dzhi[v]; }
          Lzk = Lzn;
        }
        if (!EARLY && ring) ring_voxel(A, S, w, tid, p, zg + 1, buf ^ 1, S.st[kz & 1]);
        __syncthreads();
        // buffer kz & 1 is free again: plane zg+3 streams into it
        if constexpr (TMA) {
          if (tid == 0 && staged && !*(volatile int*)abort && kz + 3 <= pz) {
            tma_issue(A, *maps, w, p, zg + 3, kz + 3 < pz, S.st[kz & 1], &bars[kz & 1]);
            pend[kz & 1] = true;
          }
        }
      }
    }
    if constexpr (TMA) {
      // after a wait gave up, copies this thread issued may still be in flight: wait for them
      // (bounded again) before the CTA moves on or exits
      if (tid == 0) {
        int never = 0;
        for (int b = 0; b < 2; ++b)
          if (pend[b]) fvtma::bar_wait(&bars[b], ph[b], &never);
      }
    }
  }
};

static __device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide max, then one atomicMax per CTA and last-CTA publication.
static __device__ void publish_lambda(double lam, double* lam_out, unsigned long long* red, double* dt_next = nullptr,
                                      double cfl = 0.0, double dx_dim = 0.0) {
  __shared__ double wmax[32];
  __shared__ bool last;
  lam = warp_max(lam);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) wmax[wid] = lam;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, wmax[i]);
    atomicMax(red, (unsigned long long)__double_as_longlong(m));
    __threadfence();
    const unsigned long long t = atomicAdd(red + 1, 1ull);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    const unsigned long long bits = atomicAdd(red, 0ull);
    const double lmax = __longlong_as_double((long long)bits);
    *lam_out = lmax;
    // every CTA read dt before taking its ticket, so the last one may overwrite it
    if (dt_next) *dt_next = cfl * dx_dim / lmax;
    red[0] = 0ull;
    red[1] = 0ull;
    __threadfence();
  }
}

// Persistent launch: the next tile of the cost-sorted list for this CTA (thread 0 takes it
// from the queue, the CTA reads it after a barrier).
static __device__ __forceinline__ int fv_next_item(unsigned int* queue) {
  __shared__ int s_item;
  if (threadIdx.x == 0) s_item = (int)atomicAdd(queue, 1u);
  __syncthreads();
  return s_item;
}

// Persistent launch: every CTA leaves the queue once, after its last (empty) fetch; the last
// one to leave resets the queue for the next launch (no CTA waits for another).
static __device__ __forceinline__ void fv_queue_exit(unsigned int* queue) {
  if (threadIdx.x == 0) {
    const unsigned int done = atomicAdd(queue + 1, 1u);
    if (done == gridDim.x - 1) {
      atomicExch(queue, 0u);
      atomicExch(queue + 1, 0u);
    }
  }
}

// Kernel variants (chosen per plan by the autotuner, dh_autotune):
//   VAR bit 0: EARLY -- the halo ring of the next plane is computed before the
//              mid-plane barrier instead of after it;
//   VAR bit 1: at most 128 registers so that two CTAs fit on an SM;
//   VAR bits 2-3: WM -- bit 2 reads W of qs from A.w_in instead of computing
//              it, bit 3 writes W of the result to A.w_out (multi-step graphs:
//              the last stage of a step hands W to the first stage of the next);
//   VAR bit 4: persistent -- the grid is SMs x resident CTAs and every CTA takes
//              tiles from the queue A.queue until it is empty;
//   VAR bit 5: the work list may hold 32x8 columns (tile class 2).
// Tile classes (per work item): 0 = one 16x16 column, 1 = four 8x8 columns (up to
// four patches), 2 = one 32x8 column.  Bits 4 and 5 are compiled for the
// register-capped variants only: the loop of the persistent form and a third
// tile class both raise the register demand, and the capped kernels are the ones
// that win on the three-dimensional workloads.
template <class PDE, bool EARLY, int WM, bool T32, bool TMA>
static __device__ __forceinline__ void fv_run_tile(const FvArgs& A, const Work& w, double* smem, double& lam,
                                                   const FvMaps<TMA>* maps, uint64_t* bars, int* abort) {
  if (w.cls == 0) FvTile<PDE, 16, 16, 1, EARLY, WM, TMA>::run(A, w, smem, lam, maps, bars, abort);
  else if (!T32 || w.cls == 1) FvTile<PDE, 8, 8, 4, EARLY, WM>::run(A, w, smem, lam);
  else if constexpr (T32) FvTile<PDE, 32, 8, 1, EARLY, WM, TMA>::run(A, w, smem, lam, maps, bars, abort);
}

//   VAR bit 6: TMA -- the z-planes of 16x16 and 32x8 columns and their ring strips are
//              brought into a double-buffered shared-memory ring by tensor copies (3D
//              Euler on plans whose levels are runs of back-to-back patches).
template <class PDE, int VAR>
__global__ void __launch_bounds__(256, (VAR & 2) ? 2 : 1)
    k_fv_stage(const __grid_constant__ FvArgs A, const __grid_constant__ FvMaps<(VAR & 64) != 0> M) {
  extern __shared__ __align__(128) double smem[];
  constexpr bool EARLY = (VAR & 1) != 0;
  constexpr int WM = (VAR >> 2) & 3;
  constexpr bool PERS = (VAR & 16) != 0, T32 = (VAR & 32) != 0, TMA = (VAR & 64) != 0;
  static_assert(!(TMA && PERS), "the TMA-staged variant runs one tile per CTA");
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ int abort_flag;
  if constexpr (TMA) {
    if (threadIdx.x == 0) {
      fvtma::bar_init(&bars[0], 1);
      fvtma::bar_init(&bars[1], 1);
      fvtma::bar_fence_init();
      abort_flag = 0;
    }
    __syncthreads();
  }
  double lam = 0.0;
  const FvArgs R = with_reg_params(A);
  if constexpr (PERS) {
    for (int t = fv_next_item(A.queue); t < A.n_work; t = fv_next_item(A.queue)) {
      fv_run_tile<PDE, EARLY, WM, T32, false>(R, A.work[t], smem, lam, nullptr, nullptr, nullptr);
      __syncthreads();  // the next tile reuses the shared memory
    }
    fv_queue_exit(A.queue);
  } else {
    fv_run_tile<PDE, EARLY, WM, T32, TMA>(R, A.work[blockIdx.x], smem, lam, &M, bars, &abort_flag);
  }
  if (A.lam_out) publish_lambda(lam, A.lam_out, A.red, A.dt_next, A.cfl, A.dx_dim);
}

// Tile set 3: one 8x8 column per 64-thread CTA (small problems: four times the CTAs of the
// 256-thread tiles, so that more SMs share the FP64 work).
template <class PDE, int VAR>
__global__ void __launch_bounds__(64, (VAR & 2) ? 8 : 1) k_fv_stage64(const __grid_constant__ FvArgs A) {
  extern __shared__ __align__(128) double smem[];
  constexpr bool EARLY = (VAR & 1) != 0;
  constexpr int WM = (VAR >> 2) & 3;
  double lam = 0.0;
  const FvArgs R = with_reg_params(A);
  FvTile<PDE, 8, 8, 1, EARLY, WM>::run(R, A.work[blockIdx.x], smem, lam);
  if (A.lam_out) publish_lambda(lam, A.lam_out, A.red, A.dt_next, A.cfl, A.dx_dim);
}

template <class PDE, int VAR>
static dh_status launch_var64(dh_plan* plan, const FvArgs& A, cudaStream_t stream) {
  constexpr bool EARLY = (VAR & 1) != 0;
  constexpr int WM = (VAR >> 2) & 3;
  constexpr size_t smem = FvTile<PDE, 8, 8, 1, EARLY, WM>::SMEM;
  static int configured_device = -1;
  if (configured_device != plan->device) {
    cudaError_t e = cudaFuncSetAttribute(k_fv_stage64<PDE, VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(k_fv_stage64)");
    configured_device = plan->device;
  }
  const int li = plan->fv_list();
  FvArgs B = A;
  B.work = plan->d_wl[li];
  B.n_work = plan->n_wl[li];
  B.queue = nullptr;
  if (B.n_work <= 0) return DH_OK;
  k_fv_stage64<PDE, VAR><<<B.n_work, 64, smem, stream>>>(B);
  return cuda_error(cudaGetLastError(), "k_fv_stage64 launch");
}

template <class PDE, int VAR>
static size_t fv_smem(bool c0, bool c1, bool c2) {
  constexpr bool EARLY = (VAR & 1) != 0;
  constexpr int WM = (VAR >> 2) & 3;
  constexpr bool TMA = (VAR & 64) != 0;
  return std::max({c0 ? FvTile<PDE, 16, 16, 1, EARLY, WM, TMA>::SMEM : (size_t)0,
                   c1 ? FvTile<PDE, 8, 8, 4, EARLY, WM>::SMEM : (size_t)0,
                   c2 ? FvTile<PDE, 32, 8, 1, EARLY, WM, TMA>::SMEM : (size_t)0});
}

template <class PDE, int VAR>
static dh_status launch_var(dh_plan* plan, const FvArgs& A, cudaStream_t stream,
                            const FvMaps<(VAR & 64) != 0>& M = FvMaps<(VAR & 64) != 0>{}) {
  constexpr bool PERS = (VAR & 16) != 0, T32 = (VAR & 32) != 0;
  const int li = plan->fv_list();
  const bool* cls = plan->wl_cls[li];
  if (cls[2] && !T32) {
    set_error("k_fv_stage: the work list holds 32x8 columns but the kernel variant has no such tile class");
    return DH_EUNSUPPORTED;
  }
  const size_t smem = fv_smem<PDE, VAR>(cls[0], cls[1], cls[2]);
  static int configured_device = -1;  // attribute is per device function; set once per process and device
  if (configured_device != plan->device) {
    cudaError_t e = cudaFuncSetAttribute(k_fv_stage<PDE, VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fv_smem<PDE, VAR>(true, true, T32));
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(k_fv_stage)");
    configured_device = plan->device;
  }
  FvArgs B = A;
  B.work = plan->d_wl[li];
  B.n_work = plan->n_wl[li];
  int grid = B.n_work;
  B.queue = nullptr;
  if (PERS) {
    // as many CTAs as fit on the GPU at once
    int nb = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fv_stage<PDE, VAR>, 256, smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(k_fv_stage)");
    grid = std::min(grid, std::max(1, nb) * plan->num_sms);
    B.queue = reinterpret_cast<unsigned int*>(plan->d_red + 3);
  }
  if (grid <= 0) return DH_OK;
  k_fv_stage<PDE, VAR><<<grid, 256, smem, stream>>>(B, M);
  return cuda_error(cudaGetLastError(), "k_fv_stage launch");
}

// The TMA-staged variants (fv_var bit 5) are instantiated in their own translation unit.
dh_status fv_launch_euler3_tma(dh_plan* plan, const FvArgs& A, int wm, cudaStream_t stream);

template <class PDE, int WM>
static dh_status launch_wm(dh_plan* plan, const FvArgs& A, cudaStream_t stream) {
  constexpr int W = WM << 2;
  const int v = plan->fv_var;
  if (v & 32) {
    if constexpr (std::is_same<PDE, PdeEuler3>::value) return fv_launch_euler3_tma(plan, A, WM, stream);
    set_error("k_fv_stage: the TMA-staged variant exists for 3D Euler only");
    return DH_EUNSUPPORTED;
  }
  if (((v >> 3) & 3) == 3) {
    if (v & 4) {
      set_error("k_fv_stage: tile set 3 runs one CTA per column (no persistent grid)");
      return DH_EUNSUPPORTED;
    }
    switch (v & 3) {
      case 0: return launch_var64<PDE, 0 | W>(plan, A, stream);
      case 1: return launch_var64<PDE, 1 | W>(plan, A, stream);
      case 2: return launch_var64<PDE, 2 | W>(plan, A, stream);
      default: return launch_var64<PDE, 3 | W>(plan, A, stream);
    }
  }
  const int ext = ((v & 4) ? 16 : 0) | ((((v >> 3) & 3) == 1) ? 32 : 0);
  if (ext && !(v & 2)) {
    set_error("k_fv_stage: the persistent grid and 32x8 columns are compiled for the register-capped variants (fv_var bit 1)");
    return DH_EUNSUPPORTED;
  }
  switch (ext | (v & 3)) {
    case 0: return launch_var<PDE, 0 | W>(plan, A, stream);
    case 1: return launch_var<PDE, 1 | W>(plan, A, stream);
    case 2: return launch_var<PDE, 2 | W>(plan, A, stream);
    case 3: return launch_var<PDE, 3 | W>(plan, A, stream);
    case 18: return launch_var<PDE, 18 | W>(plan, A, stream);
    case 19: return launch_var<PDE, 19 | W>(plan, A, stream);
    case 34: return launch_var<PDE, 34 | W>(plan, A, stream);
    case 35: return launch_var<PDE, 35 | W>(plan, A, stream);
    case 50: return launch_var<PDE, 50 | W>(plan, A, stream);
    default: return launch_var<PDE, 51 | W>(plan, A, stream);
  }
}

}  // namespace dh

#include "dh_fv_any.cuh"

namespace dh {

// W reuse is compiled for the Euler systems only (the systems whose derived
// quantities cost a reciprocal and a square root per voxel).  Plans whose patch sizes are
// not all multiples of 8 run the generic stage.
template <class PDE>
static dh_status fv_launch_pde(dh_plan* plan, const FvArgs& A, int wmode, cudaStream_t stream) {
  if (plan->fv_generic) return launch_any<PDE>(plan, A, wmode, stream);
  if constexpr (std::is_same<PDE, PdeEuler2>::value || std::is_same<PDE, PdeEuler3>::value) {
    switch (wmode & 3) {
      case 1: return launch_wm<PDE, 1>(plan, A, stream);
      case 2: return launch_wm<PDE, 2>(plan, A, stream);
      case 3: return launch_wm<PDE, 3>(plan, A, stream);
      default: break;
    }
  }
  return launch_wm<PDE, 0>(plan, A, stream);
}

// One translation unit per PDE instantiates the stage kernels (they compile in parallel).
dh_status fv_launch_adv_flux(dh_plan* plan, const FvArgs& A, int wmode, cudaStream_t stream);
dh_status fv_launch_adv_ncp(dh_plan* plan, const FvArgs& A, int wmode, cudaStream_t stream);
dh_status fv_launch_euler2(dh_plan* plan, const FvArgs& A, int wmode, cudaStream_t stream);
dh_status fv_launch_euler3(dh_plan* plan, const FvArgs& A, int wmode, cudaStream_t stream);
dh_status fv_launch_srhd(dh_plan* plan, const FvArgs& A, int wmode, cudaStream_t stream);

}  // namespace dh
