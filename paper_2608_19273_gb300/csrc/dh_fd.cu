// Finite-difference Runge-Kutta stage: 4th-order centred first derivatives and
// 6th-difference Kreiss-Oliger dissipation (paper Sec. I and Sec. IV: FD4
// with KO dissipation; KO normalisation sigma/(64 dx) is the r = 3 form):
//   L(Q) = -sum_d B_d(Q) dQ/dx_d + S(Q) + sigma/(64 dx) sum_d delta6_d Q
//   dQ/dx  = [(Q_-2 - Q_+2) + 8 (Q_+1 - Q_-1)] / (12 dx)
//   delta6 = (Q_-3 + Q_+3 - 2Q_0) - 6 (Q_-2 + Q_+2 - 2Q_0) + 15 (Q_-1 + Q_+1 - 2Q_0)
//   out = a q0 + b qs + g dt L ; acc += d dt L
// (the bracketed delta6 form is exactly zero on constant data, so constant
// states stay bitwise constant).
//
// Kernel design: a CTA owns an 8x8x4 tile of one patch (one voxel per
// thread).  The variables are staged, a group at a time, into a padded
// 14x14x10 shared-memory box holding the tile and its three-voxel face halos
// (edges and corners are never read by the axis-aligned stencils and are not
// loaded).  Halo voxels outside the patch come from the face neighbours.
// Every derivative is taken only for the variables that a column of B_d
// reads.  Systems with up to 8 unknowns stage all variables at once; the
// 59-unknown GW59 system is processed field by field (lapse/shift first,
// then the 11 scalar-wave fields), keeping per voxel only the few coupling
// quantities (alpha, beta, grad alpha, phi_b Pi_b, source sums) in registers.
#include "dh_internal.cuh"
#include "dh_pde.cuh"

namespace dh {

struct FdArgs {
  const dh_patch* patches;
  const FdWork* work;
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

// Stage variables [v0, v0 + nv) of qs into smem boxes 0..nv-1.
__device__ __forceinline__ void fd_stage_vars(const FdArgs& A, double* box, const FdWork& w, int p, int v0, int nv) {
  for (int s = threadIdx.x; s < FNSLOT; s += FNT) {
    int x, y, z;
    fd_slot(s, x, y, z);
    const int64_t e = fd_vox_index(A.patches, w.patch, p, w.x0 + x, w.y0 + y, w.z0 + z);
    const int c = fd_box(x, y, z);
    for (int v = 0; v < nv; ++v) box[v * FBOX + c] = __ldg(A.qs + (int64_t)(v0 + v) * A.vs + e);
  }
}

// 4th-order centred derivative (times 1/(12 dx)) along stride st.
__device__ __forceinline__ double fd_d1(const DevParams& P, const double* s, int c, int st, double r12) {
  return PMUL(P, fma(8.0, PSUB(P, s[c + st], s[c - st]), PSUB(P, s[c - 2 * st], s[c + 2 * st])), r12);
}
// Bracketed sixth difference (exactly 0 on constants).
__device__ __forceinline__ double fd_d6(const DevParams& P, const double* s, int c, int st) {
  const double two = PMUL(P, 2.0, s[c]);
  const double t3 = PSUB(P, PADD(P, s[c - 3 * st], s[c + 3 * st]), two);
  const double t2 = PSUB(P, PADD(P, s[c - 2 * st], s[c + 2 * st]), two);
  const double t1 = PSUB(P, PADD(P, s[c - st], s[c + st]), two);
  return fma(15.0, t1, fma(-6.0, t2, t3));
}
__device__ __forceinline__ double fd_ko3(const DevParams& P, const double* s, int c) {
  return PADD(P, PADD(P, fd_d6(P, s, c, 1), fd_d6(P, s, c, FBX)), fd_d6(P, s, c, FBX * FBY));
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

// ------------------------------------------------------------- generic (N <= 8)
template <class PDE>
__device__ void fd_tile_generic(const FdArgs& A, const FdWork& w, double* box, double& lam_thread) {
  constexpr int N = PDE::N, NV = PDE::N + PDE::M;
  const dh_patch& pt = A.patches[w.patch];
  const int p = pt.p;
  fd_stage_vars(A, box, w, p, 0, N);
  __syncthreads();
  const int t = threadIdx.x;
  const int lx = t % FTX, ly = (t / FTX) % FTY, lz = t / (FTX * FTY);
  const int c = fd_box(lx, ly, lz);
  const int64_t e = pt.offset + ((int64_t)(w.z0 + lz) * p + (w.y0 + ly)) * p + (w.x0 + lx);
  const double dx = pt.dx;
  const double r12 = 1.0 / (12.0 * dx);
  const double ko = A.sigma / (64.0 * dx);
  const double dt = *A.dt_dev;
  const double gdt = A.g * dt, ddt = A.d * dt;
  double q[NV], L[N], W[1];
#pragma unroll
  for (int v = 0; v < N; ++v) q[v] = box[v * FBOX + c];
#pragma unroll
  for (int v = 0; v < PDE::M; ++v) q[N + v] = __ldg(A.mat + (int64_t)v * A.vs + e);
  if (PDE::SRC) PDE::source(q, W, A.P, L);
  else {
#pragma unroll
    for (int v = 0; v < N; ++v) L[v] = 0.0;
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int st = d == 0 ? 1 : (d == 1 ? FBX : FBX * FBY);
    double dq[N], D[N];
#pragma unroll
    for (int v = 0; v < N; ++v) dq[v] = PDE::needs_grad(d, v) ? fd_d1(A.P, box + v * FBOX, c, st, r12) : 0.0;
    PDE::ncp(d, q, dq, A.P, D);
#pragma unroll
    for (int v = 0; v < N; ++v) L[v] = PSUB(A.P, L[v], D[v]);
  }
  double res[NV];
#pragma unroll
  for (int v = 0; v < N; ++v) {
    const double Lv = fma(ko, fd_ko3(A.P, box + v * FBOX, c), L[v]);
    res[v] = fd_combine(A, (int64_t)v * A.vs + e, q[v], Lv, gdt, ddt);
  }
  if (A.lam_out) {
#pragma unroll
    for (int v = N; v < NV; ++v) res[v] = q[v];
    double l = fmax(fmax(PDE::speed(0, res, W, A.P), PDE::speed(1, res, W, A.P)), PDE::speed(2, res, W, A.P));
    lam_thread = fmax(lam_thread, l);
  }
}

// ------------------------------------------------------------- GW59
__device__ void fd_tile_gw59(const FdArgs& A, const FdWork& w, double* box, double& lam_thread) {
  const dh_patch& pt = A.patches[w.patch];
  const int p = pt.p;
  const int t = threadIdx.x;
  const int lx = t % FTX, ly = (t / FTX) % FTY, lz = t / (FTX * FTY);
  const int c = fd_box(lx, ly, lz);
  const int64_t e = pt.offset + ((int64_t)(w.z0 + lz) * p + (w.y0 + ly)) * p + (w.x0 + lx);
  const int64_t vs = A.vs;
  const double dx = pt.dx;
  const double r12 = 1.0 / (12.0 * dx);
  const double ko = A.sigma / (64.0 * dx);
  const double dt = *A.dt_dev;
  const double gdt = A.g * dt, ddt = A.d * dt;
  constexpr int X = 1, Y = FBX, Z = FBX * FBY;

  // lapse and shift: values, grad alpha, KO
  fd_stage_vars(A, box, w, p, 55, 4);
  __syncthreads();
  const double al = box[c], bx = box[FBOX + c], by = box[2 * FBOX + c], bz = box[3 * FBOX + c];
  const DevParams& P = A.P;
  const double dal0 = fd_d1(P, box, c, X, r12), dal1 = fd_d1(P, box, c, Y, r12), dal2 = fd_d1(P, box, c, Z, r12);
  double ko_ab[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) ko_ab[v] = PMUL(P, ko, fd_ko3(P, box + v * FBOX, c));
  // phi_b Pi_b at this voxel for the source coupling
  double u[11];
#pragma unroll
  for (int bb = 0; bb < 11; ++bb) u[bb] = PMUL(P, __ldg(A.qs + (int64_t)(5 * bb) * vs + e), __ldg(A.qs + (int64_t)(5 * bb + 1) * vs + e));
  double sumPi2 = 0.0, bs0 = 0.0, bs1 = 0.0, bs2 = 0.0;

#pragma unroll 1
  for (int a = 0; a < 11; ++a) {
    __syncthreads();  // previous group's box reads are done
    fd_stage_vars(A, box, w, p, 5 * a, 5);
    __syncthreads();
    const double* sphi = box;
    const double* sPi = box + FBOX;
    const double* spx = box + 2 * FBOX;
    const double* spy = box + 3 * FBOX;
    const double* spz = box + 4 * FBOX;
    const double phi = sphi[c], Pi = sPi[c], px = spx[c], py = spy[c], pz = spz[c];
    const double dPi0 = fd_d1(P, sPi, c, X, r12), dPi1 = fd_d1(P, sPi, c, Y, r12), dPi2 = fd_d1(P, sPi, c, Z, r12);
    // coupling sum_b C_ab phi_b Pi_b
    double cs = PMUL(P, A.P.C[11 * a], u[0]);
#pragma unroll
    for (int bb = 1; bb < 11; ++bb) cs = fma(A.P.C[11 * a + bb], u[bb], cs);
    // phi: alpha Pi + beta . psi
    const double Lphi = fma(al, Pi, fma(bx, px, fma(by, py, PMUL(P, bz, pz))));
    // Pi: alpha div psi + beta . grad Pi + alpha cs
    const double dpx0 = fd_d1(P, spx, c, X, r12), dpx1 = fd_d1(P, spx, c, Y, r12), dpx2 = fd_d1(P, spx, c, Z, r12);
    const double dpy0 = fd_d1(P, spy, c, X, r12), dpy1 = fd_d1(P, spy, c, Y, r12), dpy2 = fd_d1(P, spy, c, Z, r12);
    const double dpz0 = fd_d1(P, spz, c, X, r12), dpz1 = fd_d1(P, spz, c, Y, r12), dpz2 = fd_d1(P, spz, c, Z, r12);
    const double LPi = fma(al, PADD(P, PADD(P, dpx0, dpy1), dpz2), fma(bx, dPi0, fma(by, dPi1, fma(bz, dPi2, PMUL(P, al, cs)))));
    // psi_i: alpha d_i Pi + Pi d_i alpha + beta . grad psi_i
    const double Lpx = fma(al, dPi0, fma(Pi, dal0, fma(bx, dpx0, fma(by, dpx1, PMUL(P, bz, dpx2)))));
    const double Lpy = fma(al, dPi1, fma(Pi, dal1, fma(bx, dpy0, fma(by, dpy1, PMUL(P, bz, dpy2)))));
    const double Lpz = fma(al, dPi2, fma(Pi, dal2, fma(bx, dpz0, fma(by, dpz1, PMUL(P, bz, dpz2)))));
    sumPi2 = fma(Pi, Pi, sumPi2);
    bs0 = fma(px, Pi, bs0);
    bs1 = fma(py, Pi, bs1);
    bs2 = fma(pz, Pi, bs2);
    const int64_t eb = (int64_t)(5 * a) * vs + e;
    fd_combine(A, eb, phi, fma(ko, fd_ko3(P, sphi, c), Lphi), gdt, ddt);
    fd_combine(A, eb + vs, Pi, fma(ko, fd_ko3(P, sPi, c), LPi), gdt, ddt);
    fd_combine(A, eb + 2 * vs, px, fma(ko, fd_ko3(P, spx, c), Lpx), gdt, ddt);
    fd_combine(A, eb + 3 * vs, py, fma(ko, fd_ko3(P, spy, c), Lpy), gdt, ddt);
    fd_combine(A, eb + 4 * vs, pz, fma(ko, fd_ko3(P, spz, c), Lpz), gdt, ddt);
  }
  const double Lal = fma(PMUL(P, -A.P.kappa, PMUL(P, al, al)), sumPi2, ko_ab[0]);
  const double ra = fd_combine(A, 55 * vs + e, al, Lal, gdt, ddt);
  const double r0 = fd_combine(A, 56 * vs + e, bx, fma(0.75, bs0, ko_ab[1]), gdt, ddt);
  const double r1 = fd_combine(A, 57 * vs + e, by, fma(0.75, bs1, ko_ab[2]), gdt, ddt);
  const double r2 = fd_combine(A, 58 * vs + e, bz, fma(0.75, bs2, ko_ab[3]), gdt, ddt);
  if (A.lam_out) lam_thread = fmax(lam_thread, PADD(P, ra, fmax(fmax(fabs(r0), fabs(r1)), fabs(r2))));
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

// Kernel variants (chosen per plan by the autotuner): VAR bit 1 caps the
// registers at 128 so that two CTAs fit on an SM.
template <class PDE, int VAR>
__global__ void __launch_bounds__(FNT, (VAR & 2) ? 2 : 1) k_fd_stage(const __grid_constant__ FdArgs A) {
  extern __shared__ __align__(16) double box[];
  const FdWork w = A.work[blockIdx.x];
  double lam = 0.0;
  if constexpr (PDE::N == 59) fd_tile_gw59(A, w, box, lam);
  else fd_tile_generic<PDE>(A, w, box, lam);
  if (A.lam_out) fd_publish_lambda(lam, A.lam_out, A.red);
}

template <class PDE, int VAR>
static dh_status fd_launch_var(dh_plan* plan, const FdArgs& A, cudaStream_t stream) {
  constexpr int NB = PDE::N == 59 ? 5 : PDE::N;
  const size_t smem = sizeof(double) * NB * FBOX;
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
  return (plan->fd_var & 2) ? fd_launch_var<PDE, 2>(plan, A, stream) : fd_launch_var<PDE, 0>(plan, A, stream);
}

dh_status launch_fd_stage(dh_plan* plan, const double* qs, const double* q0, double* out, double* acc,
                          const double* mat, const double* dt_dev, double a, double b, double g, double d,
                          double sigma, double* lam_out, cudaStream_t stream) {
  FdArgs A;
  A.patches = plan->d_patches;
  A.work = plan->d_fdwork;
  A.qs = qs; A.q0 = q0; A.out = out; A.acc = acc; A.mat = mat; A.dt_dev = dt_dev;
  A.a = a; A.b = b; A.g = g; A.d = d; A.sigma = sigma;
  A.lam_out = lam_out;
  A.red = plan->d_red;
  A.vs = plan->var_stride;
  A.P = plan->params;
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
