// Second-order finite-volume Runge-Kutta stage over all patches in one launch:
// MUSCL reconstruction with the minmod limiter feeding the Rusanov flux (the
// face-state step of the face-flux operator, Sec. II-A Eq. 3, where a state on
// each side of a face comes from a linear stencil over neighbouring voxels),
// for conservative systems (B = 0):
//   sigma_i = minmod(Q_i - Q_{i-1}, Q_{i+1} - Q_i)            (per component)
//   minmod(a, b) = 0 if a, b differ in sign, else the one of smaller magnitude
//   QL = Q_{f-1} + sigma_{f-1}/2,  QR = Q_f - sigma_f/2         (face f)
//   F^ = (F_d(QL) + F_d(QR))/2 - s/2 (QR - QL),  s = max(lambda_d(QL), lambda_d(QR))
//   L(Q)_i = -(1/dx) sum_d [F^_{i+1/2} - F^_{i-1/2}] + S(Q_i)
//   out = a q0 + b qs + g dt L ; acc += d dt L
// A face state carries the material parameters of the voxel it comes from.
//
// Kernel design (the FP64 pipe is the bottleneck, so every slope, face state
// and face state's flux and speed is computed once):
//   * A CTA owns an 8x8x4 tile of one patch (one voxel per thread) and stages
//     its N (+M) quantities with two-voxel face halos into shared memory by
//     plain coalesced loads; halo voxels outside the patch come from the face
//     neighbours (edges and corners are never read and not loaded).
//   * Directions are processed one at a time.  Phase 1: each thread computes
//     the limited slope of its voxel along d and its two face states (+ and -),
//     each with derived quantities, flux F_d and speed; the first threads also
//     compute the inward face state of each halo voxel next to the tile.  The
//     states go to shared memory (F, lambda, Q of each).  Phase 2: the
//     threads form the Rusanov flux of every face along d once, from the
//     stored states, in place of the left state's flux.  Phase 3: each thread
//     accumulates the difference of its two faces.  Face values hold twice the
//     flux; the factor 1/2 is folded into -1/(2 dx).
//   * minmod and all speed maxima run on the integer pipe (sign bits and
//     magnitude bits of the doubles).
//   * lambda_max of the result: warp shuffles, one atomicMax per CTA on the
//     bit pattern, last CTA publishes (no spin waits).
#include <algorithm>

#include "dh_internal.cuh"
#include "dh_pde.cuh"

namespace dh {
namespace {

constexpr int MX = 8, MY = 8, MZ = 4, MH = 2;
constexpr int MBX = MX + 2 * MH, MBY = MY + 2 * MH, MBZ = MZ + 2 * MH;
constexpr int MBOX = MBX * MBY * MBZ;                                          // 1152 slots per quantity
constexpr int MNT = MX * MY * MZ;                                              // 256 threads
constexpr int MSLOT = MNT + 2 * MH * (MY * MZ + MX * MZ + MX * MY);            // tile + face halos: 768
constexpr int MFS = (MZ + 1) * MX * MY;                                        // 320 >= (T_d + 1) * area

struct Fv2Args {
  const dh_patch* patches;
  const FdWork* work;
  const double* qs;
  const double* q0;
  double* out;
  double* acc;
  const double* mat;
  const double* dt_dev;
  double a, b, g, d;
  double* lam_out;
  unsigned long long* red;
  int64_t vs;
  DevParams P;
};

__device__ __forceinline__ int mbox(int x, int y, int z) { return ((z + MH) * MBY + (y + MH)) * MBX + (x + MH); }

// Arena index of voxel (x, y, z) of patch k; at most one coordinate outside [0, p).
__device__ __forceinline__ int64_t m_vox(const dh_patch* __restrict__ P, int k, int p, int x, int y, int z) {
  if (x < 0) { k = P[k].nbr[0]; x += p; }
  else if (x >= p) { k = P[k].nbr[1]; x -= p; }
  else if (y < 0) { k = P[k].nbr[2]; y += p; }
  else if (y >= p) { k = P[k].nbr[3]; y -= p; }
  else if (z < 0) { k = P[k].nbr[4]; z += p; }
  else if (z >= p) { k = P[k].nbr[5]; z -= p; }
  return P[k].offset + ((int64_t)z * p + y) * p + x;
}

// Slot s of the tile-plus-face-halo set -> tile-relative (x, y, z).
__device__ __forceinline__ void m_slot(int s, int& x, int& y, int& z) {
  if (s < MNT) { x = s % MX; y = (s / MX) % MY; z = s / (MX * MY); return; }
  int r = s - MNT;
  if (r < 2 * MH * MY * MZ) {
    const int side = r / (MH * MY * MZ), rr = r % (MH * MY * MZ);
    const int h = rr % MH;
    y = (rr / MH) % MY; z = rr / (MH * MY);
    x = side == 0 ? -MH + h : MX + h;
    return;
  }
  r -= 2 * MH * MY * MZ;
  if (r < 2 * MH * MX * MZ) {
    const int side = r / (MH * MX * MZ), rr = r % (MH * MX * MZ);
    x = rr % MX; const int h = (rr / MX) % MH; z = rr / (MX * MH);
    y = side == 0 ? -MH + h : MY + h;
    return;
  }
  r -= 2 * MH * MX * MZ;
  const int side = r / (MH * MX * MY), rr = r % (MH * MX * MY);
  x = rr % MX; y = (rr / MX) % MY; const int h = rr / (MX * MY);
  z = side == 0 ? -MH + h : MZ + h;
}

// minmod on the integer pipe: 0 if the signs differ, else the argument of smaller magnitude.
__device__ __forceinline__ double minmod(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  if ((ia ^ ib) < 0) return 0.0;
  return (ia & 0x7fffffffffffffffll) < (ib & 0x7fffffffffffffffll) ? a : b;
}

template <class PDE>
struct Fv2Tile {
  static constexpr int N = PDE::N, NV = PDE::N + PDE::M, NW = PDE::NW;
  static constexpr int NS = 2 * N + 1;  // one face state: F (N), lambda, Q (N)
  static constexpr size_t SMEM = sizeof(double) * ((size_t)NV * MBOX + 2 * (size_t)NS * MFS);

  // Face states of the voxel at box index c along d (box stride st): limited
  // slope, then the + state into sp[ip] (if sp != nullptr) and the - state into
  // sm[im] (if sm != nullptr); entry i of a state array sits at [component * MFS + i].
  __device__ static void states(const Fv2Args& A, const double* box, int c, int st, int d, double* sp, int ip,
                                double* sm, int im) {
    const DevParams& P = A.P;
    double q[NV], sig[N];
#pragma unroll
    for (int v = 0; v < N; ++v) {
      const double qm = box[v * MBOX + c - st], q0 = box[v * MBOX + c], qp = box[v * MBOX + c + st];
      sig[v] = minmod(SUB(P, q0, qm), SUB(P, qp, q0));
      q[v] = q0;
    }
#pragma unroll
    for (int v = N; v < NV; ++v) q[v] = box[v * MBOX + c];
#pragma unroll
    for (int sgn = 0; sgn < 2; ++sgn) {
      double* S = sgn == 0 ? sp : sm;
      if (!S) continue;
      const int idx = sgn == 0 ? ip : im;
      // +-1/2 from the kernel parameters: with a literal the compiler splits the FMA into
      // a product and a plain add
      const double h = sgn == 0 ? P.half : -P.half;
      double u[NV], W[NW > 0 ? NW : 1], F[N];
#pragma unroll
      for (int v = 0; v < N; ++v) u[v] = fma(h, sig[v], q[v]);
#pragma unroll
      for (int v = N; v < NV; ++v) u[v] = q[v];
      PDE::prims(u, P, W);
      PDE::flux(d, u, W, P, F);
#pragma unroll
      for (int v = 0; v < N; ++v) {
        S[v * MFS + idx] = F[v];
        S[(N + 1 + v) * MFS + idx] = u[v];
      }
      S[N * MFS + idx] = PDE::speed(d, u, W, P);
    }
  }

  // Twice the Rusanov flux of face f from its states SP[f] and SM[f]; the result
  // replaces the flux slots of SP[f] (no other face reads entry f).
  __device__ static void face(const DevParams& P, double* SP, const double* SM, int f) {
    const double s = max_nn(SP[N * MFS + f], SM[N * MFS + f]);
#pragma unroll
    for (int v = 0; v < N; ++v) {
      const double qL = SP[(N + 1 + v) * MFS + f], qR = SM[(N + 1 + v) * MFS + f];
      SP[v * MFS + f] = fma(-s, SUB(P, qR, qL), ADD(P, SP[v * MFS + f], SM[v * MFS + f]));
    }
  }

  __device__ static void run(const Fv2Args& A, const FdWork& w, double* smem, double& lam_thread) {
    double* box = smem;
    double* SP = smem + NV * MBOX;
    double* SM = SP + NS * MFS;
    const DevParams& P = A.P;
    const dh_patch pt = A.patches[w.patch];
    const int p = pt.p;
    const int t = threadIdx.x;
    const int tx = t % MX, ty = (t / MX) % MY, tz = t / (MX * MY);
    // -1/(2 dx): one IEEE division per CTA, shared (one voxel per thread would pay it per voxel)
    __shared__ double s_cL;
    if (t == 0) s_cL = -0.5 / pt.dx;
    // stage the tile and its two-voxel face halos
    for (int s = t; s < MSLOT; s += MNT) {
      int x, y, z;
      m_slot(s, x, y, z);
      const int64_t e = m_vox(A.patches, w.patch, p, w.x0 + x, w.y0 + y, w.z0 + z);
      const int c = mbox(x, y, z);
#pragma unroll
      for (int v = 0; v < N; ++v) box[v * MBOX + c] = __ldg(A.qs + (int64_t)v * A.vs + e);
#pragma unroll
      for (int v = 0; v < PDE::M; ++v) box[(N + v) * MBOX + c] = __ldg(A.mat + (int64_t)v * A.vs + e);
    }
    __syncthreads();
    const int me = mbox(tx, ty, tz);
    double sum[N];
#pragma unroll
    for (int v = 0; v < N; ++v) sum[v] = 0.0;
#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
      const int T = d == 0 ? MX : (d == 1 ? MY : MZ);
      const int area = MNT / T;
      const int st = d == 0 ? 1 : (d == 1 ? MBX : MBX * MBY);
      const int a = d == 0 ? tx : (d == 1 ? ty : tz);                          // along d
      const int o = d == 0 ? tz * MY + ty : (d == 1 ? tz * MX + tx : ty * MX + tx);  // across d
      // phase 1: own states; face f lies between voxels f-1 and f along d, so this
      // voxel's + state is the left state of face a+1 and its - state the right
      // state of face a.  Halo voxels next to the tile: the + state of the voxel
      // at -1 (left state of face 0) and the - state of the voxel at T (right
      // state of face T).
      states(A, box, me, st, d, SP, (a + 1) * area + o, SM, a * area + o);
      // (taken by the last warps along x and z and by warps 4 and 5 along y, so that the
      // extra work of x and y falls on different SM sub-partitions; the faces beyond 256
      // in phase 2 go to warp 0, or to warp 2 along y)
      const int ht = t - (d == 1 ? 4 * 32 : MNT - 2 * area);
      if (ht >= 0 && ht < 2 * area) {
        const int side = ht / area, oo = ht % area;
        int hx, hy, hz;
        if (d == 0) { hx = side == 0 ? -1 : MX; hy = oo % MY; hz = oo / MY; }
        else if (d == 1) { hy = side == 0 ? -1 : MY; hx = oo % MX; hz = oo / MX; }
        else { hz = side == 0 ? -1 : MZ; hx = oo % MX; hy = oo / MX; }
        const int c = mbox(hx, hy, hz);
        if (side == 0) states(A, box, c, st, d, SP, oo, nullptr, 0);
        else states(A, box, c, st, d, nullptr, 0, SM, T * area + oo);
      }
      __syncthreads();
      // phase 2: every face along d once ((T + 1) * area faces over the 256 threads)
      const int nf = (T + 1) * area;
      face(P, SP, SM, t);
      {
        const int fx = MNT + t - (d == 1 ? 2 * 32 : 0);
        if (fx >= MNT && fx < nf) face(P, SP, SM, fx);
      }
      __syncthreads();
      // phase 3: difference of this voxel's two faces
#pragma unroll
      for (int v = 0; v < N; ++v)
        sum[v] = ADD(P, sum[v], SUB(P, SP[v * MFS + (a + 1) * area + o], SP[v * MFS + a * area + o]));
      __syncthreads();
    }
    // update
    const double dt = *A.dt_dev;
    const double cL = s_cL;
    const double gdt = A.g * dt, ddt = A.d * dt;
    const bool b1 = A.b == 1.0;
    const int64_t e = pt.offset + ((int64_t)(w.z0 + tz) * p + (w.y0 + ty)) * p + (w.x0 + tx);
    double q[NV], Sv[N], res[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = box[v * MBOX + me];
    if (PDE::SRC) {
      double W[NW > 0 ? NW : 1];
      PDE::prims(q, P, W);
      PDE::source(q, W, P, Sv);
    }
#pragma unroll
    for (int v = 0; v < N; ++v) {
      const int64_t ev = (int64_t)v * A.vs + e;
      if (A.out) {
        double base = b1 ? q[v] : MUL(P, A.b, q[v]);
        if (A.q0) base = fma(A.a, __ldg(A.q0 + ev), base);
        res[v] = PDE::SRC ? fma(gdt, fma(cL, sum[v], Sv[v]), base) : fma(MUL(P, gdt, cL), sum[v], base);
      }
      if (A.acc) {
        const double r = PDE::SRC ? fma(ddt, fma(cL, sum[v], Sv[v]), A.acc[ev]) : fma(MUL(P, ddt, cL), sum[v], A.acc[ev]);
        A.acc[ev] = r;
        if (!A.out) res[v] = r;
      }
      if (A.out) A.out[ev] = res[v];
    }
    if (A.lam_out) {
#pragma unroll
      for (int v = N; v < NV; ++v) res[v] = q[v];
      double W[NW > 0 ? NW : 1];
      PDE::prims(res, P, W);
      const double l = max_nn(max_nn(PDE::speed(0, res, W, P), PDE::speed(1, res, W, P)), PDE::speed(2, res, W, P));
      lam_thread = max_nn(lam_thread, l);
    }
  }
};

__device__ void m_publish_lambda(double lam, double* lam_out, unsigned long long* red) {
  __shared__ double wmax[MNT / 32];
  __shared__ bool last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lam = max_nn(lam, __shfl_xor_sync(0xffffffffu, lam, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = lam;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < MNT / 32; ++i) m = max_nn(m, wmax[i]);
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

template <class PDE>
__global__ void __launch_bounds__(MNT, 2) k_fv2_stage(const __grid_constant__ Fv2Args A) {
  extern __shared__ __align__(16) double m_smem[];
  const FdWork w = A.work[blockIdx.x];
  double lam = 0.0;
  Fv2Tile<PDE>::run(A, w, m_smem, lam);
  if (A.lam_out) m_publish_lambda(lam, A.lam_out, A.red);
}

template <class PDE>
dh_status m_launch(dh_plan* plan, const Fv2Args& A, cudaStream_t s) {
  static int configured_device = -1;
  if (configured_device != plan->device) {
    cudaError_t e = cudaFuncSetAttribute(k_fv2_stage<PDE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Fv2Tile<PDE>::SMEM);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(k_fv2_stage)");
    configured_device = plan->device;
  }
  k_fv2_stage<PDE><<<plan->n_fdwork, MNT, Fv2Tile<PDE>::SMEM, s>>>(A);
  return cuda_error(cudaGetLastError(), "k_fv2_stage launch");
}

}  // namespace

dh_status launch_fv2_stage(dh_plan* plan, const double* qs, const double* q0, double* out, double* acc,
                           const double* mat, const double* dt_dev, double a, double b, double g, double d,
                           double* lam_out, cudaStream_t stream) {
  Fv2Args A;
  A.patches = plan->d_patches;
  A.work = plan->d_fdwork;
  A.qs = qs; A.q0 = q0; A.out = out; A.acc = acc; A.mat = mat; A.dt_dev = dt_dev;
  A.a = a; A.b = b; A.g = g; A.d = d;
  A.lam_out = lam_out;
  A.red = plan->d_red;
  A.vs = plan->var_stride;
  A.P = plan->params;
  switch (plan->pde) {
    case DH_PDE_ADV_FLUX: return m_launch<PdeAdvFlux>(plan, A, stream);
    case DH_PDE_EULER3D: return m_launch<PdeEuler3>(plan, A, stream);
    default:
      set_error("patch_update_fv_muscl: PDE %d not supported (conservative 3-D systems: ADV_FLUX, EULER3D)",
                plan->pde);
      return DH_EUNSUPPORTED;
  }
}

}  // namespace dh
