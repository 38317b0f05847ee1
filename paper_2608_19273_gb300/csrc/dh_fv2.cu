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

// Asynchronous 8-byte copy global -> shared (no register round trip) and the wait for all of
// this thread's copies.
__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

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
      // state slot of face j (along d) of line o: x faces line by line (consecutive threads,
      // which differ in x, then touch consecutive slots), y and z faces plane by plane (where
      // consecutive threads differ in o); every face's two states share one slot index
      auto slot = [&](int j, int oo) { return d == 0 ? oo * (MX + 1) + j : j * area + oo; };
      // phase 1: own states; face f lies between voxels f-1 and f along d, so this
      // voxel's + state is the left state of face a+1 and its - state the right
      // state of face a.  Halo voxels next to the tile: the + state of the voxel
      // at -1 (left state of face 0) and the - state of the voxel at T (right
      // state of face T).
      states(A, box, me, st, d, SP, slot(a + 1, o), SM, slot(a, o));
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
        if (side == 0) states(A, box, c, st, d, SP, slot(0, oo), nullptr, 0);
        else states(A, box, c, st, d, nullptr, 0, SM, slot(T, oo));
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
        sum[v] = ADD(P, sum[v], SUB(P, SP[v * MFS + slot(a + 1, o)], SP[v * MFS + slot(a, o)]));
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

// ------------------------------------------------------------- z-marching variant
// A CTA owns a (TX x TY) column of one patch (or four 8x8 columns of up to four 8^3 patches)
// and marches it through the patch's z-planes, one voxel per thread and plane:
//   * z: each thread keeps its column's states in registers -- the states of planes zk and
//     zk+1, the limited slope of plane zk and the z face below plane zk -- so every z slope,
//     z face state and z face flux is computed once (two extra states per column end);
//   * x, y: plane zk and a two-voxel ring around the column sit in a double-buffered plane
//     buffer in shared memory; each thread forms its x (then y) slope and its two face states,
//     keeps the + state in registers and publishes the - state; after a barrier it forms the
//     Rusanov flux of its + face from its own + state and its neighbour's - state; the ring
//     threads form the inward states of the voxels next to the column (the last warps, so the
//     extra work is whole warps);
//   * the ring of the next plane is loaded into registers at the top of an iteration and
//     stored into the other plane buffer at its end.
// Five barriers per plane.  Same arithmetic, in the same order, as the tile kernel: results
// agree bitwise.
template <class PDE, int TX, int TY, int G>
struct Fv2March {
  static constexpr int N = PDE::N, NV = PDE::N + PDE::M, NW = PDE::NW;
  static constexpr int NT = TX * TY * G;
  static_assert(NT == 256, "one voxel per thread and plane, 256 threads");
  static constexpr int R2 = 4 * TY + 4 * TX;           // ring slots per group: two deep on every side
  static constexpr int PS = NT + G * R2;                // plane-buffer slots
  static constexpr int RX = 2 * G * TY, RY = 2 * G * TX;  // ring voxels with a state per direction
  static constexpr int LM = TX > TY ? TX : TY;
  static constexpr int NS = NT + G * LM;                // faces: interior + one ring per group
  static constexpr int NSS = NS + G * LM;               // states: interior, ring after, ring before
  static constexpr int NST = 2 * N + 1;                 // a face state: F (N), lambda, u (N)
  static constexpr size_t SMEM = sizeof(double) * (2 * (size_t)NV * PS + (size_t)NST * NSS + (size_t)N * NS);

  __device__ static int xring(int g, int side, int h, int j) { return NT + g * R2 + (side * 2 + h) * TY + j; }
  __device__ static int yring(int g, int side, int h, int j) { return NT + g * R2 + 4 * TY + (side * 2 + h) * TX + j; }

  // Face state of q (N + M values) with slope sig along d at offset h (+-1/2): u, derived
  // quantities, flux F_d and speed.
  __device__ static void state(const DevParams& P, int d, const double* q, const double* sig, double h, double* F,
                               double& lam, double* u) {
    double W[NW > 0 ? NW : 1];
#pragma unroll
    for (int v = 0; v < N; ++v) u[v] = fma(h, sig[v], q[v]);
#pragma unroll
    for (int v = N; v < NV; ++v) u[v] = q[v];
    PDE::prims(u, P, W);
    PDE::flux(d, u, W, P, F);
    lam = PDE::speed(d, u, W, P);
  }
  __device__ static void publish(double* SS, int slot, const double* F, double lam, const double* u) {
#pragma unroll
    for (int v = 0; v < N; ++v) {
      SS[v * NSS + slot] = F[v];
      SS[(N + 1 + v) * NSS + slot] = u[v];
    }
    SS[N * NSS + slot] = lam;
  }
  // Twice the Rusanov flux from the left state (registers) and the published right state.
  __device__ static void face_lr(const DevParams& P, const double* FL, double lL, const double* uL, const double* SS,
                                 int slot, double* H) {
    const double s = max_nn(lL, SS[N * NSS + slot]);
#pragma unroll
    for (int v = 0; v < N; ++v)
      H[v] = fma(-s, SUB(P, SS[(N + 1 + v) * NSS + slot], uL[v]), ADD(P, FL[v], SS[v * NSS + slot]));
  }
  // Twice the Rusanov flux of two published states.
  __device__ static void face_ss(const DevParams& P, const double* SS, int ls, int rs, double* H) {
    const double s = max_nn(SS[N * NSS + ls], SS[N * NSS + rs]);
#pragma unroll
    for (int v = 0; v < N; ++v)
      H[v] = fma(-s, SUB(P, SS[(N + 1 + v) * NSS + rs], SS[(N + 1 + v) * NSS + ls]),
                 ADD(P, SS[v * NSS + ls], SS[v * NSS + rs]));
  }
  // Twice the Rusanov flux of two states in registers.
  __device__ static void face_rr(const DevParams& P, const double* FL, double lL, const double* uL, const double* FR,
                                 double lR, const double* uR, double* H) {
    const double s = max_nn(lL, lR);
#pragma unroll
    for (int v = 0; v < N; ++v) H[v] = fma(-s, SUB(P, uR[v], uL[v]), ADD(P, FL[v], FR[v]));
  }
  __device__ static void slope(const double* qm, const double* q0, const double* qp, const DevParams& P, double* sig) {
#pragma unroll
    for (int v = 0; v < N; ++v) sig[v] = minmod(SUB(P, q0[v], qm[v]), SUB(P, qp[v], q0[v]));
  }
  __device__ static void load(const Fv2Args& A, int64_t e, double* q) {
#pragma unroll
    for (int v = 0; v < N; ++v) q[v] = __ldg(A.qs + (int64_t)v * A.vs + e);
#pragma unroll
    for (int v = 0; v < PDE::M; ++v) q[N + v] = __ldg(A.mat + (int64_t)v * A.vs + e);
  }
  __device__ static void read_slot(const double* Qp, int slot, double* q) {
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = Qp[v * PS + slot];
  }
  // Ring slot r (t < G * R2) of plane z: its patch-relative position.
  __device__ static bool ring_pos(const Work& w, int r, int& g, int& x, int& y, int& slot) {
    g = r / R2;
    const int rr = r % R2;
    if (w.patch[g] < 0) return false;
    const int x0 = w.x0[g], y0 = w.y0[g];
    if (rr < 4 * TY) {
      const int side = rr / (2 * TY), h = (rr / TY) % 2, j = rr % TY;
      x = side == 0 ? x0 - 1 - h : x0 + TX + h;
      y = y0 + j;
      slot = xring(g, side, h, j);
    } else {
      const int r2 = rr - 4 * TY;
      const int side = r2 / (2 * TX), h = (r2 / TX) % 2, j = r2 % TX;
      x = x0 + j;
      y = side == 0 ? y0 - 1 - h : y0 + TY + h;
      slot = yring(g, side, h, j);
    }
    return true;
  }

  __device__ static void run(const Fv2Args& A, const Work& w, double* smem, double& lam_thread) {
    double* Qb[2] = {smem, smem + NV * PS};
    double* SS = smem + 2 * NV * PS;
    double* HS = SS + NST * NSS;
    const DevParams& P = A.P;
    const int t = threadIdx.x;
    const int g = t / (TX * TY), lxy = t % (TX * TY), lx = lxy % TX, ly = lxy / TX;
    const int k = w.patch[g];
    const bool act = k >= 0;
    const int kk = act ? k : w.patch[0];
    const dh_patch pt = A.patches[kk];
    const int p = pt.p, pz = w.pz, z0 = w.z0;
    const int x = (act ? w.x0[g] : 0) + lx, y = (act ? w.y0[g] : 0) + ly;
    const int own = t;
    __shared__ double s_cL;
    if (t == 0) s_cL = -0.5 / pt.dx;  // one IEEE division per CTA
    const bool ringt = t < G * R2;
    int rg = 0, rx_ = 0, ry_ = 0, rslot = 0;
    const bool rok = ringt && ring_pos(w, t, rg, rx_, ry_, rslot);
    // x / y ring states: the last warps
    const int hx = t - (NT - RX), hy = t - (NT - RX - RY);
    // ---- prologue: the column's planes z0-2 .. z0+1 and plane z0 with its ring
    double Qc[NV], Qn[NV], sc[N], Hzm[N];
    {
      double Qa[NV], Qb2[NV], sa[N];
      if (act) {
        load(A, m_vox(A.patches, k, p, x, y, z0 - 2), Qa);
        load(A, m_vox(A.patches, k, p, x, y, z0 - 1), Qb2);
        load(A, m_vox(A.patches, k, p, x, y, z0), Qc);
        load(A, m_vox(A.patches, k, p, x, y, z0 + 1), Qn);
        slope(Qa, Qb2, Qc, P, sa);
        slope(Qb2, Qc, Qn, P, sc);
        double FL[N], FR[N], uL[NV], uR[NV], lL, lR;
        state(P, 2, Qb2, sa, P.half, FL, lL, uL);
        state(P, 2, Qc, sc, -P.half, FR, lR, uR);
        face_rr(P, FL, lL, uL, FR, lR, uR, Hzm);
#pragma unroll
        for (int v = 0; v < NV; ++v) Qb[0][v * PS + own] = Qc[v];
      }
      if (rok) {
        double q[NV];
        load(A, m_vox(A.patches, w.patch[rg], p, rx_, ry_, z0), q);
#pragma unroll
        for (int v = 0; v < NV; ++v) Qb[0][v * PS + rslot] = q[v];
      }
    }
    __syncthreads();
    for (int kz = 0; kz < pz; ++kz) {
      const int zk = z0 + kz;
      const double* Qp = Qb[kz & 1];
      // next loads: the column's plane zk+2 into registers, and the ring of plane zk+1 straight
      // into the other plane buffer (asynchronous copies, waited for at the end of the iteration;
      // that buffer's last readers finished before the previous iteration's final barrier)
      double Qnn[NV];
      if (act) load(A, m_vox(A.patches, k, p, x, y, zk + 2), Qnn);
      const bool more = kz + 1 < pz;
      if (rok && more) {
        double* Qo = Qb[(kz + 1) & 1];
        const int64_t e = m_vox(A.patches, w.patch[rg], p, rx_, ry_, zk + 1);
#pragma unroll
        for (int v = 0; v < N; ++v) cp_async8(Qo + v * PS + rslot, A.qs + (int64_t)v * A.vs + e);
#pragma unroll
        for (int v = 0; v < PDE::M; ++v) cp_async8(Qo + (N + v) * PS + rslot, A.mat + (int64_t)v * A.vs + e);
      }
      double sum[N];
#pragma unroll
      for (int v = 0; v < N; ++v) sum[v] = 0.0;
#pragma unroll 1
      for (int d = 0; d < 2; ++d) {
        const int T = d == 0 ? TX : TY;
        const int a = d == 0 ? lx : ly;
        const int mslot = a > 0 ? own - (d == 0 ? 1 : TX) : (d == 0 ? xring(g, 0, 0, ly) : yring(g, 0, 0, lx));
        const int pslot = a < T - 1 ? own + (d == 0 ? 1 : TX) : (d == 0 ? xring(g, 1, 0, ly) : yring(g, 1, 0, lx));
        // phase 1: own slope and states (- published, + kept); ring voxels' inward states
        double FP[N], uP[NV], lP = 0.0;
        if (act) {
          double qm[NV], qp[NV], sig[N], FM[N], uM[NV], lM;
          read_slot(Qp, mslot, qm);
          read_slot(Qp, pslot, qp);
          slope(qm, Qc, qp, P, sig);
          state(P, d, Qc, sig, -P.half, FM, lM, uM);
          publish(SS, own, FM, lM, uM);
          state(P, d, Qc, sig, P.half, FP, lP, uP);
        }
        // ring: (hr < half) the voxel before the column (its + state and the face into the
        // column), (else) the voxel after it (its - state)
        const int hr = d == 0 ? hx : hy;
        const int RR = d == 0 ? RX : RY;
        const int LEN = d == 0 ? TY : TX;  // ring voxels per side and group
        int rgr = 0, rj = 0, rside = 0;
        bool ract = false;
        if (hr >= 0 && hr < RR) {
          rgr = hr / (2 * LEN);
          rside = (hr / LEN) % 2;
          rj = hr % LEN;
          ract = w.patch[rgr] >= 0;
          if (ract) {
            const int ci = rgr * TX * TY + (d == 0 ? rj * TX : rj);  // first interior voxel of the row / column
            const int ce = rgr * TX * TY + (d == 0 ? rj * TX + TX - 1 : (TY - 1) * TX + rj);  // last one
            double q0[NV], qa[NV], qb[NV], sig[N];
            if (rside == 0) {
              read_slot(Qp, d == 0 ? xring(rgr, 0, 1, rj) : yring(rgr, 0, 1, rj), qa);
              read_slot(Qp, d == 0 ? xring(rgr, 0, 0, rj) : yring(rgr, 0, 0, rj), q0);
              read_slot(Qp, ci, qb);
              slope(qa, q0, qb, P, sig);
              double FQ[N], uQ[NV], lQ;
              state(P, d, q0, sig, P.half, FQ, lQ, uQ);
              publish(SS, NS + rgr * LEN + rj, FQ, lQ, uQ);
            } else {
              read_slot(Qp, ce, qa);
              read_slot(Qp, d == 0 ? xring(rgr, 1, 0, rj) : yring(rgr, 1, 0, rj), q0);
              read_slot(Qp, d == 0 ? xring(rgr, 1, 1, rj) : yring(rgr, 1, 1, rj), qb);
              slope(qa, q0, qb, P, sig);
              double FM[N], uM[NV], lM;
              state(P, d, q0, sig, -P.half, FM, lM, uM);
              publish(SS, NT + rgr * LEN + rj, FM, lM, uM);
            }
          }
        }
        __syncthreads();
        // phase 2: the + face of every voxel (right state: the neighbour's - state); the face
        // into the column from the ring voxel before it
        if (act) {
          const int rs = a < T - 1 ? own + (d == 0 ? 1 : TX) : NT + g * LEN + (d == 0 ? ly : lx);
          double Hown[N];
          face_lr(P, FP, lP, uP, SS, rs, Hown);
#pragma unroll
          for (int v = 0; v < N; ++v) HS[v * NS + own] = Hown[v];
        }
        if (ract && rside == 0) {
          const int ci = rgr * TX * TY + (d == 0 ? rj * TX : rj);
          double Hb[N];
          face_ss(P, SS, NS + rgr * LEN + rj, ci, Hb);
#pragma unroll
          for (int v = 0; v < N; ++v) HS[v * NS + NT + rgr * LEN + rj] = Hb[v];
        }
        __syncthreads();
        // phase 3: difference of this voxel's two faces along d
        if (act) {
          const int ms = a > 0 ? own - (d == 0 ? 1 : TX) : NT + g * LEN + (d == 0 ? ly : lx);
#pragma unroll
          for (int v = 0; v < N; ++v) sum[v] = ADD(P, sum[v], SUB(P, HS[v * NS + own], HS[v * NS + ms]));
        }
      }
      if (act) {
        // z: slope of plane zk+1, the states on both sides of the face zk+1/2 and its flux
        double sn[N], Hzp[N];
        slope(Qc, Qn, Qnn, P, sn);
        {
          double FL[N], FR[N], uL[NV], uR[NV], lL, lR;
          state(P, 2, Qc, sc, P.half, FL, lL, uL);
          state(P, 2, Qn, sn, -P.half, FR, lR, uR);
          face_rr(P, FL, lL, uL, FR, lR, uR, Hzp);
        }
#pragma unroll
        for (int v = 0; v < N; ++v) sum[v] = ADD(P, sum[v], SUB(P, Hzp[v], Hzm[v]));
        // update of plane zk
        const double dt = *A.dt_dev;
        const double cL = s_cL;
        const double gdt = A.g * dt, ddt = A.d * dt;
        const bool b1 = A.b == 1.0;
        const int64_t e = pt.offset + ((int64_t)zk * p + y) * p + x;
        double Sv[N], res[NV];
        if (PDE::SRC) {
          double W[NW > 0 ? NW : 1];
          PDE::prims(Qc, P, W);
          PDE::source(Qc, W, P, Sv);
        }
        const dh_patch& mp = A.patches[k];
        const int64_t ek = mp.offset + ((int64_t)zk * p + y) * p + x;
        (void)e;
#pragma unroll
        for (int v = 0; v < N; ++v) {
          const int64_t ev = (int64_t)v * A.vs + ek;
          if (A.out) {
            double base = b1 ? Qc[v] : MUL(P, A.b, Qc[v]);
            if (A.q0) base = fma(A.a, __ldg(A.q0 + ev), base);
            res[v] = PDE::SRC ? fma(gdt, fma(cL, sum[v], Sv[v]), base) : fma(MUL(P, gdt, cL), sum[v], base);
          }
          if (A.acc) {
            const double r = PDE::SRC ? fma(ddt, fma(cL, sum[v], Sv[v]), A.acc[ev])
                                      : fma(MUL(P, ddt, cL), sum[v], A.acc[ev]);
            A.acc[ev] = r;
            if (!A.out) res[v] = r;
          }
          if (A.out) A.out[ev] = res[v];
        }
        if (A.lam_out) {
#pragma unroll
          for (int v = N; v < NV; ++v) res[v] = Qc[v];
          double W[NW > 0 ? NW : 1];
          PDE::prims(res, P, W);
          const double l = max_nn(max_nn(PDE::speed(0, res, W, P), PDE::speed(1, res, W, P)), PDE::speed(2, res, W, P));
          lam_thread = max_nn(lam_thread, l);
        }
        // march one plane on
#pragma unroll
        for (int v = 0; v < NV; ++v) { Qc[v] = Qn[v]; Qn[v] = Qnn[v]; }
#pragma unroll
        for (int v = 0; v < N; ++v) { sc[v] = sn[v]; Hzm[v] = Hzp[v]; }
      }
      if (more) {
        double* Qo = Qb[(kz + 1) & 1];
        if (act) {
#pragma unroll
          for (int v = 0; v < NV; ++v) Qo[v * PS + own] = Qc[v];
        }
        cp_async_wait_all();
        __syncthreads();
      }
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
__global__ void __launch_bounds__(256, 2) k_fv2_march(const __grid_constant__ Fv2Args A, const Work* work) {
  extern __shared__ __align__(16) double m_smem[];
  const Work w = work[blockIdx.x];
  double lam = 0.0;
  if (w.cls == 0) Fv2March<PDE, 16, 16, 1>::run(A, w, m_smem, lam);
  else Fv2March<PDE, 8, 8, 4>::run(A, w, m_smem, lam);
  if (A.lam_out) m_publish_lambda(lam, A.lam_out, A.red);
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
dh_status m_launch_march(dh_plan* plan, const Fv2Args& A, cudaStream_t s) {
  // the FV work lists of tile set 0: 16x16 columns, four 8x8 columns of 8^3 patches (zs: z-chunks)
  const int li = (plan->fv2_var & 1) ? 1 : 0;
  const bool* cls = plan->wl_cls[li];
  const size_t smem = std::max(cls[0] ? Fv2March<PDE, 16, 16, 1>::SMEM : (size_t)0,
                               cls[1] ? Fv2March<PDE, 8, 8, 4>::SMEM : (size_t)0);
  static int configured_device = -1;
  if (configured_device != plan->device) {
    cudaError_t e = cudaFuncSetAttribute(k_fv2_march<PDE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)std::max(Fv2March<PDE, 16, 16, 1>::SMEM, Fv2March<PDE, 8, 8, 4>::SMEM));
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(k_fv2_march)");
    configured_device = plan->device;
  }
  if (plan->n_wl[li] <= 0) return DH_OK;
  k_fv2_march<PDE><<<plan->n_wl[li], 256, smem, s>>>(A, plan->d_wl[li]);
  return cuda_error(cudaGetLastError(), "k_fv2_march launch");
}

template <class PDE>
dh_status m_launch(dh_plan* plan, const Fv2Args& A, cudaStream_t s) {
  if (plan->fv2_var != 2) return m_launch_march<PDE>(plan, A, s);
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
