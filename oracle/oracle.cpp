// Oracle: plain, slow, FP64 CPU implementation of the batched explicit patch
// update for  dQ/dt + div F(Q) + B(Q) . grad Q = S(Q)   (Eq. 1).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
// only the tests, the smoke check and the CPU-baseline leg of the benchmark
// use it.  It shares no code, header, table or helper with the CUDA library.
//
// What it computes (paper Sec. II, Eq. 2-4):
//   * Eq. 2: a cell (patch) kernel maps p^d voxels plus a halo of width h
//     (p_hat = p + 2h) holding N evolved and M material quantities to the
//     p^d x N updated quantities.  K patches are advanced together (the
//     batched kernel K~_{dt,K}).
//   * Eq. 3: the update is a composition of steps: source per voxel, the
//     face fluxes (reconstruct Q on both sides of a face, evaluate F), and
//     the final combination into the new state.
//   * Sec. II-B: each patch is an AoS block (all N+M quantities of a voxel
//     contiguous).  The oracle works on exactly that layout: it gathers every
//     patch, with its halo, from the SoA arena used at the library boundary
//     into an AoS block (the gather prologue of Eq. 4), updates it with plain
//     loops, one temporary array per step, and scatters the interior back.
//
// Readings where the paper is silent:
//   * FV face flux: Rusanov, F^ = (F(QL)+F(QR))/2 - s/2 (QR-QL), with
//     s = max(lambda_n(QL), lambda_n(QR)).
//   * Non-conservative product: path-conservative, straight-line path,
//     midpoint rule: D = B_n((QL+QR)/2) (QR-QL), half to each side.
//   * FD: 4th-order centred first derivative and 6th-difference
//     Kreiss-Oliger dissipation sigma/(64 dx) delta^6 Q.
//   * Stage form: out = a Q0 + b Qs + g dt L(Qs); acc += d dt L(Qs).
//   * CFL: dt = CFL dx / (dim lambda_max).
//
// Parity of the GW59 system with true CCZ4 is unpinned: the paper gives no
// CCZ4 equations; GW59 is a defined 59-unknown stand-in with the same
// structure (F = 0, B(Q).grad Q, nonlinear source).
//
// All arithmetic is written as templates over the scalar type T so that a
// counting build (T = Counted) can report the exact number of FP64
// operations the method performs per voxel (add, sub, mul, div, sqrt count 1;
// min, max, abs count 0).  Compile with -ffp-contract=off.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#include <limits>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- scalar types
static thread_local long long g_flops = 0;

struct Counted {
  double v;
  Counted() : v(0) {}
  Counted(double x) : v(x) {}
};
inline Counted operator+(Counted a, Counted b) { ++g_flops; return Counted(a.v + b.v); }
inline Counted operator-(Counted a, Counted b) { ++g_flops; return Counted(a.v - b.v); }
inline Counted operator*(Counted a, Counted b) { ++g_flops; return Counted(a.v * b.v); }
inline Counted operator/(Counted a, Counted b) { ++g_flops; return Counted(a.v / b.v); }
inline Counted operator-(Counted a) { return Counted(-a.v); }
inline Counted& operator+=(Counted& a, Counted b) { a = a + b; return a; }
inline Counted& operator-=(Counted& a, Counted b) { a = a - b; return a; }
inline bool operator<(Counted a, Counted b) { return a.v < b.v; }
inline bool operator>(Counted a, Counted b) { return a.v > b.v; }
inline bool operator<=(Counted a, Counted b) { return a.v <= b.v; }
inline bool operator>=(Counted a, Counted b) { return a.v >= b.v; }
inline Counted sqrt(Counted a) { ++g_flops; return Counted(std::sqrt(a.v)); }
inline Counted fabs(Counted a) { return Counted(std::fabs(a.v)); }
inline Counted fmax(Counted a, Counted b) { return Counted(std::fmax(a.v, b.v)); }
inline double val(Counted a) { return a.v; }
inline double val(double a) { return a; }

using std::sqrt;
using std::fabs;
using std::fmax;

// ---------------------------------------------------------------- patch table
// Same field order as the library's patch descriptor (interface, not code).
struct Patch {
  int32_t p;        // voxels per patch per dimension
  int32_t level;    // refinement level (informational)
  double dx;        // voxel spacing
  double x0[3];     // lower corner of the patch
  int64_t offset;   // element offset of the patch's block in the SoA arena
  int32_t nbr[6];   // face neighbours -x,+x,-y,+y,-z,+z (periodic wrap done by caller)
};
static_assert(sizeof(Patch) == 72, "patch descriptor layout");

// ---------------------------------------------------------------- PDE systems
enum Pde { ADV_FLUX = 0, ADV_NCP = 1, EULER2D = 2, EULER3D = 3, WAVE3D = 4, SRHD3D = 5, GW59 = 6 };

struct PdeInfo { int N, M, dim; bool flux, ncp, source; };

PdeInfo pde_info(int pde) {
  switch (pde) {
    case ADV_FLUX: return {1, 3, 0, true, false, false};
    case ADV_NCP: return {1, 3, 0, false, true, false};
    case EULER2D: return {4, 0, 2, true, false, false};
    case EULER3D: return {5, 0, 3, true, false, false};
    case WAVE3D: return {5, 1, 3, false, true, true};
    case SRHD3D: return {5, 5, 3, true, false, false};
    case GW59: return {59, 0, 3, false, true, true};
  }
  return {0, 0, 0, false, false, false};
}

// PDE parameters; defaults follow the workloads (gamma = 1.4 for Euler,
// Gamma = 5/3 for SRHD, damping 0.1 for the wave system, kappa = 0.1 and
// an 11x11 coupling matrix for GW59).
struct Params {
  double gamma = 1.4;        // Euler ratio of specific heats
  double Gamma = 5.0 / 3.0;  // SRHD adiabatic index
  double damp = 0.1;         // wave-system damping gamma
  double kappa = 0.1;        // GW59 lapse coupling
  double C[121] = {0};       // GW59 coupling matrix C_ab
};

Params make_params(int pde, const double* prm, int nprm) {
  Params P;
  if (!prm) return P;
  if (pde == EULER2D || pde == EULER3D) { if (nprm >= 1) P.gamma = prm[0]; }
  if (pde == SRHD3D) { if (nprm >= 1) P.Gamma = prm[0]; }
  if (pde == WAVE3D) { if (nprm >= 1) P.damp = prm[0]; }
  if (pde == GW59) {
    if (nprm >= 1) P.kappa = prm[0];
    for (int i = 0; i < 121 && 1 + i < nprm; ++i) P.C[i] = prm[1 + i];
  }
  return P;
}

const int MAXW = 8;  // per-voxel derived quantities

// Per-voxel derived quantities W (computed once per voxel).
//   Euler: W = (u_0, u_1, [u_2], p, c)    from rho, momentum, energy.
//   SRHD : W = (v_x, v_y, v_z, p, cs2, v2) from the supplied primitives.
template <class T>
void prims(int pde, const Params& P, const T* q, const T* m, T* W) {
  if (pde == EULER2D || pde == EULER3D) {
    int d = (pde == EULER2D) ? 2 : 3;
    T rho = q[0];
    T E = q[d + 1];
    T kin = T(0.0);
    for (int k = 0; k < d; ++k) {
      W[k] = q[1 + k] / rho;
      kin = kin + q[1 + k] * W[k];
    }
    T p = (T(P.gamma) - T(1.0)) * (E - T(0.5) * kin);
    W[d] = p;
    W[d + 1] = sqrt(T(P.gamma) * p / rho);
  } else if (pde == SRHD3D) {
    // m = (rho, vx, vy, vz, p): primitives recovered by con2prim.
    T rho = m[0], p = m[4];
    T v2 = m[1] * m[1] + m[2] * m[2] + m[3] * m[3];
    T rhoh = rho + T(P.Gamma) * p / (T(P.Gamma) - T(1.0));
    W[0] = m[1]; W[1] = m[2]; W[2] = m[3]; W[3] = p;
    W[4] = T(P.Gamma) * p / rhoh;  // cs^2 = Gamma p / (rho h)
    W[5] = v2;
  }
  (void)q;
}

// Physical flux F_d(Q) (Eq. 1, conservative part).
template <class T>
void flux(int pde, const Params& P, int d, const T* q, const T* m, const T* W, T* F) {
  switch (pde) {
    case ADV_FLUX:
      F[0] = m[d] * q[0];
      break;
    case EULER2D:
    case EULER3D: {
      int nd = (pde == EULER2D) ? 2 : 3;
      T u = W[d], p = W[nd];
      F[0] = q[1 + d];
      for (int k = 0; k < nd; ++k) F[1 + k] = q[1 + k] * u;
      F[1 + d] = F[1 + d] + p;
      F[nd + 1] = (q[nd + 1] + p) * u;
      break;
    }
    case SRHD3D: {
      // (D v_d, S_x v_d + p delta, S_y v_d, S_z v_d, S_d - D v_d)
      T v = W[d], p = W[3];
      F[0] = q[0] * v;
      for (int k = 0; k < 3; ++k) F[1 + k] = q[1 + k] * v;
      F[1 + d] = F[1 + d] + p;
      F[4] = q[1 + d] - q[0] * v;
      break;
    }
    default:
      break;
  }
  (void)P;
}

// Largest characteristic speed |lambda| in direction d.
template <class T>
T speed(int pde, const Params& P, int d, const T* q, const T* m, const T* W) {
  switch (pde) {
    case ADV_FLUX:
    case ADV_NCP:
      return fabs(m[d]);
    case EULER2D:
    case EULER3D: {
      int nd = (pde == EULER2D) ? 2 : 3;
      return fabs(W[d]) + W[nd + 1];
    }
    case WAVE3D:
      return m[0];
    case SRHD3D: {
      // lambda_pm = [v_d (1 - cs2) +- cs sqrt((1 - v2)(1 - v2 cs2 - v_d^2 (1 - cs2)))] / (1 - v2 cs2)
      T vd = W[d], cs2 = W[4], v2 = W[5];
      T one = T(1.0);
      T cs = sqrt(cs2);
      T den = one - v2 * cs2;
      T a = vd * (one - cs2);
      T r = cs * sqrt((one - v2) * (one - v2 * cs2 - vd * vd * (one - cs2)));
      T lp = (a + r) / den, lm = (a - r) / den;
      return fmax(fabs(lp), fabs(lm));
    }
    case GW59:
      // alpha + |beta^d|
      return q[55] + fabs(q[56 + d]);
  }
  return T(0.0);
  (void)P;
}

// Non-conservative product B_d(Qb) . dQ (Qb carries N+M entries, dQ N).
template <class T>
void ncp(int pde, const Params& P, int d, const T* qb, const T* dq, T* out) {
  (void)P;
  switch (pde) {
    case ADV_NCP: {
      out[0] = qb[1 + d] * dq[0];  // material a_d sits after the single evolved unknown
      break;
    }
    case WAVE3D: {
      // Q = (phi, Pi, psi_x, psi_y, psi_z), material c.
      // Row Pi: -c^2 dpsi_d ; row psi_d: -dPi ; other rows 0.
      T c = qb[5];
      for (int k = 0; k < 5; ++k) out[k] = T(0.0);
      out[1] = -(c * c * dq[2 + d]);
      out[2 + d] = -dq[1];
      break;
    }
    case GW59: {
      T alpha = qb[55], beta = qb[56 + d];
      for (int k = 0; k < 59; ++k) out[k] = T(0.0);
      for (int a = 0; a < 11; ++a) {
        const int o = 5 * a;
        // Pi_a:  -alpha dpsi_{a,d} - beta^d dPi_a
        out[o + 1] = -(alpha * dq[o + 2 + d]) - beta * dq[o + 1];
        // psi_{a,i}: -beta^d dpsi_{a,i}; for i = d also -alpha dPi_a - Pi_a dalpha
        for (int i = 0; i < 3; ++i) out[o + 2 + i] = -(beta * dq[o + 2 + i]);
        out[o + 2 + d] = out[o + 2 + d] - alpha * dq[o + 1] - qb[o + 1] * dq[55];
      }
      break;
    }
    default:
      break;
  }
}

// Whether the non-conservative product in direction d reads dQ_v/dx_d, i.e.
// whether column v of B_d is non-zero (only those derivatives are computed).
bool needs_grad(int pde, int d, int v) {
  switch (pde) {
    case ADV_NCP: return v == 0;
    case WAVE3D: return v == 1 || v == 2 + d;
    case GW59: return v == 55 || (v < 55 && v % 5 != 0);  // Pi_a, psi_a, alpha
  }
  return false;
}

// Source S(Q).
template <class T>
void source(int pde, const Params& P, const T* q, const T* m, T* S) {
  (void)m;
  switch (pde) {
    case WAVE3D:
      S[0] = q[1];
      S[1] = -(T(P.damp) * q[1]);
      S[2] = T(0.0); S[3] = T(0.0); S[4] = T(0.0);
      break;
    case GW59: {
      T alpha = q[55];
      T sumPi2 = T(0.0);
      T bsum[3] = {T(0.0), T(0.0), T(0.0)};
      for (int a = 0; a < 11; ++a) {
        const int o = 5 * a;
        T Pi = q[o + 1];
        // dphi_a/dt = alpha Pi_a + beta^k psi_{a,k}
        S[o] = alpha * Pi + (q[56] * q[o + 2] + q[57] * q[o + 3] + q[58] * q[o + 4]);
        // dPi_a/dt source: alpha sum_b C_ab phi_b Pi_b
        T cs = T(0.0);
        for (int b = 0; b < 11; ++b) cs = cs + T(P.C[11 * a + b]) * (q[5 * b] * q[5 * b + 1]);
        S[o + 1] = alpha * cs;
        S[o + 2] = T(0.0); S[o + 3] = T(0.0); S[o + 4] = T(0.0);
        sumPi2 = sumPi2 + Pi * Pi;
        for (int i = 0; i < 3; ++i) bsum[i] = bsum[i] + q[o + 2 + i] * Pi;
      }
      S[55] = -(alpha * alpha * sumPi2 * T(P.kappa));
      for (int i = 0; i < 3; ++i) S[56 + i] = T(0.75) * bsum[i];
      break;
    }
    default:
      break;
  }
}

// ---------------------------------------------------------------- coarse-fine coupling
// Meshes of several refinement levels (the paper's meshes are Peano spacetrees,
// Sec. IV; it defines no coupling).  Reading used: refinement ratio 2, every
// patch of level l+1 covers one octant of a patch of level l (its parent),
// same p, half the voxel spacing; a patch's face neighbour is either of its own
// level or one level coarser.
//   * Prolongation: a halo voxel taken from a coarser neighbour gets the value
//     of the coarse voxel that contains it (piecewise constant).
//   * Reflux: the first-order FV update of a coarse voxel next to the finer
//     level uses, on that face, the mean of the 2^(d-1) fine face fluxes
//     instead of its own coarse face flux (conservation across levels).
//   * Restriction: after every stage each coarse voxel covered by the finer
//     level becomes the mean of its 2^d fine voxels (out and acc).
// Lattice index of a patch along axis a at its own level, and its octant bit.
inline int lattice(const Patch& P, int a) { return (int)std::llround(P.x0[a] / (P.p * P.dx)); }
inline int octant(const Patch& P, int a) { return lattice(P, a) & 1; }

inline bool coupled_mesh(const Patch* patches, int K, int dim) {
  for (int k = 0; k < K; ++k)
    for (int f = 0; f < 2 * dim; ++f)
      if (patches[patches[k].nbr[f]].level < patches[k].level) return true;
  return false;
}

// Parent of every patch (-1 on the coarsest level): the patch one level coarser
// whose lattice cell contains it.
std::vector<int> parents(const Patch* patches, int K, int dim) {
  std::vector<int> par(K, -1);
  for (int k = 0; k < K; ++k) {
    if (patches[k].level == 0) continue;
    for (int c = 0; c < K; ++c) {
      if (patches[c].level != patches[k].level - 1) continue;
      bool in = true;
      for (int a = 0; a < dim; ++a) in = in && lattice(patches[c], a) == lattice(patches[k], a) / 2;
      if (in) { par[k] = c; break; }
    }
  }
  return par;
}

// ---------------------------------------------------------------- patch gather
// A patch with halo as the paper's AoS block: voxel (x,y,z), x,y,z in
// [-h, p+h) (z only in 3D), all N+M quantities contiguous.  Halo voxels on a
// face come from the face neighbour; edges and corners are never read by the
// axis-aligned stencils and are filled with NaN so that any use shows up.
template <class T>
struct Block {
  int p, h, dim, nv, P, Pz;
  std::vector<T> U;
  int idx(int x, int y, int z) const {
    int zz = (dim == 3) ? z + h : 0;
    return ((zz * P) + (y + h)) * P + (x + h);
  }
  T* at(int x, int y, int z) { return &U[(size_t)idx(x, y, z) * nv]; }
};

template <class T>
void gather_block(Block<T>& B, const Patch* patches, int k, int dim, int h, int N, int M,
                  int64_t var_stride, const double* q, const double* mat) {
  const Patch& pt = patches[k];
  const int p = pt.p;
  B.p = p; B.h = h; B.dim = dim; B.nv = N + M; B.P = p + 2 * h; B.Pz = (dim == 3) ? p + 2 * h : 1;
  B.U.assign((size_t)B.P * B.P * B.Pz * B.nv, T(std::numeric_limits<double>::quiet_NaN()));
  const int zlo = (dim == 3) ? -h : 0, zhi = (dim == 3) ? p + h : 1;
  for (int z = zlo; z < zhi; ++z)
    for (int y = -h; y < p + h; ++y)
      for (int x = -h; x < p + h; ++x) {
        int c[3] = {x, y, z};
        int outside = 0, dir = -1;
        for (int a = 0; a < dim; ++a)
          if (c[a] < 0 || c[a] >= p) { ++outside; dir = a; }
        if (outside > 1) continue;  // edge/corner: stays NaN
        int src = k;
        int s[3] = {x, y, z};
        if (outside == 1) {
          src = c[dir] < 0 ? pt.nbr[2 * dir] : pt.nbr[2 * dir + 1];
          if (patches[src].level < pt.level) {
            // coarser neighbour: the coarse voxel containing this halo voxel
            for (int a = 0; a < dim; ++a) {
              const int fc = c[a];
              if (a == dir) s[a] = fc < 0 ? p + (int)std::floor(fc / 2.0) : (int)std::floor((fc - p) / 2.0);
              else s[a] = octant(pt, a) * (p / 2) + fc / 2;
            }
          } else {
            s[dir] += c[dir] < 0 ? p : -p;
          }
        }
        const Patch& ps = patches[src];
        int64_t e = ps.offset + ((int64_t)(dim == 3 ? s[2] : 0) * p + s[1]) * p + s[0];
        T* u = B.at(x, y, z);
        for (int v = 0; v < N; ++v) u[v] = T(q[v * var_stride + e]);
        for (int v = 0; v < M; ++v) u[N + v] = T(mat[v * var_stride + e]);
      }
}

// ---------------------------------------------------------------- FV operator
// L(Q)_i = -(1/dx) sum_d [F^_{i+1/2} - F^_{i-1/2} + (D_{i+1/2} + D_{i-1/2})/2] + S(Q_i)
template <class T>
void fv_operator(int pde, const Params& P, Block<T>& B, double dxd, std::vector<T>& L) {
  const PdeInfo I = pde_info(pde);
  const int N = I.N, p = B.p, dim = B.dim, nv = B.nv;
  const int pz = (dim == 3) ? p : 1;
  const T dx = T(dxd);
  const size_t nvox = (size_t)p * p * pz;
  L.assign(nvox * N, T(0.0));

  // Step: derived quantities W for every voxel that is interior or on a face halo.
  std::vector<T> W((size_t)B.P * B.P * B.Pz * MAXW, T(0.0));
  const int zlo = (dim == 3) ? -1 : 0, zhi = (dim == 3) ? p + 1 : 1;
  for (int z = zlo; z < zhi; ++z)
    for (int y = -1; y < p + 1; ++y)
      for (int x = -1; x < p + 1; ++x) {
        int c[3] = {x, y, z}, outside = 0;
        for (int a = 0; a < dim; ++a) if (c[a] < 0 || c[a] >= p) ++outside;
        if (outside > 1) continue;
        T* u = B.at(x, y, z);
        prims(pde, P, u, u + N, &W[(size_t)B.idx(x, y, z) * MAXW]);
      }

  std::vector<T> sum(nvox * N, T(0.0));  // sum_d [F^+ - F^- + (D^+ + D^-)/2]
  std::vector<T> Fv, Lam, Fh, Dh;
  for (int d = 0; d < dim; ++d) {
    // Step: F_d and lambda_d per voxel along the line, one halo voxel each side.
    const int n1 = p + 2;  // voxels -1..p along d
    const size_t lines = (size_t)p * pz;  // lines orthogonal to d
    Fv.assign(lines * n1 * N, T(0.0));
    Lam.assign(lines * n1, T(0.0));
    Fh.assign(lines * (p + 1) * N, T(0.0));
    Dh.assign(lines * (p + 1) * N, T(0.0));
    auto coord = [&](size_t line, int i, int* c) {
      // line indexes the two coordinates other than d (in increasing axis order)
      int o[2] = {(int)(line % p), (int)(line / p)};
      int j = 0;
      for (int a = 0; a < 3; ++a) {
        if (a == d) c[a] = i;
        else if (a < dim) c[a] = o[j++];
        else c[a] = 0;
      }
    };
    for (size_t ln = 0; ln < lines; ++ln)
      for (int i = -1; i <= p; ++i) {
        int c[3]; coord(ln, i, c);
        T* u = B.at(c[0], c[1], c[2]);
        const T* w = &W[(size_t)B.idx(c[0], c[1], c[2]) * MAXW];
        if (I.flux) flux(pde, P, d, u, u + N, w, &Fv[(ln * n1 + (i + 1)) * N]);
        Lam[ln * n1 + (i + 1)] = speed(pde, P, d, u, u + N, w);
      }
    // Step: face values.  Face f (0..p) lies between voxel f-1 (left) and f (right).
    std::vector<T> qb(nv), dq(N);
    for (size_t ln = 0; ln < lines; ++ln)
      for (int f = 0; f <= p; ++f) {
        int cl[3], cr[3]; coord(ln, f - 1, cl); coord(ln, f, cr);
        const T* QL = B.at(cl[0], cl[1], cl[2]);
        const T* QR = B.at(cr[0], cr[1], cr[2]);
        const T* FL = &Fv[(ln * n1 + f) * N];
        const T* FR = &Fv[(ln * n1 + f + 1) * N];
        T s = fmax(Lam[ln * n1 + f], Lam[ln * n1 + f + 1]);
        T hs = T(0.5) * s;
        T* fh = &Fh[(ln * (p + 1) + f) * N];
        for (int v = 0; v < N; ++v) {
          if (I.flux) fh[v] = T(0.5) * (FL[v] + FR[v]) - hs * (QR[v] - QL[v]);
          else fh[v] = -(hs * (QR[v] - QL[v]));
        }
        if (I.ncp) {
          for (int v = 0; v < nv; ++v) qb[v] = T(0.5) * (QL[v] + QR[v]);
          for (int v = 0; v < N; ++v) dq[v] = QR[v] - QL[v];
          ncp(pde, P, d, qb.data(), dq.data(), &Dh[(ln * (p + 1) + f) * N]);
        }
      }
    // Step: accumulate the face differences of direction d into every voxel.
    for (size_t ln = 0; ln < lines; ++ln)
      for (int i = 0; i < p; ++i) {
        int c[3]; coord(ln, i, c);
        size_t vox = ((size_t)c[2] * p + c[1]) * p + c[0];
        const T* fm = &Fh[(ln * (p + 1) + i) * N];
        const T* fp = &Fh[(ln * (p + 1) + i + 1) * N];
        const T* dm = &Dh[(ln * (p + 1) + i) * N];
        const T* dp = &Dh[(ln * (p + 1) + i + 1) * N];
        for (int v = 0; v < N; ++v) {
          T term = fp[v] - fm[v];
          if (I.ncp) term = term + T(0.5) * (dp[v] + dm[v]);
          sum[vox * N + v] = sum[vox * N + v] + term;
        }
      }
  }
  // Step: assemble L = -(1/dx) sum + S.
  const T mrdx = -(T(1.0) / dx);
  std::vector<T> S(N);
  for (int z = 0; z < pz; ++z)
    for (int y = 0; y < p; ++y)
      for (int x = 0; x < p; ++x) {
        size_t vox = ((size_t)z * p + y) * p + x;
        T* u = B.at(x, y, z);
        if (I.source) source(pde, P, u, u + N, S.data());
        for (int v = 0; v < N; ++v) {
          T l = mrdx * sum[vox * N + v];
          if (I.source) l = l + S[v];
          L[vox * N + v] = l;
        }
      }
}

// ---------------------------------------------------------------- FV operator, MUSCL
// Second-order variant of the face step of Eq. 3 (Sec. II-A builds each face
// state from the voxels beside the face with a linear stencil), read as
// piecewise-linear (MUSCL) reconstruction of the evolved quantities, one
// component at a time, with the minmod slope limiter:
//   sigma_i = minmod(Q_i - Q_{i-1}, Q_{i+1} - Q_i),
//   minmod(a, b) = min(a, b) if a > 0 and b > 0, max(a, b) if a < 0 and b < 0, else 0,
//   face f between voxels f-1 and f:  QL = Q_{f-1} + sigma_{f-1}/2,  QR = Q_f - sigma_f/2,
// then the same Rusanov flux on (QL, QR):
//   F^ = (F_d(QL) + F_d(QR))/2 - s/2 (QR - QL),  s = max(lambda_d(QL), lambda_d(QR)),
//   L(Q)_i = -(1/dx) sum_d [F^_{i+1/2} - F^_{i-1/2}] + S(Q_i).
// Material parameters of a face state are those of the voxel it was
// reconstructed from.  Conservative systems only (B = 0); halo width 2.
template <class T>
T minmod(T a, T b) {
  if (a > T(0.0) && b > T(0.0)) return a < b ? a : b;
  if (a < T(0.0) && b < T(0.0)) return a > b ? a : b;
  return T(0.0);
}

template <class T>
void fv2_operator(int pde, const Params& P, Block<T>& B, double dxd, std::vector<T>& L) {
  const PdeInfo I = pde_info(pde);
  const int N = I.N, M = I.M, p = B.p, dim = B.dim;
  const int pz = (dim == 3) ? p : 1;
  const T dx = T(dxd);
  const size_t nvox = (size_t)p * p * pz;
  L.assign(nvox * N, T(0.0));
  std::vector<T> sum(nvox * N, T(0.0));
  std::vector<T> sig, Fh;
  for (int d = 0; d < dim; ++d) {
    const size_t lines = (size_t)p * pz;
    auto coord = [&](size_t line, int i, int* c) {
      int o[2] = {(int)(line % p), (int)(line / p)};
      int j = 0;
      for (int a = 0; a < 3; ++a) {
        if (a == d) c[a] = i;
        else if (a < dim) c[a] = o[j++];
        else c[a] = 0;
      }
    };
    // Step: limited slopes of voxels -1..p along each line.
    const int ns = p + 2;
    sig.assign(lines * ns * N, T(0.0));
    for (size_t ln = 0; ln < lines; ++ln)
      for (int i = -1; i <= p; ++i) {
        int cm[3], c0[3], cp[3];
        coord(ln, i - 1, cm); coord(ln, i, c0); coord(ln, i + 1, cp);
        const T* qm = B.at(cm[0], cm[1], cm[2]);
        const T* q0 = B.at(c0[0], c0[1], c0[2]);
        const T* qp = B.at(cp[0], cp[1], cp[2]);
        for (int v = 0; v < N; ++v) sig[(ln * ns + (i + 1)) * N + v] = minmod(q0[v] - qm[v], qp[v] - q0[v]);
      }
    // Step: face states, their fluxes and speeds, and the Rusanov flux of every face 0..p.
    Fh.assign(lines * (p + 1) * N, T(0.0));
    std::vector<T> QL(N + M), QR(N + M), WL(MAXW), WR(MAXW), FL(N), FR(N);
    for (size_t ln = 0; ln < lines; ++ln)
      for (int f = 0; f <= p; ++f) {
        int cl[3], cr[3];
        coord(ln, f - 1, cl); coord(ln, f, cr);
        const T* ul = B.at(cl[0], cl[1], cl[2]);
        const T* ur = B.at(cr[0], cr[1], cr[2]);
        const T* sl = &sig[(ln * ns + f) * N];
        const T* sr = &sig[(ln * ns + f + 1) * N];
        for (int v = 0; v < N; ++v) {
          QL[v] = ul[v] + T(0.5) * sl[v];
          QR[v] = ur[v] - T(0.5) * sr[v];
        }
        for (int v = 0; v < M; ++v) { QL[N + v] = ul[N + v]; QR[N + v] = ur[N + v]; }
        prims(pde, P, QL.data(), QL.data() + N, WL.data());
        prims(pde, P, QR.data(), QR.data() + N, WR.data());
        flux(pde, P, d, QL.data(), QL.data() + N, WL.data(), FL.data());
        flux(pde, P, d, QR.data(), QR.data() + N, WR.data(), FR.data());
        const T s = fmax(speed(pde, P, d, QL.data(), QL.data() + N, WL.data()),
                         speed(pde, P, d, QR.data(), QR.data() + N, WR.data()));
        const T hs = T(0.5) * s;
        T* fh = &Fh[(ln * (p + 1) + f) * N];
        for (int v = 0; v < N; ++v) fh[v] = T(0.5) * (FL[v] + FR[v]) - hs * (QR[v] - QL[v]);
      }
    // Step: accumulate the face differences of direction d into every voxel.
    for (size_t ln = 0; ln < lines; ++ln)
      for (int i = 0; i < p; ++i) {
        int c[3]; coord(ln, i, c);
        const size_t vox = ((size_t)c[2] * p + c[1]) * p + c[0];
        const T* fm = &Fh[(ln * (p + 1) + i) * N];
        const T* fp = &Fh[(ln * (p + 1) + i + 1) * N];
        for (int v = 0; v < N; ++v) sum[vox * N + v] = sum[vox * N + v] + (fp[v] - fm[v]);
      }
  }
  // Step: assemble L = -(1/dx) sum + S.
  const T mrdx = -(T(1.0) / dx);
  std::vector<T> S(N);
  for (int z = 0; z < pz; ++z)
    for (int y = 0; y < p; ++y)
      for (int x = 0; x < p; ++x) {
        const size_t vox = ((size_t)z * p + y) * p + x;
        T* u = B.at(x, y, z);
        if (I.source) source(pde, P, u, u + N, S.data());
        for (int v = 0; v < N; ++v) {
          T l = mrdx * sum[vox * N + v];
          if (I.source) l = l + S[v];
          L[vox * N + v] = l;
        }
      }
}

// ---------------------------------------------------------------- FD operator
// L(Q) = -sum_d dF_d/dx_d - sum_d B_d(Q) dQ/dx_d + S(Q) + sigma/(64 dx) sum_d delta6_d Q
//   dQ/dx  = [(Q_-2 - Q_+2) + 8 (Q_+1 - Q_-1)] / (12 dx)
//   delta6 = (Q_-3 + Q_+3 - 2Q_0) - 6 (Q_-2 + Q_+2 - 2Q_0) + 15 (Q_-1 + Q_+1 - 2Q_0)
template <class T>
void fd_operator(int pde, const Params& P, Block<T>& B, double dxd, double sigma, std::vector<T>& L) {
  const PdeInfo I = pde_info(pde);
  const int N = I.N, p = B.p, dim = B.dim;
  const int pz = (dim == 3) ? p : 1;
  const T dx = T(dxd);
  const size_t nvox = (size_t)p * p * pz;
  L.assign(nvox * N, T(0.0));
  // Step: F_d at every voxel within 2 of the interior along axis d (needed by dF_d/dx_d).
  std::vector<T> W;
  std::vector<std::vector<T>> Fd(dim);
  if (I.flux) {
    W.assign((size_t)B.P * B.P * B.Pz * MAXW, T(0.0));
    const int zlo = (dim == 3) ? -2 : 0, zhi = (dim == 3) ? p + 2 : 1;
    for (int z = zlo; z < zhi; ++z)
      for (int y = -2; y < p + 2; ++y)
        for (int x = -2; x < p + 2; ++x) {
          int c[3] = {x, y, z}, outside = 0;
          for (int a = 0; a < dim; ++a) if (c[a] < 0 || c[a] >= p) ++outside;
          if (outside > 1) continue;
          T* u = B.at(x, y, z);
          prims(pde, P, u, u + I.N, &W[(size_t)B.idx(x, y, z) * MAXW]);
        }
    for (int d = 0; d < dim; ++d) {
      Fd[d].assign((size_t)B.P * B.P * B.Pz * N, T(0.0));
      for (int z = zlo; z < zhi; ++z)
        for (int y = -2; y < p + 2; ++y)
          for (int x = -2; x < p + 2; ++x) {
            int c[3] = {x, y, z}, outside = -1;
            bool ok = true;
            for (int a = 0; a < dim; ++a)
              if (c[a] < 0 || c[a] >= p) { if (a != d) ok = false; outside = a; }
            (void)outside;
            if (!ok) continue;
            T* u = B.at(x, y, z);
            const size_t id = (size_t)B.idx(x, y, z);
            flux(pde, P, d, u, u + N, &W[id * MAXW], &Fd[d][id * N]);
          }
    }
  }
  // Step: per interior voxel, derivatives, non-conservative product, KO and source.
  std::vector<T> dq(N), bq(N), S(N);
  const T r12 = T(1.0) / (T(12.0) * dx);  // 1/(12 dx)
  const T ko = T(sigma) / (T(64.0) * dx);
  for (int z = 0; z < pz; ++z)
    for (int y = 0; y < p; ++y)
      for (int x = 0; x < p; ++x) {
        size_t vox = ((size_t)z * p + y) * p + x;
        T* u0 = B.at(x, y, z);
        T* Lv = &L[vox * N];
        if (I.source) {
          source(pde, P, u0, u0 + N, S.data());
          for (int v = 0; v < N; ++v) Lv[v] = S[v];
        }
        for (int d = 0; d < dim; ++d) {
          const T* q[7];
          size_t id[7];
          for (int o = -3; o <= 3; ++o) {
            int c[3] = {x, y, z};
            c[d] += o;
            q[o + 3] = B.at(c[0], c[1], c[2]);
            id[o + 3] = (size_t)B.idx(c[0], c[1], c[2]);
          }
          if (I.flux) {
            const T* f[7];
            for (int o = 1; o <= 5; ++o) f[o] = &Fd[d][id[o] * N];
            for (int v = 0; v < N; ++v) {
              T df = ((f[1][v] - f[5][v]) + T(8.0) * (f[4][v] - f[2][v])) * r12;
              Lv[v] = Lv[v] - df;
            }
          }
          if (I.ncp) {
            for (int v = 0; v < N; ++v)
              dq[v] = needs_grad(pde, d, v) ? ((q[1][v] - q[5][v]) + T(8.0) * (q[4][v] - q[2][v])) * r12 : T(0.0);
            ncp(pde, P, d, u0, dq.data(), bq.data());
            for (int v = 0; v < N; ++v) Lv[v] = Lv[v] - bq[v];
          }
          for (int v = 0; v < N; ++v) {
            T two = T(2.0) * q[3][v];
            T d6 = ((q[0][v] + q[6][v]) - two) - T(6.0) * ((q[1][v] + q[5][v]) - two) +
                   T(15.0) * ((q[2][v] + q[4][v]) - two);
            Lv[v] = Lv[v] + ko * d6;
          }
        }
      }
}

// ---------------------------------------------------------------- wave speed
// Maximum characteristic speed over all voxels and directions.
double max_speed(const Patch* patches, int K, int pde, const Params& P, int dim, int64_t var_stride,
                 const double* q, const double* mat) {
  const PdeInfo I = pde_info(pde);
  double lam = 0.0;
#pragma omp parallel for reduction(max : lam) if (K > 1)
  for (int k = 0; k < K; ++k) {
    const int p = patches[k].p, pz = (dim == 3) ? p : 1;
    double u[64], m[8], W[MAXW];
    for (int vox = 0; vox < p * p * pz; ++vox) {
      int64_t e = patches[k].offset + vox;
      for (int v = 0; v < I.N; ++v) u[v] = q[v * var_stride + e];
      for (int v = 0; v < I.M; ++v) m[v] = mat[v * var_stride + e];
      prims(pde, P, u, m, W);
      for (int d = 0; d < dim; ++d) lam = std::max(lam, speed(pde, P, d, u, m, W));
    }
  }
  return lam;
}

// ---------------------------------------------------------------- coupling steps
// Rusanov flux F^ = (F_d(QL) + F_d(QR))/2 - s/2 (QR - QL) of one face (qL, qR: N+M values).
template <class T>
void rusanov_face(int pde, const Params& P, int d, const T* qL, const T* qR, T* fh) {
  const PdeInfo I = pde_info(pde);
  const int N = I.N;
  T WL[MAXW], WR[MAXW], FL[64], FR[64];
  prims(pde, P, qL, qL + N, WL);
  prims(pde, P, qR, qR + N, WR);
  flux(pde, P, d, qL, qL + N, WL, FL);
  flux(pde, P, d, qR, qR + N, WR, FR);
  const T sp = fmax(speed(pde, P, d, qL, qL + N, WL), speed(pde, P, d, qR, qR + N, WR));
  const T hs = T(0.5) * sp;
  for (int v = 0; v < N; ++v) fh[v] = T(0.5) * (FL[v] + FR[v]) - hs * (qR[v] - qL[v]);
}

// Reflux and restriction after a first-order FV stage on a coupled mesh (see
// "coarse-fine coupling" above).  qs: the stage input; out/acc as in stage().
template <class T>
void couple_levels(int pde, const Params& P, int dim, const Patch* patches, int K, int64_t vs,
                   const double* qs, const double* mat, double* out, double* acc, double dt, double g,
                   double dd) {
  const PdeInfo I = pde_info(pde);
  const int N = I.N, M = I.M;
  const std::vector<int> par = parents(patches, K, dim);
  auto load = [&](int k, int x, int y, int z, T* q) {
    const int p = patches[k].p;
    const int64_t e = patches[k].offset + ((int64_t)z * p + y) * p + x;
    for (int v = 0; v < N; ++v) q[v] = T(qs[v * vs + e]);
    for (int v = 0; v < M; ++v) q[N + v] = T(mat[v * vs + e]);
    return e;
  };
  // Reflux: every face of a fine patch whose neighbour is coarser, one coarse voxel at a time.
  std::vector<T> qC(N + M), qN(N + M), qF(N + M), fc(N), ff(N), fsum(N);
  for (int k = 0; k < K; ++k) {
    const Patch& F = patches[k];
    const int p = F.p, h2 = p / 2;
    for (int f = 0; f < 2 * dim; ++f) {
      const int C = F.nbr[f];
      if (patches[C].level >= F.level) continue;
      const int a = f / 2, lo = (f % 2 == 0);  // lo: the coarse patch lies on the -a side of F
      const int b0 = (a + 1) % dim, b1 = dim == 3 ? (a + 2) % dim : -1;
      const int nj = h2, nk = dim == 3 ? h2 : 1;
      for (int kk = 0; kk < nk; ++kk)
        for (int jj = 0; jj < nj; ++jj) {
          int cc[3] = {0, 0, 0}, cn[3] = {0, 0, 0};
          cc[a] = lo ? p - 1 : 0;                         // coarse voxel next to the finer level
          cn[a] = octant(F, a) * h2 + (lo ? 0 : h2 - 1);   // coarse voxel across the face (covered)
          cc[b0] = cn[b0] = octant(F, b0) * h2 + jj;
          if (b1 >= 0) cc[b1] = cn[b1] = octant(F, b1) * h2 + kk;
          const int64_t eC = load(C, cc[0], cc[1], cc[2], qC.data());
          load(par[k], cn[0], cn[1], cn[2], qN.data());
          if (lo) rusanov_face(pde, P, a, qC.data(), qN.data(), fc.data());
          else rusanov_face(pde, P, a, qN.data(), qC.data(), fc.data());
          // fine face fluxes, summed as a balanced tree ((f00 + f10) + (f01 + f11)) so that equal
          // fluxes sum exactly
          const int nfk = dim == 3 ? 2 : 1;
          std::vector<T> pair(N);
          for (int sk = 0; sk < nfk; ++sk) {
            for (int sj = 0; sj < 2; ++sj) {
              int cf[3] = {0, 0, 0};
              cf[a] = lo ? 0 : p - 1;
              cf[b0] = 2 * jj + sj;
              if (b1 >= 0) cf[b1] = 2 * kk + sk;
              load(k, cf[0], cf[1], cf[2], qF.data());
              if (lo) rusanov_face(pde, P, a, qC.data(), qF.data(), ff.data());
              else rusanov_face(pde, P, a, qF.data(), qC.data(), ff.data());
              for (int v = 0; v < N; ++v) pair[v] = sj == 0 ? ff[v] : pair[v] + ff[v];
            }
            for (int v = 0; v < N; ++v) fsum[v] = sk == 0 ? pair[v] : fsum[v] + pair[v];
          }
          const T rn = T(1.0) / T(dim == 3 ? 4.0 : 2.0);
          const T sgn = lo ? T(-1.0) : T(1.0);  // the face is the +a face of C (lo) or its -a face
          for (int v = 0; v < N; ++v) {
            const T dL = sgn * (fsum[v] * rn - fc[v]) / T(patches[C].dx);
            const int64_t ev = v * vs + eC;
            if (out) out[ev] = val(T(out[ev]) + T(g) * T(dt) * dL);
            if (acc) acc[ev] = val(T(acc[ev]) + T(dd) * T(dt) * dL);
          }
        }
    }
  }
  // Restriction: the coarse voxels under every fine patch, finest level first.
  std::vector<int> order(K);
  for (int k = 0; k < K; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return patches[a].level > patches[b].level; });
  for (int k : order) {
    if (par[k] < 0) continue;
    const Patch& F = patches[k];
    const Patch& Pp = patches[par[k]];
    const int p = F.p, h2 = p / 2, hz = dim == 3 ? h2 : 1;
    const int nsub = dim == 3 ? 8 : 4;
    for (int z = 0; z < hz; ++z)
      for (int y = 0; y < h2; ++y)
        for (int x = 0; x < h2; ++x) {
          const int cx = octant(F, 0) * h2 + x, cy = octant(F, 1) * h2 + y, cz = dim == 3 ? octant(F, 2) * h2 + z : 0;
          const int64_t ec = Pp.offset + ((int64_t)cz * p + cy) * p + cx;
          for (int w = 0; w < 2; ++w) {
            double* arr = w == 0 ? out : acc;
            if (!arr) continue;
            for (int v = 0; v < N; ++v) {
              // balanced tree: ((x pair) + (x pair)) per z layer, then the two layers
              T layer[2] = {T(0.0), T(0.0)};
              for (int sz = 0; sz < (dim == 3 ? 2 : 1); ++sz) {
                T row[2];
                for (int sy = 0; sy < 2; ++sy) {
                  const int64_t ef = F.offset + ((int64_t)(dim == 3 ? 2 * z + sz : 0) * p + 2 * y + sy) * p + 2 * x;
                  row[sy] = T(arr[v * vs + ef]) + T(arr[v * vs + ef + 1]);
                }
                layer[sz] = row[0] + row[1];
              }
              const T sum = dim == 3 ? layer[0] + layer[1] : layer[0];
              arr[v * vs + ec] = val(sum / T((double)nsub));
            }
          }
        }
  }
}

// ---------------------------------------------------------------- stage driver
// One Runge-Kutta stage over all K patches (the batched kernel K~_{dt,K}):
//   out = a Q0 + b Qs + g dt L(Qs)   (out may be NULL)
//   acc = acc + d dt L(Qs)           (acc may be NULL)
// Returns, through lam, the maximum characteristic speed of the result
// (out if given, else acc) over all voxels and directions.
template <class T>
void stage(int scheme, int pde, const Params& P, int dim, const Patch* patches, int K, int h,
           int64_t var_stride, const double* qs, const double* q0, double* out, double* acc,
           const double* mat, double dt, double a, double b, double g, double dd, double sigma,
           double* lam, const int32_t* only = nullptr, int n_only = 0) {
  const PdeInfo I = pde_info(pde);
  const int N = I.N, M = I.M;
  const T gdt = T(g) * T(dt), ddt = T(dd) * T(dt);  // per-stage scalars g dt and d dt
  double lam_max = 0.0;
  const int n = only ? n_only : K;  // optionally only the listed patches (halos still from all)
#pragma omp parallel for schedule(dynamic, 1) reduction(max : lam_max) if (n > 1)
  for (int kk = 0; kk < n; ++kk) {
    const int k = only ? only[kk] : kk;
    Block<T> B;
    gather_block(B, patches, k, dim, h, N, M, var_stride, qs, mat);
    std::vector<T> L;
    if (scheme == 0) fv_operator(pde, P, B, patches[k].dx, L);
    else if (scheme == 2) fv2_operator(pde, P, B, patches[k].dx, L);
    else fd_operator(pde, P, B, patches[k].dx, sigma, L);
    const int p = patches[k].p, pz = (dim == 3) ? p : 1;
    const int64_t off = patches[k].offset;
    std::vector<T> res(N), W(MAXW);
    for (int z = 0; z < pz; ++z)
      for (int y = 0; y < p; ++y)
        for (int x = 0; x < p; ++x) {
          const size_t vox = ((size_t)z * p + y) * p + x;
          const int64_t e = off + (int64_t)vox;
          for (int v = 0; v < N; ++v) {
            const int64_t ev = v * var_stride + e;
            T l = L[vox * N + v];
            if (out) {
              T r = T(b) * T(qs[ev]);
              if (q0) r = T(a) * T(q0[ev]) + r;
              r = r + gdt * l;
              res[v] = r;
            }
            if (acc) {
              T r = T(acc[ev]) + ddt * l;
              if (!out) res[v] = r;
              acc[ev] = val(r);
            }
            if (out) out[ev] = val(res[v]);
          }
          if (lam && pde != SRHD3D) {
            std::vector<T> m(M > 0 ? M : 1);
            for (int v = 0; v < M; ++v) m[v] = T(mat[v * var_stride + e]);
            prims(pde, P, res.data(), m.data(), W.data());
            for (int d = 0; d < dim; ++d) {
              double s = val(speed(pde, P, d, res.data(), m.data(), W.data()));
              lam_max = std::max(lam_max, s);
            }
          }
        }
  }
  if (scheme == 0 && !only && coupled_mesh(patches, K, dim)) {
    couple_levels<T>(pde, P, dim, patches, K, var_stride, qs, mat, out, acc, dt, g, dd);
    // the wave speed of the coupled result (all voxels, covered coarse ones included)
    if (lam) lam_max = max_speed(patches, K, pde, P, dim, var_stride, out ? out : acc, mat);
  }
  if (lam) *lam = lam_max;
}

// ---------------------------------------------------------------- SRHD
template <class T>
void srhd_prim2con(double Gamma, const T* w, T* q) {
  // w = (rho, vx, vy, vz, p) -> q = (D, Sx, Sy, Sz, tau)
  T rho = w[0], p = w[4];
  T v2 = w[1] * w[1] + w[2] * w[2] + w[3] * w[3];
  T W = T(1.0) / sqrt(T(1.0) - v2);
  T hh = T(1.0) + T(Gamma) * p / ((T(Gamma) - T(1.0)) * rho);
  T rhohW2 = rho * hh * W * W;
  q[0] = rho * W;
  q[1] = rhohW2 * w[1];
  q[2] = rhohW2 * w[2];
  q[3] = rhohW2 * w[3];
  q[4] = rhohW2 - p - q[0];
}

// Newton iteration on the pressure:
//   f(p)  = ((G-1)/G) [ (E+p) - S^2/(E+p) - D sqrt(1 - S^2/(E+p)^2) ] - p
//   f'(p) = ((G-1)/G) [ 1 + S^2/(E+p)^2 - D S^2 / ((E+p)^3 sqrt(1 - S^2/(E+p)^2)) ] - 1
// Stops when |p_new - p| <= tol p_new.  A step that would leave the bracket
// (p_lo, inf) is replaced by the midpoint between the current iterate and
// p_lo (safeguard: plain Newton from a cold seed overshoots below zero for
// fast flows).  Fails on NaN or when max_iter iterations did not converge.
// Returns iterations used (>0) on success, -iterations on failure.
template <class T>
int srhd_newton(double G, T D, T S2, T E, T p_lo, T p0, double tol, int max_iter, T* p_out) {
  T p = p0;
  const T gf = T((G - 1.0) / G), one = T(1.0);
  for (int it = 1; it <= max_iter; ++it) {
    T Ep = E + p;
    T s2e = S2 / (Ep * Ep);
    T rt = sqrt(one - s2e);
    T f = gf * (Ep - S2 / Ep - D * rt) - p;
    T fp = gf * (one + s2e - D * S2 / (Ep * Ep * Ep * rt)) - one;
    T pn = p - f / fp;
    if (!(val(pn) == val(pn))) { *p_out = pn; return -it; }
    if (pn <= p_lo) {
      pn = T(0.5) * (p + p_lo);  // safeguard step: never counts as convergence
    } else if (fabs(pn - p) <= T(tol) * pn) {
      *p_out = pn;
      return it;
    }
    p = pn;
  }
  *p_out = p;
  return -max_iter;
}

// MLP 3 -> 32 tanh -> 32 tanh -> 1.  Weight vector layout (floats):
//   W1[32][3], b1[32], W2[32][32], b2[32], W3[32], b3, then z-score mean[3], std[3].
const int MLP_NW = 3 * 32 + 32 + 32 * 32 + 32 + 32 + 1;  // 1217

template <class R>
R mlp_forward(const R* w, const R* x, R* h1, R* h2) {
  const R* W1 = w; const R* b1 = W1 + 96; const R* W2 = b1 + 32; const R* b2 = W2 + 1024;
  const R* W3 = b2 + 32; const R* b3 = W3 + 32;
  for (int i = 0; i < 32; ++i) {
    R s = b1[i];
    for (int j = 0; j < 3; ++j) s += W1[3 * i + j] * x[j];
    h1[i] = std::tanh(s);
  }
  for (int i = 0; i < 32; ++i) {
    R s = b2[i];
    for (int j = 0; j < 32; ++j) s += W2[32 * i + j] * h1[j];
    h2[i] = std::tanh(s);
  }
  R y = b3[0];
  for (int j = 0; j < 32; ++j) y += W3[j] * h2[j];
  return y;
}

// Invariants of a conserved state: (|S|/E, D/E, ln(E/D)), E = tau + D.
void srhd_invariants(const double* q, double* x) {
  double D = q[0], E = q[4] + q[0];
  double S = std::sqrt(q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  x[0] = S / E;
  x[1] = D / E;
  x[2] = std::log(E / D);
}

// FP32 refinement of a seed: up to k Newton steps on the pressure in single precision.  The
// textbook f cancels badly in FP32 (1 - S^2/(E+p)^2 at high Lorentz factors, rho h - rho for
// cold gas), so the step is written with two invariants formed once in FP64 with fused
// multiply-adds, A = E^2 - S^2 and B = tau (tau + 2 D) - S^2 (= A - D^2), where
// S^2 = fma(S_x, S_x, fma(S_y, S_y, S_z S_z)).  With y = E + p and t = p (E + y) = y^2 - E^2:
// q = sqrt(y^2 - S^2) = sqrt(A + t) and q - D = (q^2 - D^2)/(q + D) = (B + t)/(q + D) are
// sums of positive terms, y f = gf q (q - D) - p y and y^2 f' = gf S^2 (q - D)/q + (gf - 1) y^2
// (gf = (Gamma - 1)/Gamma), and p <- p - y (y f)/(y^2 f').  Every FP32 operation is rounded to
// float, no fused multiply-add, on float copies of A, B, E, D and S^2.  A step whose result is
// not finite or not above the bracket's lower end (in float) stops the refinement and keeps the
// value before it.  The FP64 Newton iteration then starts from the result.  (The paper has no
// relativistic hydrodynamics; this is the reading of a seeded solve on hardware whose FP32
// throughput is far above its FP64 throughput.)
double refine_seed_f32(double Gamma, const double* q, double E, double p_lo, double seed, int k) {
  const double S2 = std::fma(q[1], q[1], std::fma(q[2], q[2], q[3] * q[3]));
  const double A = std::fma(E, E, -S2), B = std::fma(q[4], std::fma(2.0, q[0], q[4]), -S2);
  const float Af = (float)A, Bf = (float)B, Ef = (float)E, Df = (float)q[0], S2f = (float)S2, lo = (float)p_lo;
  const float gf = (float)((Gamma - 1.0) / Gamma), gm = gf - 1.0f;
  float p = (float)seed;
  for (int i = 0; i < k; ++i) {
    const float y = Ef + p;
    const float t = p * (Ef + y);
    const float qq = std::sqrt(Af + t);
    const float qmD = (Bf + t) / (qq + Df);
    const float yf = gf * qq * qmD - p * y;
    const float den = gf * S2f * qmD / qq + gm * y * y;
    const float pn = p - y * yf / den;
    if (!(pn > lo && pn < std::numeric_limits<float>::infinity())) break;
    p = pn;
  }
  return (double)p;
}

// Per-voxel quantities of the conserved state q = (D, S_x, S_y, S_z, tau) that the recovery
// uses: E = tau + D, S^2, the bracket's lower end p_lo = max(0, |S| - E) and the cold seed
// max((1 + 1e-8) p_lo + 1e-300, (Gamma - 1) tau).
template <class T>
struct C2pSetup {
  T D, E, S2, p_lo, cold;
};

template <class T>
C2pSetup<T> c2p_setup(double Gamma, const T* q) {
  C2pSetup<T> c;
  c.D = q[0];
  c.E = q[4] + q[0];
  c.S2 = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  const T S = sqrt(c.S2);
  c.p_lo = fmax(T(0.0), S - c.E);
  c.cold = fmax(T(1.0 + 1e-8) * c.p_lo + T(1e-300), T(Gamma - 1.0) * q[4]);
  return c;
}

// Newton from seed s1, then (if have2 and s1 failed) from s2; on a double failure the pressure
// is `keep`.  Writes (rho, v_x, v_y, v_z, p) with v = S/(E + p), W = 1/sqrt(1 - v^2),
// rho = D/W, and the total iterations; returns the status 0 / 1 / 2.
template <class T>
uint8_t c2p_solve(double Gamma, const T* q, const C2pSetup<T>& c, T s1, T s2, bool have2, T keep, double tol,
                  int max_iter, T* w, int* total_out) {
  T p;
  int it1 = srhd_newton<T>(Gamma, c.D, c.S2, c.E, c.p_lo, s1, tol, max_iter, &p);
  int total = it1 > 0 ? it1 : -it1;
  uint8_t st = 0;
  if (it1 <= 0) {
    int it2 = have2 ? srhd_newton<T>(Gamma, c.D, c.S2, c.E, c.p_lo, s2, tol, max_iter, &p) : -0;
    total += it2 > 0 ? it2 : -it2;
    if (have2 && it2 > 0) st = 1;
    else { st = 2; p = keep; }
  }
  const T Ep = c.E + p;
  T v[3] = {q[1] / Ep, q[2] / Ep, q[3] / Ep};
  T v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  T W = T(1.0) / sqrt(T(1.0) - v2);
  w[0] = c.D / W;
  w[1] = v[0];
  w[2] = v[1];
  w[3] = v[2];
  w[4] = p;
  *total_out = total;
  return st;
}

}  // namespace

// ============================================================= C entry points
extern "C" {

int or_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

int or_pde_nq(int pde) { return pde_info(pde).N; }
int or_pde_nm(int pde) { return pde_info(pde).M; }

// One FV stage (scheme 0), FD4+KO stage (scheme 1) or FV stage with MUSCL
// minmod reconstruction (scheme 2, halo 2, conservative systems) over all patches.
int or_stage(int scheme, int pde, int dim, const void* patches, int K, int halo, int64_t var_stride,
             const double* qs, const double* q0, double* out, double* acc, const double* mat,
             double dt, double a, double b, double g, double d, double sigma, const double* prm,
             int nprm, double* lam) {
  Params P = make_params(pde, prm, nprm);
  stage<double>(scheme, pde, P, dim, (const Patch*)patches, K, halo, var_stride, qs, q0, out, acc,
                mat, dt, a, b, g, d, sigma, lam);
  return 0;
}

// One stage on the listed patches only (halos still come from every patch):
// a sample of a workload too large for the whole oracle.
int or_stage_subset(int scheme, int pde, int dim, const void* patches, int K, int halo, int64_t var_stride,
                    const double* qs, const double* q0, double* out, double* acc, const double* mat,
                    double dt, double a, double b, double g, double d, double sigma, const double* prm,
                    int nprm, const int32_t* only, int n_only) {
  Params P = make_params(pde, prm, nprm);
  stage<double>(scheme, pde, P, dim, (const Patch*)patches, K, halo, var_stride, qs, q0, out, acc, mat, dt,
                a, b, g, d, sigma, nullptr, only, n_only);
  return 0;
}

// Maximum characteristic speed over all voxels and directions.
double or_max_wave_speed(int pde, int dim, const void* patches_v, int K, int64_t var_stride,
                         const double* q, const double* mat, const double* prm, int nprm) {
  return max_speed((const Patch*)patches_v, K, pde, make_params(pde, prm, nprm), dim, var_stride, q, mat);
}

// dt = CFL dx / (dim lambda_max)
double or_cfl_dt(double cfl, double dx, int dim, double lam) { return cfl * dx / ((double)dim * lam); }

// Whole time steps with a Runge-Kutta scheme built from stage calls:
//   rk = 1 forward Euler; rk = 3 SSP-RK3 (Shu-Osher); rk = 4 classical RK4.
// q holds Q^n on entry and Q^{n+steps} on exit.  dt_fixed > 0 fixes dt,
// else dt = CFL dx_min/(dim lambda_max) from the state at the start of each
// step.  Work buffers u1, u2 (and acc for RK4) are caller-provided arena-sized
// arrays.  dt_log (optional) receives the dt of every step.
int or_rk_steps(int scheme, int pde, int dim, const void* patches_v, int K, int halo,
                int64_t var_stride, double* q, double* u1, double* u2, double* accb,
                const double* mat, int rk, int steps, double dt_fixed, double cfl, double sigma,
                const double* prm, int nprm, double* dt_log) {
  const Patch* patches = (const Patch*)patches_v;
  const PdeInfo I = pde_info(pde);
  Params P = make_params(pde, prm, nprm);
  double dxmin = patches[0].dx;
  for (int k = 1; k < K; ++k) dxmin = std::min(dxmin, patches[k].dx);
  size_t nelem = (size_t)var_stride * I.N;
  double lam = or_max_wave_speed(pde, dim, patches_v, K, var_stride, q, mat, prm, nprm);
  // on a coupled mesh the wave speed is taken from the state after the coupling
  // steps (restriction, reflux) at the end of every step
  const bool coupled = coupled_mesh(patches, K, dim);
  for (int s = 0; s < steps; ++s) {
    double dt = dt_fixed > 0 ? dt_fixed : or_cfl_dt(cfl, dxmin, dim, lam);
    if (dt_log) dt_log[s] = dt;
    double* lp = (dt_fixed > 0 || coupled) ? nullptr : &lam;
    if (rk == 1) {
      stage<double>(scheme, pde, P, dim, patches, K, halo, var_stride, q, nullptr, u1, nullptr, mat,
                    dt, 0, 1, 1, 0, sigma, lp);
      std::memcpy(q, u1, nelem * sizeof(double));
    } else if (rk == 3) {
      stage<double>(scheme, pde, P, dim, patches, K, halo, var_stride, q, nullptr, u1, nullptr, mat,
                    dt, 0, 1, 1, 0, sigma, nullptr);
      stage<double>(scheme, pde, P, dim, patches, K, halo, var_stride, u1, q, u2, nullptr, mat, dt,
                    0.75, 0.25, 0.25, 0, sigma, nullptr);
      stage<double>(scheme, pde, P, dim, patches, K, halo, var_stride, u2, q, q, nullptr, mat, dt,
                    1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, 0, sigma, lp);
    } else if (rk == 4) {
      std::memcpy(accb, q, nelem * sizeof(double));
      stage<double>(scheme, pde, P, dim, patches, K, halo, var_stride, q, q, u1, accb, mat, dt, 1, 0,
                    0.5, 1.0 / 6.0, sigma, nullptr);
      stage<double>(scheme, pde, P, dim, patches, K, halo, var_stride, u1, q, u2, accb, mat, dt, 1, 0,
                    0.5, 1.0 / 3.0, sigma, nullptr);
      stage<double>(scheme, pde, P, dim, patches, K, halo, var_stride, u2, q, u1, accb, mat, dt, 1, 0,
                    1.0, 1.0 / 3.0, sigma, nullptr);
      stage<double>(scheme, pde, P, dim, patches, K, halo, var_stride, u1, nullptr, nullptr, accb,
                    mat, dt, 0, 0, 0, 1.0 / 6.0, sigma, lp);
      std::memcpy(q, accb, nelem * sizeof(double));
    } else {
      return -1;
    }
    if (coupled && dt_fixed <= 0) lam = or_max_wave_speed(pde, dim, patches_v, K, var_stride, q, mat, prm, nprm);
  }
  return 0;
}

// Primitive -> conserved for the Euler systems and SRHD, element-wise over n
// voxels in SoA layout (prim[v*stride + i] -> cons[v*stride + i]).
//   Euler: (rho, u.., p) -> (rho, rho u.., E = p/(gamma-1) + rho |u|^2 / 2)
//   SRHD:  (rho, v, p)   -> (D, S, tau), see srhd_prim2con.
int or_prim2con(int pde, const double* prim, double* cons, int64_t n, int64_t stride,
                const double* prm, int nprm) {
  Params P = make_params(pde, prm, nprm);
  if (pde == EULER2D || pde == EULER3D) {
    int d = (pde == EULER2D) ? 2 : 3;
    for (int64_t i = 0; i < n; ++i) {
      double rho = prim[i], p = prim[(d + 1) * stride + i];
      double kin = 0.0;
      cons[i] = rho;
      for (int k = 0; k < d; ++k) {
        double u = prim[(1 + k) * stride + i];
        cons[(1 + k) * stride + i] = rho * u;
        kin = kin + rho * u * u;
      }
      cons[(d + 1) * stride + i] = p / (P.gamma - 1.0) + 0.5 * kin;
    }
    return 0;
  }
  if (pde == SRHD3D) {
    for (int64_t i = 0; i < n; ++i) {
      double w[5], q[5];
      for (int v = 0; v < 5; ++v) w[v] = prim[v * stride + i];
      srhd_prim2con<double>(P.Gamma, w, q);
      for (int v = 0; v < 5; ++v) cons[v * stride + i] = q[v];
    }
    return 0;
  }
  return -1;
}

// Conserved -> primitive for SRHD (Newton on p).  Per voxel:
//   seed 1: MLP guess if mlp != NULL, else p_prev if given, else the cold seed
//           max((1+1e-8) p_lo + 1e-300, (Gamma-1) tau);
//   seed 2 (only if seed 1 fails): p_prev if the MLP was seed 1 and p_prev is
//           given, else the cold seed.
//   refine > 0: seed 1 is first refined by up to `refine` FP32 Newton steps
//           (refine_seed_f32); seed 2 is never refined.
//   status 0: seed 1 converged; 1: seed 2 converged; 2: both failed (the
//   pressure falls back to p_prev, or the cold seed, and the voxel counts as a
//   failure).  iters (optional) receives the total Newton iterations.
int or_con2prim(const double* cons, double* prim, int64_t n, int64_t stride, const double* p_prev,
                const float* mlp, double tol, int max_iter, uint8_t* status, int32_t* iters,
                double Gamma, int refine) {
  int fails = 0;
#pragma omp parallel for reduction(+ : fails) if (n > 4096)
  for (int64_t i = 0; i < n; ++i) {
    double q[5];
    for (int v = 0; v < 5; ++v) q[v] = cons[v * stride + i];
    const C2pSetup<double> c = c2p_setup<double>(Gamma, q);
    double s1, s2;
    bool have2;
    if (mlp) {
      double xd[3];
      srhd_invariants(q, xd);
      float x[3], h1[32], h2[32];
      for (int j = 0; j < 3; ++j) x[j] = (float)((xd[j] - (double)mlp[MLP_NW + j]) / (double)mlp[MLP_NW + 3 + j]);
      float y = mlp_forward<float>(mlp, x, h1, h2);
      // with the FP32 refinement the seed itself is formed in FP32 as well
      double ps = refine > 0 ? (double)((float)c.E * std::exp(y)) : c.E * std::exp((double)y);
      double lo = c.p_lo * (1.0 + 1e-12);
      s1 = ps > lo ? ps : c.cold;
      s2 = p_prev ? p_prev[i] : c.cold;
      have2 = true;
    } else {
      s1 = p_prev ? p_prev[i] : c.cold;
      s2 = c.cold;
      have2 = (p_prev != nullptr);
    }
    if (refine > 0) s1 = refine_seed_f32(Gamma, q, c.E, c.p_lo, s1, refine);
    double w[5];
    int total = 0;
    const uint8_t st = c2p_solve<double>(Gamma, q, c, s1, s2, have2, p_prev ? p_prev[i] : c.cold, tol, max_iter, w,
                                         &total);
    if (st == 2) ++fails;
    for (int v = 0; v < 5; ++v) prim[v * stride + i] = w[v];
    if (status) status[i] = st;
    if (iters) iters[i] = total;
  }
  return fails;
}

// Exact FP64 operation count (counting build) of the recovery of n voxels with the plain seed
// (p_prev, else the cold seed): the same setup, Newton iterations and recovery as or_con2prim.
// *iters_out receives the total number of Newton iterations.
long long or_count_con2prim(const double* cons, int64_t n, int64_t stride, const double* p_prev, double tol,
                            int max_iter, double Gamma, long long* iters_out) {
  g_flops = 0;
  long long it_sum = 0;
  for (int64_t i = 0; i < n; ++i) {
    Counted q[5];
    for (int v = 0; v < 5; ++v) q[v] = Counted(cons[v * stride + i]);
    const C2pSetup<Counted> c = c2p_setup<Counted>(Gamma, q);
    const Counted s1 = p_prev ? Counted(p_prev[i]) : c.cold;
    Counted w[5];
    int total = 0;
    c2p_solve<Counted>(Gamma, q, c, s1, c.cold, p_prev != nullptr, s1, tol, max_iter, w, &total);
    it_sum += total;
  }
  if (iters_out) *iters_out = it_sum;
  return g_flops;
}

// Exact FP64 operation count of the maximum characteristic speed of n voxels (flat arrays,
// variable v of voxel i at v * stride + i): derived quantities and the speed in every direction.
long long or_count_max_speed(int pde, int dim, const double* q, const double* mat, int64_t n, int64_t stride,
                             const double* prm, int nprm) {
  const Params P = make_params(pde, prm, nprm);
  const PdeInfo I = pde_info(pde);
  g_flops = 0;
  for (int64_t i = 0; i < n; ++i) {
    Counted u[64], m[8], W[MAXW];
    for (int v = 0; v < I.N; ++v) u[v] = Counted(q[v * stride + i]);
    for (int v = 0; v < I.M; ++v) m[v] = Counted(mat[v * stride + i]);
    prims(pde, P, u, m, W);
    Counted lam(0.0);
    for (int d = 0; d < dim; ++d) lam = fmax(lam, speed(pde, P, d, u, m, W));
  }
  return g_flops;
}

// The FP32 refinement alone (refine_seed_f32) of n seeds: out[i] = the refined seed of voxel i.
void or_refine_seed(const double* cons, int64_t n, int64_t stride, const double* seed, int k, double Gamma,
                    double* out) {
  for (int64_t i = 0; i < n; ++i) {
    double q[5];
    for (int v = 0; v < 5; ++v) q[v] = cons[v * stride + i];
    const C2pSetup<double> c = c2p_setup<double>(Gamma, q);
    out[i] = refine_seed_f32(Gamma, q, c.E, c.p_lo, seed[i], k);
  }
}

// Inputs of the MLP (z-scored with mean/std in the weight vector) for n voxels.
void or_srhd_invariants(const double* cons, int64_t n, int64_t stride, double* x) {
  for (int64_t i = 0; i < n; ++i) {
    double q[5];
    for (int v = 0; v < 5; ++v) q[v] = cons[v * stride + i];
    srhd_invariants(q, &x[3 * i]);
  }
}

// FP64 forward pass and gradient of the loss  (1/B) sum_i (y_i - t_i)^2
// with respect to the 1217 weights, by plain backpropagation.
double or_mlp_loss_grad(const double* w, const double* x, const double* t, int B, double* grad) {
  const double* W1 = w; const double* W2 = W1 + 128; const double* W3 = W2 + 1056;
  if (grad) std::fill(grad, grad + MLP_NW, 0.0);
  double loss = 0.0;
  for (int i = 0; i < B; ++i) {
    double h1[32], h2[32];
    double y = mlp_forward<double>(w, &x[3 * i], h1, h2);
    double r = y - t[i];
    loss += r * r;
    if (!grad) continue;
    double gy = 2.0 * r / B;
    double* gW1 = grad; double* gb1 = gW1 + 96; double* gW2 = gb1 + 32; double* gb2 = gW2 + 1024;
    double* gW3 = gb2 + 32; double* gb3 = gW3 + 32;
    double g2[32], g1[32];
    for (int j = 0; j < 32; ++j) {
      gW3[j] += gy * h2[j];
      g2[j] = gy * W3[j] * (1.0 - h2[j] * h2[j]);
    }
    gb3[0] += gy;
    for (int a = 0; a < 32; ++a) {
      gb2[a] += g2[a];
      for (int j = 0; j < 32; ++j) gW2[32 * a + j] += g2[a] * h1[j];
    }
    for (int j = 0; j < 32; ++j) {
      double s = 0.0;
      for (int a = 0; a < 32; ++a) s += W2[32 * a + j] * g2[a];
      g1[j] = s * (1.0 - h1[j] * h1[j]);
    }
    for (int a = 0; a < 32; ++a) {
      gb1[a] += g1[a];
      for (int j = 0; j < 3; ++j) gW1[3 * a + j] += g1[a] * x[3 * i + j];
    }
  }
  return loss / B;
  (void)W1;
}

// FP64 MLP forward for n inputs (already z-scored).
void or_mlp_forward(const double* w, const double* x, int64_t n, double* y) {
  for (int64_t i = 0; i < n; ++i) {
    double h1[32], h2[32];
    y[i] = mlp_forward<double>(w, &x[3 * i], h1, h2);
  }
}

// Adam step (Kingma & Ba 2015) in FP64: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// w -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
void or_adam(double* w, double* m, double* v, const double* g, int n, int t, double lr, double b1,
             double b2, double eps) {
  double c1 = 1.0 - std::pow(b1, t), c2 = 1.0 - std::pow(b2, t);
  for (int i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    w[i] -= lr * (m[i] / c1) / (std::sqrt(v[i] / c2) + eps);
  }
}

// Exact FP64 operation count of one stage (or one full RK step when rk > 0)
// on a single patch of size p that is its own periodic neighbour.  Used to
// derive the per-voxel algorithmic flop count: the halo share grows like p^(d-1).
long long or_count_flops(int scheme, int pde, int dim, int p, int halo, int rk, int with_lam,
                         const double* qs, const double* mat, const double* prm, int nprm) {
  Params P = make_params(pde, prm, nprm);
  const PdeInfo I = pde_info(pde);
  Patch pt;
  std::memset(&pt, 0, sizeof(pt));
  pt.p = p; pt.dx = 1.0 / 64.0;
  for (int i = 0; i < 6; ++i) pt.nbr[i] = 0;
  const int pz = (dim == 3) ? p : 1;
  const int64_t nv = (int64_t)p * p * pz;
  std::vector<double> u1(nv * I.N), u2(nv * I.N), q(qs, qs + nv * I.N), acc(nv * I.N);
  double lam;
  g_flops = 0;
  double dt = 1e-3;
  if (rk == 0) {
    stage<Counted>(scheme, pde, P, dim, &pt, 1, halo, nv, qs, nullptr, u1.data(), nullptr, mat, dt, 0, 1,
                   1, 0, 0.1, with_lam ? &lam : nullptr);
  } else if (rk == 1) {
    stage<Counted>(scheme, pde, P, dim, &pt, 1, halo, nv, q.data(), nullptr, u1.data(), nullptr, mat,
                   dt, 0, 1, 1, 0, 0.1, with_lam ? &lam : nullptr);
  } else if (rk == 3) {
    stage<Counted>(scheme, pde, P, dim, &pt, 1, halo, nv, q.data(), nullptr, u1.data(), nullptr, mat,
                   dt, 0, 1, 1, 0, 0.1, nullptr);
    stage<Counted>(scheme, pde, P, dim, &pt, 1, halo, nv, u1.data(), q.data(), u2.data(), nullptr,
                   mat, dt, 0.75, 0.25, 0.25, 0, 0.1, nullptr);
    stage<Counted>(scheme, pde, P, dim, &pt, 1, halo, nv, u2.data(), q.data(), q.data(), nullptr, mat,
                   dt, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, 0, 0.1, with_lam ? &lam : nullptr);
  } else if (rk == 4) {
    acc = q;
    stage<Counted>(scheme, pde, P, dim, &pt, 1, halo, nv, q.data(), q.data(), u1.data(), acc.data(),
                   mat, dt, 1, 0, 0.5, 1.0 / 6.0, 0.1, nullptr);
    stage<Counted>(scheme, pde, P, dim, &pt, 1, halo, nv, u1.data(), q.data(), u2.data(), acc.data(),
                   mat, dt, 1, 0, 0.5, 1.0 / 3.0, 0.1, nullptr);
    stage<Counted>(scheme, pde, P, dim, &pt, 1, halo, nv, u2.data(), q.data(), u1.data(), acc.data(),
                   mat, dt, 1, 0, 1.0, 1.0 / 3.0, 0.1, nullptr);
    stage<Counted>(scheme, pde, P, dim, &pt, 1, halo, nv, u1.data(), nullptr, nullptr, acc.data(), mat,
                   dt, 0, 0, 0, 1.0 / 6.0, 0.1, with_lam ? &lam : nullptr);
  }
  return g_flops;
}

}  // extern "C"
