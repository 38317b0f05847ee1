// First-order FV stage for plans with patch sizes that are not multiples of 8 (the paper's
// typical 3^3 and 6^3 cells, Sec. IV): the same operator as the z-marching stage (Rusanov face
// flux and non-conservative product of Sec. II-A Eq. 3, the stage combination and the lambda
// epilogue), in a simpler tiling that fits any p.
//
// A CTA of 256 threads takes one work item: up to eight whole small patches of equal p (each
// patch a group), a 2x2x2 block of face-adjacent 3^3 patches as one 6^3 box, or one box of a
// larger patch (6x6x6, 7x7x4 or 8x8x3 voxels in 3D, 16x15 or 15x16 in 2D, smaller at the patch's
// upper ends).  One voxel per thread.  Every item keeps within the limits below (checked on the
// host when the plan is made).
//   1. Every cell of the box and its one-voxel face halo (edges and corners are never read) is
//      loaded into shared memory with its derived quantities W (read from the W arena of the
//      stage input, or computed).
//   2. Per direction d: every line cell of d (the box and its halo layers at both ends along d) forms
//      its flux F_d and speed lambda_d into the line arrays; after a barrier every face along d
//      is formed once (one per thread) into the face arrays; after another barrier every voxel
//      adds the difference of its two faces.
//   3. The stage combination, W of the result and lambda of the result as in the marching stage.
// Shared memory: box cells x (N + M quantities, W), line cells x (F_d, lambda_d), faces x (the
// face values, and the non-conservative products of NCP systems); 70.7 KB for the Euler
// equations in 3D, three CTAs per SM.
#pragma once

namespace dh {

constexpr int ANY_NT = 256;      // threads per CTA; voxels per item at most
constexpr int ANY_SLOTS = 512;   // box cells with halo (all groups) per item
constexpr int ANY_LINES = 320;   // line cells of one direction per item
constexpr int ANY_FACES = 256;   // faces of one direction per item (one per thread)

// Integer division by a run-time divisor without the integer divide sequence: for
// 0 <= n < 2^15 and 1 <= d < 2^24, (n + 1/2)/d is never an integer and lies at least 1/(2n + 1)
// (relative) from one, while (n + 1/2) * fl(1/d) in float errs by at most 2^-23 (relative):
// truncation gives floor(n/d) exactly.  Every cell, face and group index here is below 2^10.
struct ADiv {
  int d;
  float r;
  __device__ explicit ADiv(int d_) : d(d_), r(1.0f / (float)d_) {}  // IEEE-rounded quotient
  __device__ int q(int n) const { return (int)(((float)n + 0.5f) * r); }
};

template <class PDE>
struct FvAny {
  static constexpr int N = PDE::N, NV = PDE::N + PDE::M, NW = PDE::NW > 0 ? PDE::NW : 1, DIM = PDE::DIM;
  static constexpr int NF = PDE::NCP ? 2 : 1;  // face arrays: flux (and non-conservative product)
  static constexpr size_t SMEM =
      sizeof(double) * ((size_t)ANY_SLOTS * (NV + NW) + (size_t)ANY_LINES * (N + 1) + (size_t)ANY_FACES * NF * N);

  template <int WM>
  __device__ static void run(const FvArgs& A, const AnyWork& w, double* smem, double& lam_thread) {
    double* Q = smem;                 // [NV][ANY_SLOTS]: box cells
    double* Wc = Q + NV * ANY_SLOTS;  // [NW][ANY_SLOTS]
    double* F = Wc + NW * ANY_SLOTS;  // [N][ANY_LINES]: line cells of one direction
    double* L = F + N * ANY_LINES;    // [ANY_LINES]
    double* H = L + ANY_LINES;        // [N][ANY_FACES]: face values of one direction
    double* Dn = H + N * ANY_FACES;   // [N][ANY_FACES]: non-conservative products (NCP systems)
    const DevParams& P = A.P;
    const int bx = w.bx, by = w.by, bz = DIM == 3 ? w.bz : 1, ng = w.ng;
    const int SX = bx + 2, SY = by + 2, SZ = DIM == 3 ? bz + 2 : 1;
    const int SG = SX * SY * SZ;  // cells per group
    const int nvg = bx * by * bz;  // voxels per group
    const int tid = threadIdx.x;
    const int g = tid / nvg, li = tid % nvg;
    const bool act = g < ng;
    const int lx = li % bx, ly = (li / bx) % by, lz = li / (bx * by);
    const int p = A.patches[w.patch[0]].p;  // every group or block member of an item has the same p
    const double dt = *A.dt_dev;             // read before the lambda epilogue may rewrite it
    const double gdt = A.g * dt, ddt = A.d * dt;

    // 1. the box and its face halo, with W: the cells that are read, enumerated group by group as
    //    the box (x fastest), then the two halo layers across x, y and z (edges and corners are
    //    never read and never visited)
    const int HX = by * bz, HY = bx * bz, HZ = DIM == 3 ? bx * by : 0;
    const int CG = nvg + 2 * (HX + HY + HZ);  // cells read per group
    const ADiv dCG(CG), dBX(bx), dBXY(bx * by), dBY(by), dHX(HX), dHY(HY), dHZ(HZ > 0 ? HZ : 1);
    for (int j = tid; j < ng * CG; j += ANY_NT) {
      const int gg = dCG.q(j);
      int r = j - gg * CG, cx, cy, cz;
      if (r < nvg) {
        cz = DIM == 3 ? dBXY.q(r) : 0;
        const int rxy = r - cz * bx * by;
        cy = dBX.q(rxy);
        cx = rxy - cy * bx;
      } else if ((r -= nvg) < 2 * HX) {
        const int side = dHX.q(r), t = r - side * HX;
        cx = side ? bx : -1;
        cz = dBY.q(t);
        cy = t - cz * by;
      } else if ((r -= 2 * HX) < 2 * HY) {
        const int side = dHY.q(r), t = r - side * HY;
        cy = side ? by : -1;
        cz = dBX.q(t);
        cx = t - cz * bx;
      } else {
        r -= 2 * HY;
        const int side = dHZ.q(r), t = r - side * HZ;
        cz = side ? bz : -1;
        cy = dBX.q(t);
        cx = t - cy * bx;
      }
      const int s = gg * SG + ((DIM == 3 ? cz + 1 : 0) * SY + (cy + 1)) * SX + (cx + 1);
      int64_t e;
      if (w.mp > 0) {
        // a 2x2x2 block of mp^3 patches: the member holding the cell, and the cell's
        // coordinates in it (at most one outside [0, mp): a face neighbour of that member)
        const int mx = cx >= w.mp, my = cy >= w.mp, mz = cz >= w.mp;
        e = vox_index(A.patches, nullptr, __ldg(w.patch + mx + 2 * my + 4 * mz), w.mp, cx - mx * w.mp,
                      cy - my * w.mp, cz - mz * w.mp);
      } else {
        e = vox_index(A.patches, nullptr, __ldg(w.patch + gg), p, w.x0 + cx, w.y0 + cy, DIM == 3 ? w.z0 + cz : 0);
      }
      double q[NV], W[NW];
#pragma unroll
      for (int v = 0; v < N; ++v) q[v] = __ldg(A.qs + v * A.vs + e);
#pragma unroll
      for (int v = 0; v < PDE::M; ++v) q[N + v] = __ldg(A.mat + v * A.vs + e);
      if (WM & 1) {
#pragma unroll
        for (int i = 0; i < NW; ++i) W[i] = __ldg(A.w_in + i * A.vs + e);
      } else {
        PDE::prims(q, P, W);
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) Q[v * ANY_SLOTS + s] = q[v];
#pragma unroll
      for (int i = 0; i < NW; ++i) Wc[i * ANY_SLOTS + s] = W[i];
    }
    __syncthreads();

    // 2. per direction: line fluxes and speeds, then this voxel's two faces
    const int me = g * SG + ((DIM == 3 ? lz + 1 : 0) * SY + (ly + 1)) * SX + (lx + 1);
    double sum[N], dsum[N];
#pragma unroll
    for (int v = 0; v < N; ++v) { sum[v] = 0.0; dsum[v] = 0.0; }
#pragma unroll 1
    for (int d = 0; d < DIM; ++d) {
      // the line cells of d (the box and the halo layer at each of its ends along d) of every
      // group, x fastest; their fluxes and speeds go to the line arrays at index j
      const int LX = bx + 2 * (d == 0), LY = by + 2 * (d == 1), LZ = DIM == 3 ? bz + 2 * (d == 2) : 1;
      const int LG = LX * LY * LZ;
      const ADiv dLG(LG), dLX(LX), dLY(LY);
      for (int j = tid; j < ng * LG; j += ANY_NT) {
        const int gg = dLG.q(j), r = j - gg * LG, t = dLX.q(r), hi = dLY.q(t);
        const int cx = r - t * LX - (d == 0), cy = t - hi * LY - (d == 1), cz = hi - (d == 2);
        const int s = gg * SG + ((DIM == 3 ? cz + 1 : 0) * SY + (cy + 1)) * SX + (cx + 1);
        double q[NV], W[NW], Fd[N];
#pragma unroll
        for (int v = 0; v < NV; ++v) q[v] = Q[v * ANY_SLOTS + s];
#pragma unroll
        for (int i = 0; i < NW; ++i) W[i] = Wc[i * ANY_SLOTS + s];
        if (PDE::FLUX) {
          PDE::flux(d, q, W, P, Fd);
#pragma unroll
          for (int v = 0; v < N; ++v) F[v * ANY_LINES + j] = Fd[v];
        }
        L[j] = PDE::speed(d, q, W, P);
      }
      __syncthreads();
      // every face along d once, one per thread, in x-fastest order (consecutive threads touch
      // consecutive cells: no shared-memory bank conflicts in any direction).  The face grid is
      // the voxel grid with one more layer along d: the face at c_d = pos lies between the cells
      // at pos - 1 and pos (pos = 0 and pos = b_d take a halo cell).
      const int FX = bx + (d == 0), FY = by + (d == 1), FZ = DIM == 3 ? bz + (d == 2) : 1;
      const int FG = FX * FY * FZ;  // faces per group
      {
        const int st = d == 0 ? 1 : (d == 1 ? SX : SX * SY), lst = d == 0 ? 1 : (d == 1 ? LX : LX * LY);
        const ADiv dFG(FG), dFX(FX), dFY(FY);
        const int fi = tid;
        if (fi < ng * FG) {
          const int gg = dFG.q(fi), r = fi - gg * FG, t = dFX.q(r), cz = dFY.q(t);
          const int cx = r - t * FX, cy = t - cz * FY;
          const int cR = gg * SG + ((DIM == 3 ? cz + 1 : 0) * SY + (cy + 1)) * SX + (cx + 1), cLf = cR - st;
          // the same two cells in the line arrays (line coordinates are shifted by one along d)
          const int jR = gg * LG + ((DIM == 3 ? cz + (d == 2) : 0) * LY + (cy + (d == 1))) * LX + (cx + (d == 0));
          const int jL = jR - lst;
          const double sf = max_nn(L[jL], L[jR]);
          double dq[N];
#pragma unroll
          for (int v = 0; v < N; ++v) {
            dq[v] = SUB(P, Q[v * ANY_SLOTS + cR], Q[v * ANY_SLOTS + cLf]);
            H[v * ANY_FACES + fi] = PDE::FLUX ? fma(-sf, dq[v], ADD(P, F[v * ANY_LINES + jL], F[v * ANY_LINES + jR]))
                                              : MUL(P, -sf, dq[v]);
          }
          if (PDE::NCP) {
            double qb[NV], Dv[N];
#pragma unroll
            for (int v = 0; v < NV; ++v) qb[v] = MUL(P, 0.5, ADD(P, Q[v * ANY_SLOTS + cLf], Q[v * ANY_SLOTS + cR]));
            PDE::ncp(d, qb, dq, P, Dv);
#pragma unroll
            for (int v = 0; v < N; ++v) Dn[v * ANY_FACES + fi] = Dv[v];
          }
        }
      }
      __syncthreads();
      if (act) {
        // this voxel's two faces along d: face coordinates pos = l_d and l_d + 1
        const int fm = g * FG + ((DIM == 3 ? lz : 0) * FY + ly) * FX + lx;
        const int fp = fm + (d == 0 ? 1 : (d == 1 ? FX : FX * FY));
#pragma unroll
        for (int v = 0; v < N; ++v) {
          sum[v] = ADD(P, sum[v], SUB(P, H[v * ANY_FACES + fp], H[v * ANY_FACES + fm]));
          if (PDE::NCP) dsum[v] = ADD(P, dsum[v], ADD(P, Dn[v * ANY_FACES + fp], Dn[v * ANY_FACES + fm]));
        }
      }
      // (the next direction writes F and L first, which no thread reads any more, then -- after a
      // barrier -- H)
    }

    // 3. stage combination, W and lambda of the result
    if (!act) return;
    int k, x, y, z;
    if (w.mp > 0) {
      const int mx = lx >= w.mp, my = ly >= w.mp, mz = lz >= w.mp;
      k = __ldg(w.patch + mx + 2 * my + 4 * mz);
      x = lx - mx * w.mp; y = ly - my * w.mp; z = lz - mz * w.mp;
    } else {
      k = __ldg(w.patch + g);
      x = w.x0 + lx; y = w.y0 + ly; z = DIM == 3 ? w.z0 + lz : 0;
    }
    const double cL = -0.5 / A.patches[k].dx;  // faces hold twice the flux
    const double cS = gdt * cL, cA = ddt * cL;
    const bool b1 = A.b == 1.0;
    const int pk = w.mp > 0 ? w.mp : p;
    const int64_t e = A.patches[k].offset + ((int64_t)z * pk + y) * pk + x;
    double Qk[NV], Sv[N], res[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Qk[v] = Q[v * ANY_SLOTS + me];
    if (PDE::SRC) {
      double Wk[NW];
      PDE::prims(Qk, P, Wk);
      PDE::source(Qk, Wk, P, Sv);
    }
#pragma unroll
    for (int v = 0; v < N; ++v) {
      const double s = PDE::NCP ? ADD(P, sum[v], dsum[v]) : sum[v];
      const int64_t ev = v * A.vs + e;
      if (!PDE::SRC && A.form != 0) {
        double o;
        if (A.form == 1) {
          o = fma(cS, s, Qk[v]);
          A.acc[ev] = s;
        } else if (A.form == 2) {
          const double t = ADD(P, A.acc[ev], s);
          o = fma(cS, t, __ldg(A.q0 + ev));
          A.acc[ev] = t;
        } else {
          o = fma(cS, s, fma(cA, A.acc[ev], __ldg(A.q0 + ev)));
        }
        res[v] = o;
        A.out[ev] = o;
        continue;
      }
      if (A.out) {
        double base = b1 ? Qk[v] : MUL(P, A.b, Qk[v]);
        if (A.q0) base = fma(A.a, __ldg(A.q0 + ev), base);
        res[v] = PDE::SRC ? fma(gdt, fma(cL, s, Sv[v]), base) : fma(cS, s, base);
      }
      if (A.acc) {
        const double r = PDE::SRC ? fma(ddt, fma(cL, s, Sv[v]), A.acc[ev]) : fma(cA, s, A.acc[ev]);
        A.acc[ev] = r;
        if (!A.out) res[v] = r;
      }
      if (A.out) A.out[ev] = res[v];
    }
    if (A.lam_out || (WM & 2)) {
#pragma unroll
      for (int v = N; v < NV; ++v) res[v] = Qk[v];
      double Wr[NW];
      PDE::prims(res, P, Wr);
      if (WM & 2) {
#pragma unroll
        for (int i = 0; i < NW; ++i) A.w_out[i * A.vs + e] = Wr[i];
      }
      if (A.lam_out) {
        double l = max_nn(PDE::speed(0, res, Wr, P), PDE::speed(1, res, Wr, P));
        if (DIM == 3) l = max_nn(l, PDE::speed(2, res, Wr, P));
        lam_thread = max_nn(lam_thread, l);
      }
    }
  }
};

template <class PDE, int WM>
__global__ void __launch_bounds__(ANY_NT) k_fv_any(const __grid_constant__ FvArgs A, const AnyWork* __restrict__ work) {
  extern __shared__ __align__(128) double smem[];
  double lam = 0.0;
  FvAny<PDE>::template run<WM>(A, work[blockIdx.x], smem, lam);
  if (A.lam_out) publish_lambda(lam, A.lam_out, A.red, A.dt_next, A.cfl, A.dx_dim);
}

template <class PDE, int WM>
static dh_status launch_any_wm(dh_plan* plan, const FvArgs& A, cudaStream_t stream) {
  constexpr size_t smem = FvAny<PDE>::SMEM;
  static int configured_device = -1;
  if (configured_device != plan->device) {
    cudaError_t e = cudaFuncSetAttribute(k_fv_any<PDE, WM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(k_fv_any)");
    configured_device = plan->device;
  }
  if (plan->n_any <= 0) return DH_OK;
  k_fv_any<PDE, WM><<<plan->n_any, ANY_NT, smem, stream>>>(A, plan->d_any);
  return cuda_error(cudaGetLastError(), "k_fv_any launch");
}

template <class PDE>
static dh_status launch_any(dh_plan* plan, const FvArgs& A, int wmode, cudaStream_t stream) {
  if constexpr (std::is_same<PDE, PdeEuler2>::value || std::is_same<PDE, PdeEuler3>::value) {
    switch (wmode & 3) {
      case 1: return launch_any_wm<PDE, 1>(plan, A, stream);
      case 2: return launch_any_wm<PDE, 2>(plan, A, stream);
      case 3: return launch_any_wm<PDE, 3>(plan, A, stream);
      default: break;
    }
  }
  return launch_any_wm<PDE, 0>(plan, A, stream);
}

}  // namespace dh
