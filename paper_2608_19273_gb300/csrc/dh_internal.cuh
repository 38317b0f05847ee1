// Internal declarations shared by the CUDA translation units of libdh.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/dh.h"

namespace dh {

// PDE parameters passed by value to every kernel.  one/mone/zero hold 1, -1
// and 0: kernels multiply or add them in fused multiply-adds so that plain
// adds and multiplies are issued as DFMA (see dh_pde.cuh).
struct DevParams {
  double one, mone, zero;
  double half;    // 0.5 as a run-time value (an FMA with it stays one FMA)
  double gamma;   // Euler ratio of specific heats
  double gm1;     // gamma - 1
  double Gamma;   // SRHD adiabatic index
  double Gq;      // Gamma / (Gamma - 1)
  double damp;    // wave-system damping
  double kappa;   // GW59 lapse coupling
  double C[121];  // GW59 coupling matrix, row-major
};

// One CTA's worth of work of the FV stage for patch sizes that are not multiples of 8: up to
// eight whole patches of equal p (ng groups, origin 0), one box of one patch (ng = 1) of
// bx x by x bz voxels from (x0, y0, z0), or (mp > 0) one box made of a 2x2x2 block of face-
// adjacent patches of mp^3 voxels (patch[mx + 2 my + 4 mz] holds block member (mx, my, mz)).
struct AnyWork {
  int32_t patch[8];
  int16_t x0, y0, z0;
  int8_t bx, by, bz, ng;
  int8_t mp;
};

// One CTA's worth of FV/FD work: up to 4 groups, each a (TX x TY) column of
// one patch that the CTA marches through all z-planes of that patch.
struct Work {
  int32_t cls;    // tile class: 0 = one 16x16 column; 1 = four 8x8 columns; 2 = one 32x8 column;
                  // 3 = one 8x8 column (a 64-thread CTA)
  int32_t pz;     // planes to march (p in 3D, 1 in 2D) ...
  int32_t z0;     // ... starting at this plane of the patch
  int32_t patch[4];
  int16_t x0[4];
  int16_t y0[4];
};

// Interior voxels per CTA of the AoAoS gather/scatter kernels (a multiple of
// every segment length, 8..64).
constexpr int AO_UNIT_VOXELS = 4096;

// Reflux entry of coupled refinement levels: coarse voxel eC of patch C next to
// fine patch F across F's face (axis, lo: C on F's -axis side), the covered
// coarse voxel eN of F's parent N across that face, and the first of the
// 2^(d-1) fine voxels eF of F on the face (the others at +sb0, +sb1, +sb0+sb1).
struct AmrReflux {
  int C, N, F;
  int eC, eN, eF;
  int sb0, sb1;
  int axis, lo;
};

// One FD tile: an 8x8x4 block of one patch.
struct FdWork {
  int32_t patch;
  int16_t x0, y0, z0, pad;
};

}  // namespace dh

struct dh_plan {
  int pde = 0, dim = 3, K = 0, halo = 1;
  int64_t var_stride = 0;
  int nq = 0, nm = 0;
  int device = 0;
  double dx_min = 0;
  dh::DevParams params{};
  std::vector<dh_patch> h_patches;
  dh_patch* d_patches = nullptr;
  // FV tile work lists (cost-descending), one per tile set and z-split, list 2 * tile + zs:
  //   tile set 0: 16x16 columns for p % 16 == 0, groups of four 8x8 columns otherwise;
  //            1: as 0, but 32x8 columns for p % 32 == 0;
  //            2: groups of four 8x8 columns for every patch (64 threads per column);
  //            3: one 8x8 column per 64-thread CTA for every patch (small problems: more CTAs);
  //   zs 1: columns of more than 16 planes march in chunks of <= 16 planes, and a thin
  //         last wave is filled with half-height chunks.
  static constexpr int NWL = 8;
  dh::Work* d_wl[NWL] = {};
  int n_wl[NWL] = {};
  bool wl_cls[NWL][4] = {};  // tile classes present in each list
  // kernel variants chosen by the autotuner.  fv_var bits 0-1: halo ring before the
  // mid-plane barrier, register cap for two CTAs per SM; bit 2: persistent grid with a tile
  // queue; bits 3-4: tile set
  int fv_var = 2, fv_zs = 0, fd_var = 0;
  int fv_list() const { return 2 * ((fv_var >> 3) & 3) + fv_zs; }
  // second-order FV stage: 0 = z-march of whole patches, 1 = z-march in chunks of <= 16 planes
  // (both on the work lists of tile set 0), 2 = 8x8x4 tiles
  int fv2_var = 2;  // second-order stage: 8x8x4 tiles (faster than the z-march on the measured mixes)
  // FD tile list (8x8x4 tiles)
  dh::FdWork* d_fdwork = nullptr;
  int n_fdwork = 0;
  // Patch sizes that are not all multiples of 8: the FV stage runs k_fv_any over d_any (the
  // FD, MUSCL and coupled-level paths, whose tiles need multiples of 8, refuse such plans).
  bool fv_generic = false;
  dh::AnyWork* d_any = nullptr;
  int n_any = 0;
  // levels for the TMA staging of the FD stage: maximal runs of patches of equal p
  // stored back to back (offset step p^3) whose face neighbours lie in the same run
  bool tma_ok = false;
  int n_lvl = 0;
  int lvl_p[8] = {0}, lvl_K[8] = {0};
  int64_t lvl_off[8] = {0};
  int2* d_lvl = nullptr;  // per patch: (level, index within the level)
  // AoAoS gather/scatter units: (patch, first voxel), up to AO_UNIT_VOXELS voxels each
  int2* d_aunits = nullptr;
  int n_aunits = 0;
  // coupled refinement levels (dh_amr.cu): octant bits per patch, reflux entries
  // grouped by face direction, (fine patch, parent) pairs finest level first
  bool coupled = false;
  int* d_amr_oct = nullptr;
  dh::AmrReflux* d_amr_reflux = nullptr;
  int amr_reflux_off[7] = {0, 0, 0, 0, 0, 0, 0};
  bool amr_reflux_single = false;  // no coarse voxel has entries in two directions: one launch
  int2* d_amr_restrict = nullptr;
  std::vector<int> amr_restrict_off;
  // derived quantities W (NW-variable arena) handed from the last stage of a time step to
  // the first stage of the next inside a captured multi-step graph (Euler systems)
  double* d_w = nullptr;  // two NW-variable arenas back to back (stage results alternate)
  // offload mode: device copy of the bound block pointer table (dh_offload_bind)
  double** d_offload = nullptr;
  int offload_nq = 0, offload_halo = 0;
  // staged offload (dh_offload_bind_staged): the host span of the blocks is copied
  // to / from a device staging buffer by the copy engine; the table points into it
  bool offload_staged = false;
  char* d_stage = nullptr;
  size_t stage_cap = 0, stage_bytes = 0;
  char* stage_host = nullptr;
  int debug_flags = 0;    // test hooks (bit 0: TMA barriers armed but no copy issued)
  // scratch: [0] running max (bit pattern of a non-negative double), [1] CTA ticket counter,
  // [2] error flags (bit 0: a bounded TMA wait gave up), [3] tile queue of a persistent FV
  // launch (two 32-bit words: next tile, CTAs done), [4..7] unused
  static constexpr int NRED = 8;
  unsigned long long* d_red = nullptr;
  int num_sms = 0;
  // set by the runtime around the last FV stage of a time step whose successor's dt that
  // stage computes in its lambda epilogue (multi-step sequences), NULL otherwise
  double* dt_fold = nullptr;
  double dt_fold_cfl = 0.0;
  // con2prim settings used by dh_rk_step for SRHD3D
  const float* c2p_mlp = nullptr;
  double c2p_tol = 1e-12;
  int c2p_max_iter = 50;
  int c2p_refine = 0;  // FP32 Newton steps applied to the first seed
  int32_t* c2p_fail = nullptr;
  // captured multi-step graph and optional per-stage timing events
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<cudaEvent_t> ev_start, ev_stop;
  int graph_stages = 0, graph_kernels = 0;
};

namespace dh {

void set_error(const char* fmt, ...);
dh_status cuda_error(cudaError_t e, const char* what);
int pde_nq(int pde);
int pde_nm(int pde);
int pde_dim(int pde);

// Fill the derived constants of DevParams (call after setting gamma, Gamma, ...).
inline void finish_params(DevParams& P) {
  P.one = 1.0;
  P.mone = -1.0;
  P.zero = 0.0;
  P.half = 0.5;
  P.gm1 = P.gamma - 1.0;
  P.Gq = P.Gamma / (P.Gamma - 1.0);
}

std::vector<int2> aoas_units(const dh_patch* patches, int K, int dim);
dh_status amr_build(dh_plan* plan, const dh_patch* patches, int K, int dim);
// Maximum characteristic speed from the derived quantities W of a state (Euler systems).
dh_status max_wave_speed_w(dh_plan* plan, const double* w, double* lam_out_dev, cudaStream_t s);
// form: as launch_fv_stage (0: acc += d dt L; 1-3: SSP-RK3 stage-sum form, acc = raw sums);
// w_out: the derived quantities of out written by the stage, refreshed for the voxels the
// coupling changes (NULL: none kept)
dh_status amr_couple(dh_plan* plan, const double* qs, const double* mat, double* out, double* acc,
                     const double* dt_dev, double g, double d, cudaStream_t s, int form = 0,
                     double* w_out = nullptr);
dh_status aoas_move(dh_plan* plan, bool gather, const double* const* blocks, int nq, int v0, int nv, int halo,
                    double* arena, cudaStream_t s);

// n_steps whole Runge-Kutta steps launched eagerly, with the same hand-over of derived
// quantities between stages that a captured multi-step graph uses (same kernels, same results).
dh_status rk_steps(dh_plan* plan, int scheme, int rk, int n_steps, double* q, double* u1, double* u2, double* acc,
                   const double* mat, double* dt, double* lam, double cfl, double sigma, cudaStream_t s);

dh_status launch_fd_stage(dh_plan* plan, const double* qs, const double* q0, double* out, double* acc,
                          const double* mat, const double* dt_dev, double a, double b, double g, double d,
                          double sigma, double* lam_out, cudaStream_t stream);

dh_status launch_fv2_stage(dh_plan* plan, const double* qs, const double* q0, double* out, double* acc,
                           const double* mat, const double* dt_dev, double a, double b, double g, double d,
                           double* lam_out, cudaStream_t stream);

// wmode: bit 0 reads the derived quantities W of qs from w_in, bit 1 writes W of the
// result to w_out (a different arena when both are set); 0 outside multi-step graphs.
// form: 0 for the general stage; 1-3 for stage 1-3 of SSP-RK3 in stage-sum form, acc
// holding the raw face-flux sum of the earlier stages (coupled plans: amr_couple with the
// same form follows).
dh_status launch_fv_stage(dh_plan* plan, const double* qs, const double* q0, double* out, double* acc,
                          const double* mat, const double* dt_dev, double a, double b, double g, double d,
                          double* lam_out, cudaStream_t stream, int wmode = 0, const double* w_in = nullptr,
                          double* w_out = nullptr, int form = 0);

}  // namespace dh
