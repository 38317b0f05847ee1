// Time-stepping runtime: whole Runge-Kutta steps built from stage calls, and
// their capture into a CUDA graph owned by the plan.
//
// A Runge-Kutta scheme calls the cell update several times per time step with
// tableau-dependent dt, with a face-neighbour synchronisation (halo refresh)
// between calls (paper Sec. II).  Here every stage is one batched launch over
// all patches; the halo refresh is implicit because each stage reads its halos
// from the previous stage's output in global memory.  dt lives in device
// memory and is recomputed on the device from the maximum wave speed that the
// last stage of the previous step produced, so a graph of many steps replays
// without any host round trip.
#include <algorithm>
#include <cstring>

#include <nvtx3/nvToolsExt.h>

#include "dh_internal.cuh"

namespace dh {

struct Timer;
// Hand-over of the derived quantities W from stage to stage inside a multi-step graph:
// stage j of the graph writes W of its result into buf[j % 2] and stage j + 1 (whose input
// that result is) reads it from there.
struct WChain {
  bool on = false;
  int next = 0, total = 0;
  double* buf[2] = {nullptr, nullptr};
};
static dh_status stage_call(dh_plan* plan, int scheme, const double* qs, const double* q0, double* out,
                            double* acc, const double* mat, const double* dt, double a, double b, double g,
                            double d, double sigma, double* lam, Timer& T, cudaStream_t s, WChain* wc = nullptr,
                            bool prims_current = false, int form = 0);

struct Timer {
  dh_plan* plan;
  bool on;
  cudaStream_t s;
  int next = 0;
  dh_status begin() {
    if (!on) return DH_OK;
    if (next >= (int)plan->ev_start.size()) { set_error("graph timing: too many stages"); return DH_EINVAL; }
    return cuda_error(cudaEventRecordWithFlags(plan->ev_start[next], s, cudaEventRecordExternal), "event record");
  }
  dh_status end() {
    if (!on) return DH_OK;
    dh_status st = cuda_error(cudaEventRecordWithFlags(plan->ev_stop[next], s, cudaEventRecordExternal), "event record");
    ++next;
    return st;
  }
};

#define DH_TRY(x) do { dh_status _st = (x); if (_st != DH_OK) return _st; } while (0)

// One stage launch, timed (when timing is on) around the stage kernel only.
static dh_status stage_call(dh_plan* plan, int scheme, const double* qs, const double* q0, double* out,
                            double* acc, const double* mat, const double* dt, double a, double b, double g,
                            double d, double sigma, double* lam, Timer& T, cudaStream_t s, WChain* wc,
                            bool prims_current, int form) {
  if (plan->pde == DH_PDE_SRHD3D) {
    // primitives of the stage input, seeded by the previous primitives (in place), unless
    // they were just recovered from this very input (the step start's wave speed)
    double* prim = const_cast<double*>(mat);
    if (!prims_current)
      DH_TRY(con2prim(plan, qs, prim, prim + 4 * plan->var_stride, plan->c2p_mlp, plan->c2p_tol, plan->c2p_max_iter,
                      plan->c2p_refine, nullptr, nullptr, plan->c2p_fail, s));
    lam = nullptr;
  }
  // NVTX range per stage (host-side marker for profilers; a no-op without one attached)
  struct Range {
    explicit Range(const char* n) { nvtxRangePushA(n); }
    ~Range() { nvtxRangePop(); }
  } range(scheme == 0 ? "dh FV stage" : (scheme == 2 ? "dh FV2 stage" : "dh FD stage"));
  DH_TRY(T.begin());
  if (scheme == 0 && (form || (wc && wc->on))) {
    int wmode = 0;
    const double* w_in = nullptr;
    double* w_out = nullptr;
    if (wc && wc->on) {
      const int j = wc->next++;
      wmode = (j > 0 ? 1 : 0) | (j + 1 < wc->total ? 2 : 0);
      w_in = wc->buf[(j + 1) & 1];
      w_out = wc->buf[j & 1];
    }
    DH_TRY(launch_fv_stage(plan, qs, q0, out, acc, mat, dt, a, b, g, d, plan->coupled ? nullptr : lam, s, wmode,
                           w_in, w_out, form));
    if (plan->coupled) {
      // reflux and restriction (refreshing W of the voxels they change), then the wave
      // speed of the coupled result
      DH_TRY(amr_couple(plan, qs, mat, out, acc, dt, g, d, s, form, (wmode & 2) ? w_out : nullptr));
      if (lam && (wmode & 2)) DH_TRY(max_wave_speed_w(plan, w_out, lam, s));
      else if (lam) DH_TRY(max_wave_speed(plan, out, mat, lam, s));
    }
  } else if (scheme == 0) DH_TRY(patch_update_fv(plan, qs, q0, out, acc, mat, dt, a, b, g, d, lam, s));
  else if (scheme == 2) DH_TRY(patch_update_fv_muscl(plan, qs, q0, out, acc, mat, dt, a, b, g, d, lam, s));
  else DH_TRY(patch_update_fd_ko(plan, qs, q0, out, acc, mat, dt, a, b, g, d, sigma, lam, s));
  return T.end();
}

// Whether the last FV stage of a step can compute the next step's dt in its lambda epilogue:
// its kernel publishes the wave speed of the step's result itself (not on coupled levels, where
// the speed is taken after the coupling, nor for SRHD, whose speed comes from the primitives).
static bool dt_foldable(const dh_plan* plan, int scheme, double cfl) {
  return scheme == 0 && cfl > 0 && !plan->coupled && plan->pde != DH_PDE_SRHD3D;
}

// Sets the plan's fold request for the duration of one stage call.
struct FoldScope {
  dh_plan* plan;
  FoldScope(dh_plan* p, double* dt, double cfl) : plan(p) {
    plan->dt_fold = dt;
    plan->dt_fold_cfl = cfl;
  }
  ~FoldScope() { plan->dt_fold = nullptr; }
};

// One time step.  bufs: q (state, in/out), u1, u2 (stage buffers), acc (RK4).
// In a sequence of steps: cfl_done -- the previous step's last stage already computed this
// step's dt; fold -- this step's last stage computes the next step's dt; fe_dst -- forward
// Euler writes the new state there (the caller alternates buffers) instead of into u1 and
// copying it back to q.
static dh_status rk_step(dh_plan* plan, int scheme, int rk, double* q, double* u1, double* u2, double* acc,
                         const double* mat, double* dt, double* lam, double cfl, double sigma, Timer& T,
                         cudaStream_t s, WChain* wc = nullptr, bool cfl_done = false, bool fold = false,
                         double* fe_dst = nullptr) {
  const size_t bytes = sizeof(double) * (size_t)plan->nq * (size_t)plan->var_stride;
  double* lam_last = cfl > 0 ? lam : nullptr;
  double* const fold_dt = fold ? dt : nullptr;
  // SRHD: with a CFL step the primitives of q are recovered here for the wave speed and
  // then serve the first stage as well
  const bool srhd_cur = cfl > 0 && plan->pde == DH_PDE_SRHD3D;
  if (cfl > 0 && plan->pde == DH_PDE_SRHD3D) {
    // the wave speed needs the primitives of q: recover them, then take the maximum
    double* prim = const_cast<double*>(mat);
    DH_TRY(con2prim(plan, q, prim, prim + 4 * plan->var_stride, plan->c2p_mlp, plan->c2p_tol, plan->c2p_max_iter,
                    plan->c2p_refine, nullptr, nullptr, plan->c2p_fail, s));
    DH_TRY(max_wave_speed(plan, q, prim, lam, s));
  }
  if (cfl > 0 && !cfl_done) DH_TRY(dh_cfl_dt(plan, lam, cfl, dt, s));
  if (rk == 1) {
    double* dst = fe_dst ? fe_dst : u1;
    {
      FoldScope f(plan, fold_dt, cfl);
      DH_TRY(stage_call(plan, scheme, q, nullptr, dst, nullptr, mat, dt, 0, 1, 1, 0, sigma, lam_last, T, s, nullptr,
                        srhd_cur));
    }
    if (!fe_dst) DH_TRY(cuda_error(cudaMemcpyAsync(q, u1, bytes, cudaMemcpyDeviceToDevice, s), "copy u1 -> q"));
  } else if (rk == 3 && scheme == 0 && acc) {
    // the stage-sum form of the same scheme: acc carries the raw face-flux sum of the earlier stages
    DH_TRY(stage_call(plan, scheme, q, nullptr, u1, acc, mat, dt, 0, 1, 1, 0, sigma, nullptr, T, s, wc, srhd_cur, 1));
    DH_TRY(stage_call(plan, scheme, u1, q, u2, acc, mat, dt, 0, 0, 0.25, 0, sigma, nullptr, T, s, wc, false, 2));
    FoldScope f(plan, fold_dt, cfl);
    DH_TRY(stage_call(plan, scheme, u2, q, q, acc, mat, dt, 0, 0, 2.0 / 3.0, 1.0 / 6.0, sigma, lam_last, T, s, wc,
                      false, 3));
  } else if (rk == 3) {
    DH_TRY(stage_call(plan, scheme, q, nullptr, u1, nullptr, mat, dt, 0, 1, 1, 0, sigma, nullptr, T, s, wc, srhd_cur));
    DH_TRY(stage_call(plan, scheme, u1, q, u2, nullptr, mat, dt, 0.75, 0.25, 0.25, 0, sigma, nullptr, T, s, wc));
    FoldScope f(plan, fold_dt, cfl);
    DH_TRY(stage_call(plan, scheme, u2, q, q, nullptr, mat, dt, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, 0, sigma, lam_last,
                      T, s, wc));
  } else if (rk == 4) {
    DH_TRY(cuda_error(cudaMemcpyAsync(acc, q, bytes, cudaMemcpyDeviceToDevice, s), "copy q -> acc"));
    DH_TRY(stage_call(plan, scheme, q, nullptr, u1, acc, mat, dt, 0, 1, 0.5, 1.0 / 6.0, sigma, nullptr, T, s, nullptr,
                      srhd_cur));
    DH_TRY(stage_call(plan, scheme, u1, q, u2, acc, mat, dt, 1, 0, 0.5, 1.0 / 3.0, sigma, nullptr, T, s));
    DH_TRY(stage_call(plan, scheme, u2, q, u1, acc, mat, dt, 1, 0, 1.0, 1.0 / 3.0, sigma, nullptr, T, s));
    {
      FoldScope f(plan, fold_dt, cfl);
      DH_TRY(stage_call(plan, scheme, u1, nullptr, nullptr, acc, mat, dt, 0, 0, 0, 1.0 / 6.0, sigma, lam_last, T, s));
    }
    DH_TRY(cuda_error(cudaMemcpyAsync(q, acc, bytes, cudaMemcpyDeviceToDevice, s), "copy acc -> q"));
  } else {
    set_error("dh_rk_step: rk must be 1, 3 or 4");
    return DH_EINVAL;
  }
  return DH_OK;
}

// n_steps consecutive steps: from the second step on, each step's dt is computed by the
// previous step's last stage (where foldable), and forward Euler alternates between q and u1
// instead of copying every step's result back to q (one copy at the end if n_steps is odd).
static dh_status rk_sequence(dh_plan* plan, int scheme, int rk, int n_steps, double* q, double* u1, double* u2,
                             double* acc, const double* mat, double* dt, double* lam, double cfl, double sigma,
                             Timer& T, cudaStream_t s, WChain* wc) {
  const bool fold = dt_foldable(plan, scheme, cfl);
  const bool pingpong = rk == 1 && n_steps > 1;
  double* cur = q;
  double* oth = u1;
  for (int i = 0; i < n_steps; ++i) {
    const bool done = fold && i > 0, next = fold && i + 1 < n_steps;
    if (pingpong) {
      DH_TRY(rk_step(plan, scheme, rk, cur, oth, u2, acc, mat, dt, lam, cfl, sigma, T, s, nullptr, done, next, oth));
      std::swap(cur, oth);
    } else {
      DH_TRY(rk_step(plan, scheme, rk, q, u1, u2, acc, mat, dt, lam, cfl, sigma, T, s, wc, done, next));
    }
  }
  if (cur != q) {
    const size_t bytes = sizeof(double) * (size_t)plan->nq * (size_t)plan->var_stride;
    DH_TRY(cuda_error(cudaMemcpyAsync(q, cur, bytes, cudaMemcpyDeviceToDevice, s), "copy result -> q"));
  }
  return DH_OK;
}

static dh_status check_rk(dh_plan* plan, int scheme, int rk, double* q, double* u1, double* u2, double* acc,
                          const double* mat, double* dt, double* lam, double cfl) {
  if (!plan) { set_error("plan is NULL"); return DH_EINVAL; }
  if (scheme < 0 || scheme > 2) { set_error("scheme must be 0 (FV), 1 (FD) or 2 (FV, MUSCL)"); return DH_EINVAL; }
  if (!q || !u1 || !dt || (rk == 3 && !u2) || (rk == 4 && (!u2 || !acc))) {
    set_error("dh_rk_step: missing state or stage buffer");
    return DH_EINVAL;
  }
  if (cfl > 0 && !lam) { set_error("dh_rk_step: cfl > 0 needs lam_dev"); return DH_EINVAL; }
  if (acc && (acc == q || acc == u1 || acc == u2)) { set_error("dh_rk_step: acc aliases a state buffer"); return DH_EINVAL; }
  if (plan->pde == DH_PDE_SRHD3D && !mat) { set_error("dh_rk_step: SRHD3D needs the primitive arena as mat"); return DH_EINVAL; }
  if (rk != 1 && rk != 3 && rk != 4) { set_error("dh_rk_step: rk must be 1, 3 or 4"); return DH_EINVAL; }
  if (plan->fv_generic && scheme != 0) {
    set_error("dh_rk_step: FD and MUSCL stages need patch sizes that are multiples of 8");
    return DH_EUNSUPPORTED;
  }
  return DH_OK;
}

// Whether n consecutive steps hand the derived quantities W of each stage result to the next
// stage (SSP-RK3 FV steps of the Euler systems with a device-side CFL step).
static bool w_reuse(dh_plan* plan, int scheme, int rk, int n_steps, double cfl) {
  return scheme == 0 && rk == 3 && cfl > 0 && n_steps > 1 &&
         (plan->pde == DH_PDE_EULER2D || plan->pde == DH_PDE_EULER3D);
}

// The plan's two W arenas (allocated once, on first use, and kept by the plan).
static dh_status w_chain(dh_plan* plan, int n_steps, WChain& wc) {
  const size_t nw = (size_t)(plan->dim + 3) * (size_t)plan->var_stride;
  if (!plan->d_w) DH_TRY(cuda_error(cudaMalloc(&plan->d_w, 2 * sizeof(double) * nw), "W arenas"));
  wc.on = true;
  wc.next = 0;
  wc.total = 3 * n_steps;
  wc.buf[0] = plan->d_w;
  wc.buf[1] = plan->d_w + nw;
  return DH_OK;
}

dh_status rk_steps(dh_plan* plan, int scheme, int rk, int n_steps, double* q, double* u1, double* u2, double* acc,
                   const double* mat, double* dt, double* lam, double cfl, double sigma, cudaStream_t s) {
  DH_TRY(check_rk(plan, scheme, rk, q, u1, u2, acc, mat, dt, lam, cfl));
  Timer T{plan, false, s};
  WChain wc;
  if (w_reuse(plan, scheme, rk, n_steps, cfl)) DH_TRY(w_chain(plan, n_steps, wc));
  return rk_sequence(plan, scheme, rk, n_steps, q, u1, u2, acc, mat, dt, lam, cfl, sigma, T, s, wc.on ? &wc : nullptr);
}

}  // namespace dh

using namespace dh;

extern "C" {

dh_status dh_plan_set_con2prim(dh_plan* plan, const float* mlp_w, double tol, int32_t max_iter,
                               int32_t seed_refine, int32_t* fail_count_dev) {
  if (!plan) { set_error("plan is NULL"); return DH_EINVAL; }
  if (!(tol > 0.0) || max_iter < 1 || max_iter > 1000 || seed_refine < 0 || seed_refine > 8) {
    set_error("dh_plan_set_con2prim: bad tol, max_iter or seed_refine");
    return DH_EINVAL;
  }
  plan->c2p_mlp = mlp_w;
  plan->c2p_tol = tol;
  plan->c2p_max_iter = max_iter;
  plan->c2p_refine = seed_refine;
  plan->c2p_fail = fail_count_dev;
  return DH_OK;
}

dh_status dh_rk_step(dh_plan* plan, int32_t scheme, int32_t rk, double* q, double* u1, double* u2, double* acc,
                     const double* mat, double* dt_dev, double* lam_dev, double cfl, double sigma_ko,
                     void* stream) {
  DH_TRY(check_rk(plan, scheme, rk, q, u1, u2, acc, mat, dt_dev, lam_dev, cfl));
  Timer T{plan, false, (cudaStream_t)stream};
  return rk_step(plan, scheme, rk, q, u1, u2, acc, mat, dt_dev, lam_dev, cfl, sigma_ko, T, (cudaStream_t)stream);
}

dh_status dh_graph_capture(dh_plan* plan, int32_t scheme, int32_t rk, int32_t n_steps, double* q, double* u1,
                           double* u2, double* acc, const double* mat, double* dt_dev, double* lam_dev, double cfl,
                           double sigma_ko, int32_t timing, void* stream) {
  DH_TRY(check_rk(plan, scheme, rk, q, u1, u2, acc, mat, dt_dev, lam_dev, cfl));
  if (n_steps <= 0 || n_steps > 100000) { set_error("dh_graph_capture: n_steps out of range"); return DH_EINVAL; }
  if (!stream) { set_error("dh_graph_capture: needs a non-default stream"); return DH_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  // release a previous graph and timing events
  if (plan->graph_exec) { cudaGraphExecDestroy(plan->graph_exec); plan->graph_exec = nullptr; }
  for (cudaEvent_t e : plan->ev_start) cudaEventDestroy(e);
  for (cudaEvent_t e : plan->ev_stop) cudaEventDestroy(e);
  plan->ev_start.clear();
  plan->ev_stop.clear();
  const int stages = (rk == 1 ? 1 : rk) * n_steps;
  if (timing) {
    for (int i = 0; i < stages; ++i) {
      cudaEvent_t a, b;
      DH_TRY(cuda_error(cudaEventCreate(&a), "cudaEventCreate"));
      DH_TRY(cuda_error(cudaEventCreate(&b), "cudaEventCreate"));
      plan->ev_start.push_back(a);
      plan->ev_stop.push_back(b);
    }
  }
  // hand the derived quantities of the state from one step to the next (SSP-RK3 FV, Euler)
  WChain wc;
  if (w_reuse(plan, scheme, rk, n_steps, cfl)) DH_TRY(w_chain(plan, n_steps, wc));
  DH_TRY(cuda_error(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture"));
  Timer T{plan, timing != 0, s};
  dh_status st = rk_sequence(plan, scheme, rk, n_steps, q, u1, u2, acc, mat, dt_dev, lam_dev, cfl, sigma_ko, T, s,
                             wc.on ? &wc : nullptr);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &graph);
  if (st != DH_OK) { if (graph) cudaGraphDestroy(graph); return st; }
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&plan->graph_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) { plan->graph_exec = nullptr; return cuda_error(e, "cudaGraphInstantiate"); }
  plan->graph_stages = timing ? stages : 0;
  const int nst = rk == 1 ? 1 : rk;
  const int srhd = plan->pde == DH_PDE_SRHD3D;
  // coupled levels: per stage one reflux launch per face direction in use and one restriction
  // launch per level; the last stage's wave speed is a separate launch
  int cpl = 0;
  if (plan->coupled && scheme == 0) {
    if (plan->amr_reflux_single) cpl += plan->amr_reflux_off[6] > 0;
    else
      for (int f = 0; f < 6; ++f) cpl += plan->amr_reflux_off[f + 1] > plan->amr_reflux_off[f];
    for (size_t l = 0; l + 1 < plan->amr_restrict_off.size(); ++l)
      cpl += plan->amr_restrict_off[l + 1] > plan->amr_restrict_off[l];
  }
  const int cpl_lam = plan->coupled && scheme == 0 && cfl > 0 && !srhd;
  // the CFL step: one launch per step, or only the first step's where later steps take their dt
  // from the previous step's last stage
  const int cfl_steps = cfl > 0 ? (dt_foldable(plan, scheme, cfl) ? 1 : n_steps) : 0;
  plan->graph_kernels = n_steps * nst * (1 + srhd + cpl) + cfl_steps * (1 + srhd + cpl_lam);
  return DH_OK;
}

dh_status dh_graph_launch(dh_plan* plan, void* stream) {
  if (!plan || !plan->graph_exec) { set_error("dh_graph_launch: no captured graph"); return DH_EINVAL; }
  return cuda_error(cudaGraphLaunch(plan->graph_exec, (cudaStream_t)stream), "cudaGraphLaunch");
}

dh_status dh_graph_info(dh_plan* plan, int32_t* n_kernels, int32_t* n_timed_stages) {
  if (!plan || !plan->graph_exec) { set_error("dh_graph_info: no captured graph"); return DH_EINVAL; }
  if (n_kernels) *n_kernels = plan->graph_kernels;
  if (n_timed_stages) *n_timed_stages = plan->graph_stages;
  return DH_OK;
}

dh_status dh_graph_stage_times(dh_plan* plan, float* ms_out, int32_t n) {
  if (!plan || !ms_out || n < 0 || n > plan->graph_stages) {
    set_error("dh_graph_stage_times: bad arguments or graph captured without timing");
    return DH_EINVAL;
  }
  for (int i = 0; i < n; ++i) {
    cudaError_t e = cudaEventElapsedTime(&ms_out[i], plan->ev_start[i], plan->ev_stop[i]);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventElapsedTime");
  }
  return DH_OK;
}

}  // extern "C"
