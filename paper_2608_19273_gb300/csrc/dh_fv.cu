// Finite-volume stage: argument checks and dispatch on the plan's PDE (the kernels are
// in dh_fv_stage.cuh, instantiated by dh_fv_<pde>.cu).
#include "dh_fv_stage.cuh"

namespace dh {

dh_status launch_fv_stage(dh_plan* plan, const double* qs, const double* q0, double* out, double* acc,
                          const double* mat, const double* dt_dev, double a, double b, double g, double d,
                          double* lam_out, cudaStream_t stream, int wmode, const double* w_in, double* w_out,
                          int form) {
  // a stage that reads and writes W needs two arenas: other CTAs read halo W of the input
  if (((wmode & 1) && !w_in) || ((wmode & 2) && !w_out) || (wmode == 3 && w_in == w_out)) {
    set_error("launch_fv_stage: W arenas missing or aliased");
    return DH_EINVAL;
  }
  if (form < 0 || form > 3 || (form && (!acc || !out || (form > 1 && !q0)))) {
    set_error("launch_fv_stage: stage-sum form %d needs acc, out (and q0)", form);
    return DH_EINVAL;
  }
  FvArgs A;
  A.patches = plan->d_patches;
  A.work = nullptr;
  A.queue = nullptr;
  A.n_work = 0;
  A.qs = qs; A.q0 = q0; A.out = out; A.acc = acc; A.mat = mat; A.dt_dev = dt_dev;
  A.a = a; A.b = b; A.g = g; A.d = d;
  A.lam_out = lam_out;
  // a multi-step sequence asks the last stage of a step to compute the next step's dt
  A.dt_next = lam_out ? plan->dt_fold : nullptr;
  A.cfl = plan->dt_fold_cfl;
  A.dx_dim = plan->dx_min / plan->dim;
  A.red = plan->d_red;
  A.oct = plan->coupled ? plan->d_amr_oct : nullptr;
  A.w_in = w_in;
  A.w_out = w_out;
  A.form = form;
  A.vs = plan->var_stride;
  A.lvl = plan->d_lvl;
  A.err = reinterpret_cast<unsigned int*>(plan->d_red + 2);
  A.debug_no_issue = plan->debug_flags & 1;
  A.P = plan->params;
  switch (plan->pde) {
    case DH_PDE_ADV_FLUX: return fv_launch_adv_flux(plan, A, wmode, stream);
    case DH_PDE_ADV_NCP: return fv_launch_adv_ncp(plan, A, wmode, stream);
    case DH_PDE_EULER2D: return fv_launch_euler2(plan, A, wmode, stream);
    case DH_PDE_EULER3D: return fv_launch_euler3(plan, A, wmode, stream);
    case DH_PDE_SRHD3D: return fv_launch_srhd(plan, A, wmode, stream);
    default:
      set_error("patch_update_fv: PDE %d not supported by the FV stage", plan->pde);
      return DH_EUNSUPPORTED;
  }
}

}  // namespace dh
