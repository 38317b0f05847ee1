/* dh.h -- C ABI of libdh: the batched explicit patch update on GB300 (sm_103a).
 *
 * The library advances K patches of p^d voxels (d = 2 or 3) of a hyperbolic
 * PDE system
 *
 *     dQ/dt + div F(Q) + B(Q) . grad Q = S(Q)                  (paper Eq. 1)
 *
 * by one explicit Runge-Kutta stage per call.  The problem statement follows
 * the paper's batched cell kernel K~_{dt,K} (Sec. II, Eq. 2): a list of K
 * patches, cells per patch p, halo width h, voxel spacing dx, time step dt and
 * the PDE id; N evolved quantities and M material parameters per voxel
 * (Sec. II: materials do not evolve).
 *
 * Conventions for every entry point
 *   - All device buffers are owned by the caller (typically torch tensors)
 *     and passed as raw device pointers.  The library never allocates memory
 *     per call.  A plan owns only its device patch/work tables and a few
 *     bytes of reduction scratch, all freed by dh_plan_destroy.
 *   - Compute calls are asynchronous on `stream` (a cudaStream_t; NULL means
 *     the legacy default stream).  Errors that can be detected on the host
 *     (bad sizes, NULL pointers, unsupported PDE) are returned synchronously
 *     and nothing is launched.  Launch failures return DH_ECUDA.
 *   - Data errors found on the device never trap: they are reported through
 *     status arrays and counters (con2prim).
 *   - dh_last_error() returns a thread-local message for the last failure.
 *   - One plan's calls must not overlap on the GPU: issue them on one stream,
 *     or order the streams with events.  A plan owns one pair of reduction
 *     slots that every call writing a wave speed (lam_out_dev, max_wave_speed,
 *     dh_rk_step with cfl > 0) accumulates into and resets, and one set of
 *     graph, derived-quantity and offload buffers; two calls of one plan that
 *     run at the same time race on them.  Different plans share nothing and
 *     may run concurrently on different streams.
 *
 * State layout ("SoA arena").  A state with V variables is one device array
 * of V * var_stride doubles.  Variable v of voxel (x, y, z) of patch k is at
 *     v * var_stride + patches[k].offset + (z * p + y) * p + x
 * (z = 0 in 2D).  Only interior voxels are stored; halos are gathered from
 * the face neighbours inside the kernels (the paper's gather prologue,
 * Sec. III-C Eq. 4, done on the fly).  Material parameters use a second
 * arena with the same offsets and var_stride.  offset must be a multiple of
 * 16 elements and var_stride a multiple of 32 (128-byte aligned blocks).
 */
#ifndef DH_H
#define DH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DH_OK = 0,
  DH_EINVAL = -1,        /* invalid argument (sizes, NULL pointers, aliasing, patch table) */
  DH_ECUDA = -2,         /* a CUDA call failed; see dh_last_error() */
  DH_EUNSUPPORTED = -3,  /* PDE, scheme or patch size not supported by this entry point */
  DH_ENOMEM = -4,        /* plan allocation failed */
  DH_ETIMEOUT = -5       /* a bounded device wait gave up (reserved) */
} dh_status;

/* PDE systems (Eq. 1 instances).  N evolved / M material quantities:
 *   ADV_FLUX  N=1 M=3  dq/dt + div(a q) = 0, a(x) = material velocity
 *   ADV_NCP   N=1 M=3  dq/dt + a . grad q = 0 (non-conservative form)
 *   EULER2D   N=4 M=0  (rho, rho u, rho v, E), ideal gas gamma
 *   EULER3D   N=5 M=0  (rho, rho u, rho v, rho w, E), ideal gas gamma
 *   WAVE3D    N=5 M=1  (phi, Pi, psi_x, psi_y, psi_z), material c(x)
 *   SRHD3D    N=5 M=5  (D, S_x, S_y, S_z, tau); the material arena carries
 *                      the primitives (rho, v_x, v_y, v_z, p) from con2prim
 *   GW59      N=59 M=0 59-unknown gravitational-wave stand-in: 11 coupled
 *                      scalar waves, lapse and shift, F = 0, B(Q).grad Q and a
 *                      nonlinear source (a defined substitute for CCZ4) */
typedef enum {
  DH_PDE_ADV_FLUX = 0,
  DH_PDE_ADV_NCP = 1,
  DH_PDE_EULER2D = 2,
  DH_PDE_EULER3D = 3,
  DH_PDE_WAVE3D = 4,
  DH_PDE_SRHD3D = 5,
  DH_PDE_GW59 = 6
} dh_pde;

/* One patch (the paper's cell with its embedded p^d mesh, Sec. II).
 * 72 bytes, natural alignment. */
typedef struct dh_patch {
  int32_t p;        /* voxels per patch per dimension */
  int32_t level;    /* refinement level (informational) */
  double dx;        /* VOXEL spacing (the paper's patch width is p * dx) */
  double x0[3];     /* lower corner of the patch */
  int64_t offset;   /* element offset of this patch's block in the arena */
  int32_t nbr[6];   /* face neighbours -x,+x,-y,+y,-z,+z; same p and dx;
                       periodic wrap is resolved by the caller; 2D: -1 in z */
} dh_patch;

typedef struct dh_plan dh_plan;

/* Create a plan for K patches (Sec. II Eq. 2: list of patches, p, h, PDE).
 *   pde, dim   : dh_pde and 2 or 3 (must match the PDE's dimension; the
 *                advection systems accept 3 only)
 *   patches    : host array of K patch records, copied by the plan
 *   halo       : halo width h: 1 for the FV stage, 3 for the FD4+KO stage
 *   var_stride : elements between two variables in every arena
 *   params     : PDE parameters (host, may be NULL for defaults):
 *                EULER*: [gamma=1.4]  SRHD3D: [Gamma=5/3]  WAVE3D: [damping=0.1]
 *                GW59: [kappa=0.1, C_ab (121 values, row-major)]
 * Patch sizes: 2 <= p <= 256.  Plans whose sizes are all multiples of 8 run
 * every stage kernel; other plans (the paper's typical 3^3 and 6^3 cells,
 * Sec. IV) run the first-order FV stage (patch_update_fv, dh_rk_step and the
 * graphs with scheme 0) through a generic kernel -- 2x2x2 blocks of
 * face-adjacent 3^3 patches as one 6^3 box, other small patches whole (up to
 * eight to a CTA), boxes of at most 256 voxels of larger ones (see
 * dh_generic_work_list) -- and refuse the FD4, MUSCL and coupled-level paths
 * (DH_EUNSUPPORTED, or DH_EINVAL at plan creation for coupled tables); the
 * autotuner has nothing to choose for them.  A face neighbour has the
 * same p, dx and level, or -- coupled refinement levels -- is one level
 * coarser with the same p and twice the dx; every patch above the coarsest
 * level present must then cover one octant of a patch one level coarser (its
 * parent, found from x0: lattice index round(x0 / (p dx)) halved), which stays
 * in the list.  On such a plan patch_update_fv (first-order FV, conservative
 * systems) adds, inside the same stage: piecewise-constant prolongation of the
 * fine halos (a halo voxel takes the value of the coarse voxel containing it),
 * reflux (a coarse voxel next to the finer level uses the mean of the fine
 * face fluxes on that face) and restriction (covered coarse voxels become the
 * mean of their 2^d fine voxels).  The paper's meshes are Peano spacetrees
 * (Sec. IV); it defines no coupling, these are the readings used.
 * Returns DH_EINVAL on a malformed table, DH_ENOMEM or DH_ECUDA if the device
 * tables cannot be created. */
dh_status dh_plan_create(dh_plan** plan, int32_t pde, int32_t dim, const dh_patch* patches, int32_t K,
                         int32_t halo, int64_t var_stride, const double* params, int32_t n_params);
dh_status dh_plan_destroy(dh_plan* plan);

/* One finite-volume Runge-Kutta stage over all K patches in one launch
 * (paper Sec. II-A Eq. 3: source per voxel, face fluxes from the two
 * neighbouring voxels, combination into the new state; Sec. II: RK stages
 * call the cell update with tableau-dependent dt):
 *     L(Q)_i = -(1/dx) sum_d [F^_{i+1/2} - F^_{i-1/2} + (D_{i+1/2} + D_{i-1/2})/2] + S(Q_i)
 *     F^     = (F_d(QL) + F_d(QR))/2 - s/2 (QR - QL),  s = max(lambda_d(QL), lambda_d(QR))
 *     D      = B_d((QL + QR)/2) (QR - QL)
 *     out    = a*q0 + b*qs + g*dt*L(qs)       (skipped if out == NULL)
 *     acc    = acc + d*dt*L(qs)               (skipped if acc == NULL)
 * qs  : stage input (N-variable arena); halos are read from neighbour patches.
 * q0  : N-variable arena or NULL (then a must be 0).  out may equal q0
 *       (element-wise read before write); out and acc must not alias qs.
 * mat : M-variable material arena (NULL if M = 0).
 * dt_dev : device pointer to one double (so CUDA graphs replay without the host).
 * lam_out_dev : NULL, or a device double that receives the maximum
 *       characteristic speed of the result (out, else acc) over all voxels and
 *       directions (not available for SRHD3D: use max_wave_speed on the
 *       primitives).  Requires plan halo >= 1. */
dh_status patch_update_fv(dh_plan* plan, const double* qs, const double* q0, double* out, double* acc,
                          const double* mat, const double* dt_dev, double a, double b, double g, double d,
                          double* lam_out_dev, void* stream);

/* One FD stage: 4th-order centred differences with 6th-difference
 * Kreiss-Oliger dissipation (paper Sec. I and Sec. IV: FD4 with KO):
 *     L(Q) = -sum_d dF_d/dx_d - sum_d B_d(Q) dQ/dx_d + S(Q) + sigma/(64 dx) sum_d delta6_d Q
 *     dQ/dx  = [(Q_-2 - Q_+2) + 8 (Q_+1 - Q_-1)] / (12 dx)
 *     delta6 = Q_-3 - 6 Q_-2 + 15 Q_-1 - 20 Q_0 + 15 Q_+1 - 6 Q_+2 + Q_+3
 * Same stage combination and arguments as patch_update_fv.  Requires halo 3. */
dh_status patch_update_fd_ko(dh_plan* plan, const double* qs, const double* q0, double* out, double* acc,
                             const double* mat, const double* dt_dev, double a, double b, double g,
                             double d, double sigma_ko, double* lam_out_dev, void* stream);

/* Second-order FV stage: the face states of patch_update_fv's Rusanov flux
 * come from MUSCL reconstruction with the minmod limiter (the face-state
 * stencil of the face-flux operator, Sec. II-A Eq. 3):
 *     sigma_i = minmod(Q_i - Q_{i-1}, Q_{i+1} - Q_i)   per component,
 *     minmod(a, b) = 0 if a, b differ in sign, else the one of smaller magnitude,
 *     QL = Q_{f-1} + sigma_{f-1}/2,  QR = Q_f - sigma_f/2  at face f,
 *     F^ = (F_d(QL) + F_d(QR))/2 - s/2 (QR - QL),  s = max(lambda_d(QL), lambda_d(QR)).
 * Conservative 3-D systems (ADV_FLUX, EULER3D; DH_EUNSUPPORTED otherwise);
 * needs a plan with halo >= 2.  Same arguments and stage combination as
 * patch_update_fv (lam_out_dev: speed of the cell-average result). */
dh_status patch_update_fv_muscl(dh_plan* plan, const double* qs, const double* q0, double* out, double* acc,
                                const double* mat, const double* dt_dev, double a, double b, double g, double d,
                                double* lam_out_dev, void* stream);

/* lam_out_dev <- max over voxels and directions of the characteristic speed of q
 * (the paper's scalar eigenvalue functions, Sec. II-B).  SRHD3D (mat = the
 * primitives): a voxel's speed grows with |v_d|, so only the direction of its
 * largest |v_d| is evaluated; the result is that direction's speed, within one
 * ulp of the maximum over three separately rounded speeds. */
dh_status max_wave_speed(dh_plan* plan, const double* q, const double* mat, double* lam_out_dev, void* stream);

/* Conservative -> primitive recovery for SRHD3D over the plan's voxels
 * (relativistic hydro is not in the paper; textbook definitions):
 * per voxel, FP64 Newton iteration on the pressure
 *   f(p) = ((G-1)/G) [(E+p) - S^2/(E+p) - D sqrt(1 - S^2/(E+p)^2)] - p,  E = tau + D,
 * within the bracket p > max(0, |S| - E) (a step leaving it is replaced by the
 * midpoint to the bound), stopping when |p_new - p| <= tol p_new, at most
 * max_iter steps; then v = S/(E+p), rho = D sqrt(1 - v^2).
 *   cons   : 5-variable arena (D, S_x, S_y, S_z, tau)
 *   prim   : 5-variable arena (rho, v_x, v_y, v_z, p), written
 *   p_prev : NULL or a pressure array (arena layout, one variable): the plain seed
 *   mlp_w  : NULL or 1224 floats (device): FP32 MLP seed p = E exp(mlp(x)),
 *            x = z-scored (|S|/E, D/E, ln(E/D)); then p_prev (or the cold seed
 *            max((1+1e-8) p_lo + 1e-300, (G-1) tau)) is the fallback
 *   seed_refine : 0..8 FP32 Newton steps applied to the first seed (the MLP's,
 *            else p_prev, else the cold seed) before the FP64 iteration.  The
 *            step uses A = E^2 - S^2 and B = tau (tau + 2 D) - S^2, formed once
 *            in FP64 with fused multiply-adds (S^2 = fma(S_x, S_x, fma(S_y, S_y,
 *            S_z S_z))); with y = E + p, t = p (E + y), q = sqrt(A + t) and
 *            q - D = (B + t)/(q + D) (no cancellation), p <- p - y (y f)/(y^2 f')
 *            with y f = gf q (q - D) - p y, y^2 f' = gf S^2 (q - D)/q + (gf - 1) y^2,
 *            gf = (G-1)/G; every FP32 operation rounded to float, no fused
 *            multiply-add; a step whose result is not finite or not above p_lo
 *            stops the refinement.  The refined seed lies within about 1e-6 of
 *            the root, so the FP64 iteration usually stops after two steps.
 *            With the MLP seed and seed_refine > 0 the seed E exp(y) is formed in
 *            FP32.  The fallback seed is never refined.  0: the plain recovery.
 *   status : NULL or one byte per voxel: 0 first seed converged, 1 fallback
 *            converged, 2 both failed (pressure = p_prev or the cold seed)
 *   iters  : NULL or Newton iterations per voxel (int32)
 *   fail_count_dev : NULL or a device int32 incremented by the number of status-2 voxels
 * Never traps on unphysical input. */
dh_status con2prim(dh_plan* plan, const double* cons, double* prim, const double* p_prev, const float* mlp_w,
                   double tol, int32_t max_iter, int32_t seed_refine, uint8_t* status, int32_t* iters,
                   int32_t* fail_count_dev, void* stream);
/* Same recovery on a flat array of n voxels (variable v of voxel i at v*stride + i). */
dh_status con2prim_flat(const double* cons, double* prim, int64_t n, int64_t stride, const double* p_prev,
                        const float* mlp_w, double Gamma, double tol, int32_t max_iter, int32_t seed_refine,
                        uint8_t* status, int32_t* iters, int32_t* fail_count_dev, void* stream);

/* MLP pressure seed (3 -> 32 tanh -> 32 tanh -> 1, FP32; not in the paper).
 * Weight vector: 1224 floats = W1[32][3], b1[32], W2[32][32], b2[32], W3[32],
 * b3, input mean[3], input std[3], pad.  Loss: mean of (y - ln(p/E))^2.
 * dh_mlp_features : raw inputs x (n x 3 floats) and, if p != NULL, targets
 *                   y = ln(p/E) (n floats) from a flat conserved array.
 * dh_mlp_standardize : writes the mean/std of x into w[1217..1222]
 *                   (scratch: >= 6 doubles; more allows more parallel partial sums).
 * dh_mlp_forward  : y = mlp(x) for raw inputs (z-scored inside).
 * dh_mlp_grad     : grad[0..1216] = d loss / d w over samples [offset, offset+B),
 *                   grad[1217] = loss; partials: ceil(B/64) * 1224 floats.
 *                   Deterministic (fixed-order sums, no atomics).
 * dh_mlp_adam     : one Adam step (Kingma & Ba) at step count t.
 * dh_mlp_train    : `steps` steps of grad + Adam (lr, beta 0.9/0.999, eps 1e-8)
 *                   over consecutive batches of the (pre-shuffled) data; step
 *                   counter starts at t0 + 1; loss_log (optional) gets one
 *                   float per step. */
dh_status dh_mlp_features(const double* cons, const double* p, int64_t n, int64_t stride, float* x, float* y,
                          void* stream);
dh_status dh_mlp_standardize(const float* x, int64_t n, float* w, double* scratch, int32_t scratch_len,
                             void* stream);
dh_status dh_mlp_forward(const float* w, const float* x, int64_t n, float* y, void* stream);
dh_status dh_mlp_grad(const float* w, const float* x, const float* t, int64_t offset, int32_t B, float* partials,
                      float* grad, void* stream);
dh_status dh_mlp_adam(float* w, float* m, float* v, const float* g, int32_t t, float lr, float b1, float b2,
                      float eps, void* stream);
dh_status dh_mlp_train(float* w, float* m, float* v, const float* x, const float* t, int64_t n, int32_t batch,
                       int32_t steps, int32_t t0, float lr, float* partials, float* grad, float* loss_log,
                       void* stream);

/* AoAoS <-> SoA arena: the gather prologue K~^(0) and scatter epilogue
 * K~^(S+1) around the batched kernel (paper Sec. III-C Eq. 4; AoAoS layout
 * Sec. II-B).  The caller's data are K separately allocated patch blocks,
 * each an array of structs over the patch AND its halo of width aos_halo
 * (p^ = p + 2 aos_halo voxels per dimension, Sec. II Eq. 2):
 *     block_k[((z * p^ + y) * p^ + x) * nq + v]      (halo-inclusive x, y, z; z = 0 in 2D)
 * aos_patches_dev : DEVICE array of K device pointers, block k for patch k of
 *                   the plan; blocks are 8-byte aligned and do not overlap
 *                   each other or the arena.  The caller owns all of them.
 * arena           : nq-variable arena (nq * var_stride doubles, plan offsets).
 * gather : arena[v*var_stride + off_k + (z*p + y)*p + x] = block_k[(((z+h)*p^ + y+h)*p^ + x+h)*nq + v]
 * scatter: the reverse assignment.
 * Only the p^d interior voxels are copied: halo entries of the blocks are
 * neither read nor written, and arena elements outside the patches keep
 * their values.  A combined state of N evolved and M material quantities per
 * voxel gathers into one (N+M)-variable arena whose first N variables serve
 * as qs and whose last M (at arena + N*var_stride) serve as mat.
 * nq in [1, 256], aos_halo in [0, 8]; DH_EINVAL otherwise.  Bit-exact copies.
 * The blocks may live in device memory or in page-locked host memory, which
 * the GPU reads and writes in place over NVLink-C2C (see dh_offload_bind). */
dh_status dh_gather_aoas(dh_plan* plan, const double* const* aos_patches_dev, int32_t nq, int32_t aos_halo,
                         double* arena, void* stream);
dh_status dh_scatter_aoas(dh_plan* plan, const double* arena, double* const* aos_patches_dev, int32_t nq,
                          int32_t aos_halo, void* stream);

/* Offload mode (paper Sec. III-C/D, Sec. IV): the caller's K patch blocks stay
 * in host memory in the AoAoS layout above; each call gathers them into the
 * device arena, advances n_steps time steps there and scatters the result
 * back.  Page-locked host memory is read and written in place by the gather
 * and scatter kernels (the host<->device transfer happens inside them).
 * dh_offload_bind: blocks is a HOST array of K pointers (block k for patch k);
 *   every block must be device memory, managed memory or page-locked host
 *   memory (cudaHostAlloc, cudaHostRegister, pinned torch tensors), 8-byte
 *   aligned, holding (p_k + 2 aos_halo)^d * nq doubles of one allocation;
 *   pageable memory is rejected with DH_EINVAL.  nq >= N + M: quantities
 *   0..N-1 are the evolved state, N..N+M-1 the material (SRHD: primitives).
 *   The plan keeps a device copy of the table (allocated once, replaced by a
 *   later bind).
 * dh_offload_run: gather all nq quantities into `arena` (an nq-variable device
 *   arena: qs = arena, mat = arena + N*var_stride); if cfl > 0 take the wave
 *   speed of the gathered state; n_steps x dh_rk_step (same scheme, rk, cfl,
 *   sigma and buffer rules; u1/u2/acc are N-variable device arenas), launched
 *   as a graph captured by dh_graph_capture would run them (for n_steps > 1
 *   SSP-RK3 FV steps of the Euler systems hand the derived quantities of each
 *   stage result to the next stage, in two arenas the plan allocates once);
 *   scatter
 *   quantities 0..nq_back-1 of every interior voxel back into the blocks
 *   (nq_back = N returns the evolved state; N + M also the material).
 *   Asynchronous on `stream`; the blocks hold the result once it completes. */
dh_status dh_offload_bind(dh_plan* plan, const double* const* blocks, int32_t nq, int32_t aos_halo);
/* dh_offload_bind_staged: as dh_offload_bind for page-locked HOST blocks, but each
 *   run moves them with the copy engine instead of SM loads over NVLink-C2C: the
 *   span from the lowest block to the end of the highest is copied into a device
 *   staging buffer with one cudaMemcpyAsync, gathered from there, and after the
 *   scatter the whole span is copied back with one cudaMemcpyAsync.  So the
 *   span should be one page-locked allocation, and nothing outside the blocks
 *   within it may change while a run is in flight (it is written back as it
 *   was read).  The copies use no SM time, so the kernels of a second problem
 *   on another stream run while they are in flight.  The plan allocates the
 *   staging buffer (span bytes) once, and again only for a larger span.
 *   DH_EINVAL if a block is not page-locked host memory or the span exceeds
 *   4x the blocks' bytes. */
dh_status dh_offload_bind_staged(dh_plan* plan, const double* const* blocks, int32_t nq, int32_t aos_halo);
dh_status dh_offload_run(dh_plan* plan, int32_t scheme, int32_t rk, int32_t n_steps, double* arena, double* u1,
                         double* u2, double* acc, double* dt_dev, double* lam_dev, double cfl, double sigma_ko,
                         int32_t nq_back, void* stream);

/* dt_dev <- cfl * dx_min / (dim * lam_dev[0]) on the device (the CFL rule). */
dh_status dh_cfl_dt(dh_plan* plan, const double* lam_dev, double cfl, double* dt_dev, void* stream);

/* Primitive -> conserved, element-wise over the plan's voxels (initial data).
 *   EULER*: (rho, u.., p) -> (rho, rho u.., p/(gamma-1) + rho |u|^2/2)
 *   SRHD3D: (rho, v, p)   -> (D, S, tau) */
dh_status dh_prim2con(dh_plan* plan, const double* prim, double* cons, void* stream);

/* One full time step of a Runge-Kutta scheme built from stage calls
 * (paper Sec. II: RK schemes call the cell update several times per step
 * with tableau-dependent dt and refresh halos between calls):
 *   rk = 1 forward Euler:  q <- q + dt L(q)              (u1 scratch)
 *   rk = 3 SSP-RK3 (Shu-Osher): u1 = q + dt L(q); u2 = 3/4 q + 1/4 u1 + 1/4 dt L(u1);
 *          q <- 1/3 q + 2/3 u2 + 2/3 dt L(u2)
 *   rk = 4 classical RK4 with acc = q + dt/6 (k1 + 2 k2 + 2 k3 + k4), q <- acc
 * scheme 0 = FV stage (patch_update_fv), 1 = FD4+KO stage (patch_update_fd_ko),
 * 2 = second-order FV stage (patch_update_fv_muscl).
 * If cfl > 0, dt_dev is first set on the device to cfl dx_min / (dim lam_dev[0])
 * and the last stage writes the new maximum wave speed into lam_dev, so
 * lam_dev must hold the speed of q on entry (max_wave_speed).  If cfl <= 0
 * the caller's dt_dev is used unchanged.  All buffers are N-variable arenas
 * owned by the caller; u2 is needed for rk >= 3 and acc for rk = 4.
 * rk = 3 with scheme 0 and acc != NULL: the same scheme
 * in its Butcher (stage-sum) form, u1 = q + dt L0, u2 = q + dt/4 (L0 + L1),
 * q <- q + dt/6 (L0 + L1) + 2 dt/3 L2, with acc (N variables, not aliasing the
 * other buffers) holding the raw face-flux sums of the earlier stages: fewer
 * FP64 operations per stage; results agree with the Shu-Osher form to
 * rounding, and a constant state stays bitwise constant.
 * SRHD3D: mat is the primitive arena (rho, v, p) and is updated in place:
 * before every stage con2prim recovers the primitives of the stage input,
 * seeded by the current primitives (settings from dh_plan_set_con2prim); with
 * cfl > 0 the step starts with con2prim(q) and max_wave_speed. */
dh_status dh_rk_step(dh_plan* plan, int32_t scheme, int32_t rk, double* q, double* u1, double* u2, double* acc,
                     const double* mat, double* dt_dev, double* lam_dev, double cfl, double sigma_ko,
                     void* stream);

/* con2prim settings used by dh_rk_step for SRHD3D: MLP seed weights (NULL:
 * plain Newton from the previous primitives), tolerance, iteration cap, FP32
 * refinement steps of the first seed (see con2prim) and an optional device
 * failure counter.  Defaults: NULL, 1e-12, 50, 0, NULL. */
dh_status dh_plan_set_con2prim(dh_plan* plan, const float* mlp_w, double tol, int32_t max_iter,
                               int32_t seed_refine, int32_t* fail_count_dev);

/* Capture n_steps consecutive dh_rk_step calls (same arguments) into one CUDA
 * graph owned by the plan (replacing any previous one); nothing runs during
 * capture.  stream must be a non-default stream.  If timing != 0, event
 * records are placed around every stage launch so that dh_graph_stage_times
 * can report per-stage device times of the most recent replay. */
dh_status dh_graph_capture(dh_plan* plan, int32_t scheme, int32_t rk, int32_t n_steps, double* q, double* u1,
                           double* u2, double* acc, const double* mat, double* dt_dev, double* lam_dev, double cfl,
                           double sigma_ko, int32_t timing, void* stream);
/* Replay the captured graph on stream. */
dh_status dh_graph_launch(dh_plan* plan, void* stream);
/* Number of kernel launches in the graph and of timed stages. */
dh_status dh_graph_info(dh_plan* plan, int32_t* n_kernels, int32_t* n_timed_stages);
/* Device time (ms) of the first n timed stages of the last completed replay
 * (the caller synchronises first). */
dh_status dh_graph_stage_times(dh_plan* plan, float* ms_out, int32_t n);

/* Autotuner.  Times every compiled variant of the plan's stage kernel on the
 * caller's buffers (one stage out = qs + dt L(qs), `reps` launches each after a
 * warm-up, CUDA events on `stream`) and keeps the fastest in the plan:
 *   FV (scheme 0): halo ring computed before or after the mid-plane barrier
 *                  x register cap (1 or 2 CTAs per SM) x grid (one CTA per
 *                  tile, or persistent: SMs x resident CTAs taking tiles from an
 *                  atomic queue) x tile shape (16x16 columns; 32x8 columns for
 *                  32^3 patches; 8x8 columns grouped four to a CTA -- shapes
 *                  that change nothing for the plan's patch sizes are skipped;
 *                  one 8x8 column per 64-thread CTA) x TMA staging of the column
 *                  planes (3D Euler)
 *                  x z-march in whole patches or in chunks of <= 16 planes;
 *                  the persistent grid and the 32x8 columns with the register
 *                  cap only (20 to 48 candidates);
 *   FV2 (scheme 2): the three variants of dh_plan_set_variant_muscl;
 *   FD (scheme 1): register cap x shared-memory staging by plain loads or by
 *                  TMA tensor copies (2 candidates, or 6 with TMA -- 4 for
 *                  GW59; TMA only when every level is a run of back-to-back
 *                  patches, see dh_plan_set_variant).
 * `out` is overwritten.  If cache_path is NULL the environment variable
 * DH_TUNE_CACHE names the cache file (no cache when it is unset).  With a cache
 * file the choice is first looked up
 * there (one JSON object per line, keyed by GPU name, PDE, scheme and patch-size
 * histogram) and, when timed, appended to it.  choice_out (optional, 4 ints):
 * fv_var, fv_zs, fd_var, 1 if taken from the cache.  times_out (optional,
 * DH_TUNE_MAX_CANDIDATES floats): ms per launch of each candidate, in the order
 * tile shape, grid, z-march, then fv_var bits 0-1 (unused entries untouched). */
#define DH_TUNE_MAX_CANDIDATES 64
dh_status dh_autotune(dh_plan* plan, int32_t scheme, const double* qs, double* out, const double* mat,
                      const double* dt_dev, int32_t reps, const char* cache_path, int32_t* choice_out,
                      float* times_out, void* stream);
/* Autotuner over whole time steps: as dh_autotune (same candidates, cache and
 * outputs; cache key marked with the step kind), but every timed call runs
 * n_steps time steps exactly as dh_rk_step, dh_offload_run and a captured
 * graph run them -- for SSP-RK3 FV steps of the Euler systems with acc and
 * cfl > 0 the stage-sum form with the derived quantities handed from stage to
 * stage -- so that the choice fits the kernels a graph replays.  Same buffer
 * rules as dh_rk_step.  q (and for SRHD3D the primitive arena mat) is advanced
 * by (1 + reps) x n_steps steps per candidate: pass scratch copies.  lam_dev
 * must hold the wave speed of q on entry when cfl > 0. */
dh_status dh_autotune_steps(dh_plan* plan, int32_t scheme, int32_t rk, int32_t n_steps, double* q, double* u1,
                            double* u2, double* acc, const double* mat, double* dt_dev, double* lam_dev, double cfl,
                            double sigma_ko, int32_t reps, const char* cache_path, int32_t* choice_out,
                            float* times_out, void* stream);
/* Select a variant directly: fv_var 0..23 (bit 0: ring before the barrier,
 * bit 1: two CTAs per SM, bit 2: persistent grid with a tile queue, bits 3-4:
 * tile shape 0 = 16x16 columns for p % 16 == 0 and 8x8 columns grouped four to a
 * CTA otherwise, 1 = as 0 but 32x8 columns for p % 32 == 0, 2 = 8x8 columns
 * grouped four to a CTA for every patch, 3 = one 8x8 column per 64-thread CTA
 * (small problems); bit 5: TMA-staged column planes (3D Euler); bit 2, tile
 * shape 1 and bit 5 need bit 1, bit 5 excludes bit 2 and tile shapes 2 and 3,
 * tile shape 3 excludes bit 2; DH_EINVAL otherwise), fv_zs 0..1 (z-chunks of <= 16 planes,
 * and a thin last wave filled with half-height chunks of the cheapest columns), fd_var
 * 0, 2, 4 or 6 (bit 1: two CTAs per SM; bit 2: TMA staging, which needs every
 * run of equal-size patches to be stored back to back with its face
 * neighbours inside the run; DH_EUNSUPPORTED otherwise), or, for systems of
 * at most five variables (not GW59), 12 / 20: TMA staging with register caps
 * for three / four CTAs per SM. */
dh_status dh_plan_set_variant(dh_plan* plan, int32_t fv_var, int32_t fv_zs, int32_t fd_var);

/* Variant of the second-order FV stage (patch_update_fv_muscl), also chosen by
 * dh_autotune / dh_autotune_steps with scheme 2 (choice_out[0] is then fv2_var):
 *   0 z-march: a CTA marches a 16x16 column (four 8x8 columns of 8^3
 *     patches) through the patch, keeping the z states of its voxels in
 *     registers and exchanging x/y states through shared memory;
 *   1 the same in chunks of at most 16 planes;
 *   2 (default) 8x8x4 tiles staged with their two-voxel face halos.
 * Every variant gives the same results (the same operations in the same order). */
dh_status dh_plan_set_variant_muscl(dh_plan* plan, int32_t fv2_var);

/* Error flags raised on the device by the plan's kernels (bit 0: a bounded
 * wait for a TMA copy gave up: the FD stage skipped the tile, the FV stage
 * finished the tile on stale data -- either way the launch's results are
 * invalid).  Synchronous; clear != 0 resets them. */
dh_status dh_plan_errors(dh_plan* plan, uint32_t* flags, int32_t clear);

/* Test hooks (0 in normal use).  Bit 0: the TMA-staged FD and FV stages arm
 * their barriers but issue no copy, so that their bounded waits run out and the
 * error flag path can be exercised without any fault. */
dh_status dh_plan_set_debug(dh_plan* plan, int32_t flags);

/* Diagnostic: for n doubles x, y_nr[i] = the kernels' Newton-Raphson
 * reciprocal of x[i] and y_div[i] = 1.0 / x[i] (IEEE division), so that a test
 * can bound the reciprocal's error.  All three arrays are device arrays of n. */
dh_status dh_check_recip(const double* x, double* y_nr, double* y_div, int64_t n, void* stream);

/* Diagnostic: for n doubles x, y_sqrt[i] and y_rsqrt[i] = the kernels' square
 * root and reciprocal square root of x[i] (the hardware estimate refined by one
 * third-order step for normal, finite x > 0; sqrt and rsqrt themselves for other
 * arguments), so that a test can bound their error against correctly rounded
 * values.  All three arrays are device arrays of n. */
dh_status dh_check_sqrt(const double* x, double* y_sqrt, double* y_rsqrt, int64_t n, void* stream);

/* Diagnostic (host only, no CUDA call): the work list that dh_plan_create builds
 * for the generic FV stage of a table whose patch sizes are not all multiples of
 * 8 (one CTA per item).  *n_items receives the number of items; with items !=
 * NULL, 16 int32 per item are written to the host array items (capacity
 * max_items items): the patch ids patch[0..7] (-1 where unused), the box origin
 * x0, y0, z0 inside the patch, the box extents bx, by, bz, the group count ng
 * (whole patches of equal size packed into one item) and mp (3 for a 2x2x2 block
 * of face-adjacent 3^3 patches run as one 6^3 box: member (mx, my, mz) is
 * patch[mx + 2 my + 4 mz]; 0 otherwise).  The table is checked only for patch
 * sizes in [2, 256] and neighbour ids in [0, K) (DH_EINVAL otherwise). */
dh_status dh_generic_work_list(int32_t dim, const dh_patch* patches, int32_t K, int32_t* items, int32_t max_items,
                               int32_t* n_items);

/* Diagnostic: the integer-pipe conversions of the recovery's FP32 seed paths
 * against the hardware conversions.  For n doubles x and n floats g (device
 * arrays): f_int[i] / f_hw[i] = x[i] rounded to float by bit operations / by
 * the hardware; d_int[i] / d_hw[i] = g[i] widened to double likewise.  The
 * pairs are bitwise equal (NaNs aside) by construction. */
dh_status dh_check_convert(const double* x, float* f_int, float* f_hw, const float* g, double* d_int, double* d_hw,
                           int64_t n, void* stream);

/* Diagnostic: FP64 FMA throughput probe used to measure the FP64 roofline
 * peak on the running GPU.  Launches n_threads (a multiple of 256) threads;
 * each runs 8 independent chains of `iters` fused multiply-adds
 * (8 * iters * n_threads FMAs = 16 * iters * n_threads FLOP) and writes one
 * double to out_dev[thread].  out_dev must hold n_threads doubles. */
dh_status dh_probe_dfma(double* out_dev, int64_t n_threads, int32_t iters, void* stream);

/* The FV stage for callers that cannot allocate device memory (a host
 * framework whose pool owns the device, a plugin host that forbids
 * allocations after start-up, a real-time loop that must not block in the
 * allocator).  The paper has no counterpart: it is a deployment variant of
 * patch_update_fv.  It takes the plan-creation arguments (host patch table,
 * K, var_stride, params) together with the stage arguments of
 * patch_update_fv, and keeps the patch table, the work list and the
 * reduction slots in one file-scope device array of 1,310,976 bytes that
 * every GPU loading the library holds until exit.  Limits: K <= 8192 patches
 * and at most 16384 tile work items (a 16x16 column of a patch, or four 8x8
 * columns); larger inputs return DH_EINVAL.  PDEs: ADV_FLUX, ADV_NCP,
 * EULER2D, EULER3D; halo 1; patch sizes multiples of 8 in [8, 256] (other
 * sizes, which dh_plan_create accepts, return DH_EINVAL here); every face
 * neighbour on the same level (coupled refinement levels, which
 * dh_plan_create accepts, return DH_EINVAL here).
 * Each call copies the patch table and the work list it builds into static
 * host buffers of the library and uploads them from there with
 * cudaMemcpyAsync (staged before the call returns, so `patches` may be freed
 * or reused as soon as the call returns, page-locked or not), clears the
 * reduction slots, then launches the stage on `stream`; it calls no
 * cudaMalloc, cudaFree or other allocating routine.  All calls share the one
 * array and overwrite the previous call's contents, so calls that overlap on
 * the GPU race.  The first call on a device looks up the array's address
 * (cudaGetSymbolAddress) with that device current: make it before any stream
 * capture. */
dh_status patch_update_fv_noalloc(int32_t pde, int32_t dim, const dh_patch* patches, int32_t K,
                                  int64_t var_stride, const double* params, int32_t n_params,
                                  const double* qs, const double* q0, double* out, double* acc,
                                  const double* mat, const double* dt_dev, double a, double b, double g,
                                  double d, double* lam_out_dev, void* stream);

const char* dh_last_error(void);

/* Library version string. */
const char* dh_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DH_H */
