"""GPU parity of the FV stage (patch_update_fv) against the FP64 oracle.

Tolerance: 1e-12 relative per voxel, relative to max(|r|, s_v) with s_v the
largest magnitude of variable v over the workload (values that cross zero)."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_parity, dev, host, require_cuda
from helpers import arena, from_grid, single_level, to_grid, voxel_mask
from paper_2608_19273_gb300 import dh, synth

pytestmark = pytest.mark.gpu
FV = 0


def _euler_cons(orc, mesh, seed, pde=synth.PDE_EULER3D):
    return orc.prim2con(pde, synth.euler_prims(mesh, seed), mesh.var_stride)


@pytest.mark.parametrize("scale", [8, 4])
@pytest.mark.parametrize("coef", [(0.0, 1.0, 1.0), (0.75, 0.25, 0.25), (1 / 3, 2 / 3, 2 / 3)])
def test_euler3d_single_stage(orc, scale, coef):
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=scale)
    q0 = _euler_cons(orc, mesh, 21)
    qs = _euler_cons(orc, mesh, 22)
    a, b, g = coef
    dt = 1.7e-3
    ref = np.zeros_like(qs)
    lam_ref = orc.stage(FV, 3, 3, mesh.patches, 1, mesh.var_stride, qs, q0=q0 if a else None, out=ref, dt=dt,
                        a=a, b=b, g=g, want_lam=True)
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        d_qs, d_q0 = dev(torch, qs), dev(torch, q0)
        d_out = torch.zeros_like(d_qs)
        d_dt = torch.tensor([dt], dtype=torch.float64, device="cuda")
        d_lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dh.patch_update_fv(plan, d_qs, d_q0 if a else None, d_out, None, None, d_dt, a, b, g, 0.0, d_lam)
        torch.cuda.synchronize()
        out = host(d_out)
        lam = float(host(d_lam)[0])
    m = voxel_mask(mesh)
    assert_parity(out, ref, m, what="euler3d stage")
    assert abs(lam - lam_ref) <= 1e-14 * lam_ref


@pytest.mark.parametrize("pde", [synth.PDE_ADV_FLUX, synth.PDE_ADV_NCP])
@pytest.mark.parametrize("axis,sign", [(0, 1), (1, -1), (2, 1)])
@pytest.mark.parametrize("p", [8, 16])
def test_advection_exact_shift(orc, pde, axis, sign, p):
    """|a| dt/dx = 1: the GPU stage moves dyadic data by exactly one voxel (bitwise)."""
    torch = require_cuda()
    mesh = single_level((2, 2, 2), p, 1.0 / 128)
    rng = np.random.default_rng(5)
    G = synth.dyadic_field(rng, (2 * p,) * 3)
    q = from_grid(mesh, G, arena(mesh, 1)[0])[None].copy()
    mat = arena(mesh, 3)
    mat[axis] = sign * 1.0
    with dh.Plan(pde, 3, mesh.patches, 1, mesh.var_stride) as plan:
        d_out = torch.zeros(q.shape, dtype=torch.float64, device="cuda")
        d_dt = torch.tensor([1.0 / 128], dtype=torch.float64, device="cuda")
        dh.patch_update_fv(plan, dev(torch, q), None, d_out, None, dev(torch, mat), d_dt, 0, 1, 1, 0)
        out = host(d_out)
    assert np.array_equal(to_grid(mesh, out[0]), np.roll(G, sign, axis=2 - axis))


def test_free_stream_bitwise_gpu(orc):
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=4)
    q = arena(mesh, 5)
    for v, c in enumerate([1.3, 0.37, -0.21, 0.11, 2.9]):
        q[v] = c
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        d_out = torch.zeros(q.shape, dtype=torch.float64, device="cuda")
        d_dt = torch.tensor([0.37], dtype=torch.float64, device="cuda")
        dh.patch_update_fv(plan, dev(torch, q), None, d_out, None, None, d_dt, 0, 1, 1, 0)
        out = host(d_out)
    m = voxel_mask(mesh)
    assert np.array_equal(out[:, m], q[:, m])


def test_euler2d_workload_10_steps(orc):
    """The full 2D workload: 64 patches of 16^2, 10 forward-Euler steps with device-side CFL dt."""
    torch = require_cuda()
    w = synth.workload("euler2d")
    mesh = w.mesh
    q = _euler_cons(orc, mesh, w.seed, synth.PDE_EULER2D)
    ref = q.copy()
    dts = orc.rk_steps(FV, 2, 2, mesh.patches, 1, mesh.var_stride, ref, rk=1, steps=10, cfl=0.4)
    with dh.Plan(2, 2, mesh.patches, 1, mesh.var_stride) as plan:
        a = dev(torch, q)
        b = torch.zeros_like(a)
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        dh.max_wave_speed(plan, a, None, lam)
        got_dt = []
        for s in range(10):
            dh.dh_cfl_dt(plan, lam, 0.4, dt)
            got_dt.append(float(host(dt)[0]))
            dh.patch_update_fv(plan, a, None, b, None, None, dt, 0, 1, 1, 0, lam)
            a, b = b, a
        out = host(a)
    m = voxel_mask(mesh)
    assert_parity(out, ref, m, what="euler2d 10 steps")
    assert np.max(np.abs(np.array(got_dt) - dts) / dts) < 1e-14


def test_euler3d_ssprk3_steps(orc):
    """Three SSP-RK3 steps (9 stages) on the AMR-like mix at reduced patch counts."""
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=4)
    q = _euler_cons(orc, mesh, 31)
    ref = q.copy()
    dts = orc.rk_steps(FV, 3, 3, mesh.patches, 1, mesh.var_stride, ref, rk=3, steps=3, cfl=0.4)
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        Q = dev(torch, q)
        U1, U2 = torch.zeros_like(Q), torch.zeros_like(Q)
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        dh.max_wave_speed(plan, Q, None, lam)
        for s in range(3):
            dh.dh_cfl_dt(plan, lam, 0.4, dt)
            dh.patch_update_fv(plan, Q, None, U1, None, None, dt, 0, 1, 1, 0)
            dh.patch_update_fv(plan, U1, Q, U2, None, None, dt, 0.75, 0.25, 0.25, 0)
            dh.patch_update_fv(plan, U2, Q, Q, None, None, dt, 1 / 3, 2 / 3, 2 / 3, 0, lam)
        out = host(Q)
        dt_last = float(host(dt)[0])
    m = voxel_mask(mesh)
    assert_parity(out, ref, m, what="euler3d 3 SSP-RK3 steps")
    assert abs(dt_last - dts[-1]) <= 1e-14 * dts[-1]


@pytest.mark.parametrize("p", [8, 16, 32])
def test_single_self_periodic_patch(orc, p):
    """K = 1: a patch that is its own neighbour in every direction."""
    torch = require_cuda()
    mesh = single_level((1, 1, 1), p, 1.0 / 64)
    q = _euler_cons(orc, mesh, 40 + p)
    ref = np.zeros_like(q)
    orc.stage(FV, 3, 3, mesh.patches, 1, mesh.var_stride, q, out=ref, dt=1e-3)
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        d_out = torch.zeros(q.shape, dtype=torch.float64, device="cuda")
        d_dt = torch.tensor([1e-3], dtype=torch.float64, device="cuda")
        dh.patch_update_fv(plan, dev(torch, q), None, d_out, None, None, d_dt, 0, 1, 1, 0)
        out = host(d_out)
    assert_parity(out, ref, voxel_mask(mesh), what=f"self-periodic p={p}")


def test_newton_reciprocal_within_one_ulp():
    """The kernels' reciprocal (hardware estimate + one third-order refinement step) against IEEE 1.0/x."""
    torch = require_cuda()
    rng = np.random.default_rng(17)
    x = np.concatenate([np.exp(rng.uniform(-30, 30, 400000)), -np.exp(rng.uniform(-30, 30, 100000)),
                        np.array([1.0, 2.0, 0.5, 3.0, 1e-300, 1e300, 0.1, 7.0])])
    d_x = dev(torch, x)
    y_nr, y_div = torch.zeros_like(d_x), torch.zeros_like(d_x)
    dh.dh_check_recip(d_x, y_nr, y_div)
    a, b = host(y_nr), host(y_div)
    ulp = np.abs(a.view(np.int64) - b.view(np.int64))
    assert ulp.max() <= 1, ulp.max()
    assert np.array_equal(b, 1.0 / x)


def test_refined_square_root_and_reciprocal_square_root_within_two_ulps():
    """The kernels' sqrt and 1/sqrt (hardware estimate + one third-order step of the binomial series)
    against correctly rounded values, over the whole normal range; zero, subnormal, infinite,
    negative and NaN arguments take sqrt and rsqrt themselves."""
    torch = require_cuda()
    rng = np.random.default_rng(19)
    x = np.concatenate([np.exp(rng.uniform(-700, 700, 400000)), rng.uniform(1.0, 4.0, 100000),
                        np.array([1.0, 2.0, 4.0, 0.25, 3.0, 2.2250738585072014e-308, 1.7976931348623157e308])])
    d_x = dev(torch, x)
    y_s, y_r = torch.zeros_like(d_x), torch.zeros_like(d_x)
    dh.dh_check_sqrt(d_x, y_s, y_r)
    s, r = host(y_s), host(y_r)
    ulp_s = np.abs(s.view(np.int64) - np.sqrt(x).view(np.int64))
    r_ref = (np.longdouble(1) / np.sqrt(x.astype(np.longdouble))).astype(np.float64)
    ulp_r = np.abs(r.view(np.int64) - r_ref.view(np.int64))
    print(f"sqrt: max {ulp_s.max()} ulp, {np.mean(ulp_s == 0):.3f} exact; 1/sqrt: max {ulp_r.max()} ulp")
    assert ulp_s.max() <= 2 and ulp_r.max() <= 2
    special = np.array([0.0, 5e-324, 1e-310, np.inf, -1.0, np.nan])
    d_x = dev(torch, special)
    y_s, y_r = torch.zeros_like(d_x), torch.zeros_like(d_x)
    dh.dh_check_sqrt(d_x, y_s, y_r)
    s, r = host(y_s), host(y_r)
    with np.errstate(divide="ignore", invalid="ignore"):
        assert np.array_equal(s, np.sqrt(special), equal_nan=True)
        r_ref = (np.longdouble(1) / np.sqrt(special.astype(np.longdouble))).astype(np.float64)
    assert r[0] == np.inf and r[3] == 0.0 and np.isnan(r[4]) and np.isnan(r[5])
    assert np.all(np.abs(r[1:3].view(np.int64) - r_ref[1:3].view(np.int64)) <= 2)


def test_graph_hands_derived_quantities_to_the_next_step(orc):
    """Inside a multi-step SSP-RK3 graph the last stage of a step stores the derived quantities of
    its result and the next step's first stage reads them: bitwise the same state and dt as eager
    dh_rk_step calls (which recompute them)."""
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=4)
    q = _euler_cons(orc, mesh, 37)
    res = []
    for graph in (False, True):
        with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
            Q = dev(torch, q)
            U1, U2 = torch.zeros_like(Q), torch.zeros_like(Q)
            lam = torch.zeros(1, dtype=torch.float64, device="cuda")
            dt = torch.zeros(1, dtype=torch.float64, device="cuda")
            dh.max_wave_speed(plan, Q, None, lam)
            torch.cuda.synchronize()
            if graph:
                s = torch.cuda.Stream()
                dh.dh_rk_step(plan, FV, 3, Q.clone(), U1, U2, None, None, dt.clone(), lam.clone(), 0.4, 0.0, s)
                s.synchronize()
                dh.dh_graph_capture(plan, FV, 3, 4, Q, U1, U2, None, None, dt, lam, 0.4, 0.0, 0, s)
                dh.dh_graph_launch(plan, s)
                s.synchronize()
            else:
                for _ in range(4):
                    dh.dh_rk_step(plan, FV, 3, Q, U1, U2, None, None, dt, lam, 0.4, 0.0)
            res.append((host(Q), host(dt), host(lam)))
    m = voxel_mask(mesh)
    assert np.array_equal(res[0][0][:, m], res[1][0][:, m])
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][2], res[1][2])


@pytest.mark.parametrize("dim", [3, 2])
def test_ssprk3_stage_sum_form(orc, dim):
    """SSP-RK3 steps through dh_rk_step with acc (the stage-sum form u2 = q + dt/4 (L0 + L1),
    q <- q + dt/6 (L0 + L1) + 2 dt/3 L2) against the oracle's Shu-Osher steps, and the same steps
    replayed from a captured graph (derived-quantity hand-over on): bitwise equal to the eager steps."""
    torch = require_cuda()
    if dim == 3:
        mesh, pde = synth.euler3d_amr_mesh(scale=4), synth.PDE_EULER3D
    else:
        mesh, pde = synth.workload("euler2d").mesh, synth.PDE_EULER2D
    q = _euler_cons(orc, mesh, 41, pde)
    ref = q.copy()
    dts = orc.rk_steps(FV, pde, dim, mesh.patches, 1, mesh.var_stride, ref, rk=3, steps=3, cfl=0.4)
    res = []
    for graph in (False, True):
        with dh.Plan(pde, dim, mesh.patches, 1, mesh.var_stride) as plan:
            Q = dev(torch, q)
            U1, U2, R = torch.zeros_like(Q), torch.zeros_like(Q), torch.zeros_like(Q)
            lam = torch.zeros(1, dtype=torch.float64, device="cuda")
            dt = torch.zeros(1, dtype=torch.float64, device="cuda")
            dh.max_wave_speed(plan, Q, None, lam)
            torch.cuda.synchronize()
            if graph:
                s = torch.cuda.Stream()
                dh.dh_rk_step(plan, FV, 3, Q.clone(), U1, U2, R, None, dt.clone(), lam.clone(), 0.4, 0.0, s)
                s.synchronize()
                dh.dh_graph_capture(plan, FV, 3, 3, Q, U1, U2, R, None, dt, lam, 0.4, 0.0, 0, s)
                dh.dh_graph_launch(plan, s)
                s.synchronize()
            else:
                for _ in range(3):
                    dh.dh_rk_step(plan, FV, 3, Q, U1, U2, R, None, dt, lam, 0.4, 0.0)
            res.append((host(Q), float(host(dt)[0])))
    m = voxel_mask(mesh)
    assert_parity(res[0][0], ref, m, what=f"euler{dim}d SSP-RK3 stage-sum form")
    assert abs(res[0][1] - dts[-1]) <= 1e-14 * dts[-1]
    assert np.array_equal(res[0][0][:, m], res[1][0][:, m]) and res[0][1] == res[1][1]


def test_ssprk3_stage_sum_form_free_stream_bitwise():
    """A constant state stays bitwise constant through SSP-RK3 steps in the stage-sum form (every
    stage adds a multiple of an exactly zero face-flux sum to q)."""
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=4)
    q = arena(mesh, 5)
    for v, c in enumerate([1.3, 0.37, -0.21, 0.11, 2.9]):
        q[v] = c
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        Q = dev(torch, q)
        U1, U2, R = torch.zeros_like(Q), torch.zeros_like(Q), torch.zeros_like(Q)
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        dh.max_wave_speed(plan, Q, None, lam)
        for _ in range(2):
            dh.dh_rk_step(plan, FV, 3, Q, U1, U2, R, None, dt, lam, 0.4, 0.0)
        got = host(Q)
    m = voxel_mask(mesh)
    assert np.array_equal(got[:, m], q[:, m])


def test_stage_sum_form_rejects_aliased_acc():
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=8)
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        Q = torch.ones((5, mesh.var_stride), dtype=torch.float64, device="cuda")
        U1, U2 = torch.zeros_like(Q), torch.zeros_like(Q)
        dt = torch.tensor([1e-3], dtype=torch.float64, device="cuda")
        with pytest.raises(dh.DhError):
            dh.dh_rk_step(plan, FV, 3, Q, U1, U2, U1, None, dt, None, 0.0, 0.0)


@pytest.mark.parametrize("fv_var", [0, 3, 24, 27])
@pytest.mark.parametrize("n_steps", [10, 9])
def test_euler2d_graph_steps_fold_dt_and_alternate_buffers(orc, fv_var, n_steps):
    """The 2D workload as a captured graph of forward-Euler steps: the steps alternate between the
    state and the stage buffer (one copy at the end when their number is odd), and from the second
    step on each step's dt is written by the previous step's stage in its lambda epilogue (one CFL
    launch per graph).  Result and every step's dt against the oracle, with 16x16 columns and with
    one 8x8 column per 64-thread CTA; the graph holds n_steps + 1 kernel launches."""
    torch = require_cuda()
    w = synth.workload("euler2d")
    mesh = w.mesh
    q = _euler_cons(orc, mesh, w.seed, synth.PDE_EULER2D)
    ref = q.copy()
    dts = orc.rk_steps(FV, 2, 2, mesh.patches, 1, mesh.var_stride, ref, rk=1, steps=2 * n_steps, cfl=0.4)
    with dh.Plan(2, 2, mesh.patches, 1, mesh.var_stride) as plan:
        dh.dh_plan_set_variant(plan, fv_var, 0, 0)
        Q = dev(torch, q)
        U1 = torch.empty_like(Q)
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        dh.max_wave_speed(plan, Q, None, lam)
        s = torch.cuda.Stream()
        torch.cuda.synchronize()
        dh.dh_graph_capture(plan, FV, 1, n_steps, Q, U1, None, None, None, dt, lam, 0.4, 0.0, 0, s)
        n_kernels, _ = dh.dh_graph_info(plan)
        assert n_kernels == n_steps + 1
        dh.dh_graph_launch(plan, s)
        s.synchronize()
        dt_mid = float(host(dt)[0])
        dh.dh_graph_launch(plan, s)
        s.synchronize()
        got, dt_last = host(Q), float(host(dt)[0])
    # dt_dev holds the dt of the last step taken (the graph's last step does not fold)
    assert abs(dt_mid - dts[n_steps - 1]) <= 1e-15 * dts[n_steps - 1]
    assert abs(dt_last - dts[-1]) <= 1e-15 * dts[-1]
    assert_parity(got, ref, voxel_mask(mesh), what=f"euler2d graph, {2 * n_steps} steps, variant {fv_var}")
