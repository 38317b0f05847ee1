"""GPU parity of the first-order FV stage on coupled refinement levels (ratio 2:
prolongation into fine halos inside the stage kernel, reflux, restriction)
against the oracle.  Tolerance 1e-12 relative per voxel (max(|r|, s_v))."""
import numpy as np
import pytest

from gpu_util import assert_parity, dev, host, require_cuda
from paper_2608_19273_gb300 import dh, synth

pytestmark = pytest.mark.gpu
FV = 0


def _mesh(dim=3, nc=4, p=8, lo=1, m=2):
    return synth.coupled_mesh(nc, p, 1.0 / (nc * p), lo, m, dim=dim)


def _mask(mesh):
    m = np.zeros(mesh.var_stride, dtype=bool)
    for pt in mesh.patches:
        m[int(pt["offset"]):int(pt["offset"]) + int(pt["p"]) ** mesh.dim] = True
    return m


def _cons(orc, mesh, seed):
    rng = np.random.default_rng(seed)
    specs = [(1.0, 0.5)] + [(0.0, 0.5)] * mesh.dim + [(1.0, 0.5)]
    prim = synth.coupled_fields(mesh, rng, specs)
    pde = synth.PDE_EULER3D if mesh.dim == 3 else synth.PDE_EULER2D
    return pde, orc.prim2con(pde, prim, mesh.var_stride)


@pytest.mark.parametrize("dim", [3, 2])
@pytest.mark.parametrize("coef", [(0.0, 1.0, 1.0, 0.0), (0.75, 0.25, 0.25, 0.0), (1.0, 0.0, 0.5, 1 / 6)])
def test_coupled_stage(orc, dim, coef):
    torch = require_cuda()
    mesh = _mesh(dim)
    pde, qs = _cons(orc, mesh, 90 + dim)
    _, q0 = _cons(orc, mesh, 95 + dim)
    a, b, g, d = coef
    dt = 2e-3
    rng = np.random.default_rng(7)
    acc0 = rng.normal(size=qs.shape) if d else None
    ref = np.zeros_like(qs)
    ref_acc = acc0.copy() if d else None
    lam_ref = orc.stage(FV, pde, dim, mesh.patches, 1, mesh.var_stride, qs, q0=q0 if a else None, out=ref,
                        acc=ref_acc, dt=dt, a=a, b=b, g=g, d=d, want_lam=True)
    with dh.Plan(pde, dim, mesh.patches, 1, mesh.var_stride) as plan:
        out = torch.zeros(qs.shape, dtype=torch.float64, device="cuda")
        acc = dev(torch, acc0) if d else None
        d_dt = torch.tensor([dt], dtype=torch.float64, device="cuda")
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dh.patch_update_fv(plan, dev(torch, qs), dev(torch, q0) if a else None, out, acc, None, d_dt, a, b, g, d, lam)
        got = host(out)
        m = _mask(mesh)
        assert_parity(got, ref, m, what=f"coupled stage {dim}D {coef}")
        if d:
            assert_parity(host(acc), ref_acc, m, what="coupled stage acc")
        assert abs(float(host(lam)[0]) - lam_ref) <= 1e-14 * lam_ref


@pytest.mark.parametrize("dim", [3, 2])
def test_coupled_ssprk3_steps_and_graph(orc, dim):
    """Three SSP-RK3 steps with device dt through dh_rk_step, and the same steps replayed from a
    captured CUDA graph (bitwise equal to the eager steps)."""
    torch = require_cuda()
    mesh = _mesh(dim)
    pde, q = _cons(orc, mesh, 100 + dim)
    ref = q.copy()
    dts = orc.rk_steps(FV, pde, dim, mesh.patches, 1, mesh.var_stride, ref, rk=3, steps=3, cfl=0.4)
    outs = []
    for use_graph in (False, True):
        with dh.Plan(pde, dim, mesh.patches, 1, mesh.var_stride) as plan:
            Q = dev(torch, q)
            U1, U2 = torch.zeros_like(Q), torch.zeros_like(Q)
            lam = torch.zeros(1, dtype=torch.float64, device="cuda")
            dt = torch.zeros(1, dtype=torch.float64, device="cuda")
            dh.max_wave_speed(plan, Q, None, lam)
            if use_graph:
                torch.cuda.synchronize()
                s = torch.cuda.Stream()
                dh.dh_rk_step(plan, FV, 3, Q.clone(), U1, U2, None, None, dt.clone(), lam.clone(), 0.4, 0.0, s)
                s.synchronize()
                dh.dh_graph_capture(plan, FV, 3, 3, Q, U1, U2, None, None, dt, lam, 0.4, 0.0, 0, s)
                dh.dh_graph_launch(plan, s)
                s.synchronize()
            else:
                for _ in range(3):
                    dh.dh_rk_step(plan, FV, 3, Q, U1, U2, None, None, dt, lam, 0.4, 0.0)
            outs.append((host(Q), float(host(dt)[0])))
    m = _mask(mesh)
    assert_parity(outs[0][0], ref, m, what=f"coupled {dim}D SSP-RK3 steps")
    assert abs(outs[0][1] - dts[-1]) <= 1e-14 * dts[-1]
    assert np.array_equal(outs[0][0][:, m], outs[1][0][:, m])


def test_coupled_free_stream_bitwise():
    torch = require_cuda()
    mesh = _mesh(3)
    q = np.zeros((5, mesh.var_stride))
    for v, c in enumerate([1.3, 0.37, -0.21, 0.11, 2.9]):
        q[v, :] = c
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        Q = dev(torch, q)
        U1 = torch.zeros_like(Q)
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        dh.max_wave_speed(plan, Q, None, lam)
        for _ in range(2):
            dh.dh_rk_step(plan, FV, 1, Q, U1, None, None, None, dt, lam, 0.4, 0.0)
        got = host(Q)
    m = _mask(mesh)
    assert np.array_equal(got[:, m], q[:, m])


def test_coupled_linear_profile_exact_on_gpu(orc):
    """ADV_FLUX, a = (1, 0, 0), q = x / 2: the level-border values of the pinned oracle test
    (-1.5 alpha in the first fine layer, -0.75 alpha after the block) come out exactly."""
    torch = require_cuda()
    mesh = _mesh(3)
    X = synth.voxel_centres_any(mesh)
    alpha = 0.5
    q = (alpha * X[0])[None].copy()
    mat = np.zeros((3, mesh.var_stride))
    mat[0, :] = 1.0
    ref = np.zeros_like(q)
    orc.stage(FV, synth.PDE_ADV_FLUX, 3, mesh.patches, 1, mesh.var_stride, q, out=ref, mat=mat, dt=1.0, a=0, b=0,
              g=1)
    with dh.Plan(synth.PDE_ADV_FLUX, 3, mesh.patches, 1, mesh.var_stride) as plan:
        out = torch.zeros(q.shape, dtype=torch.float64, device="cuda")
        d_dt = torch.tensor([1.0], dtype=torch.float64, device="cuda")
        dh.patch_update_fv(plan, dev(torch, q), None, out, None, dev(torch, mat), d_dt, 0, 0, 1, 0)
        got = host(out)[0]
    m = _mask(mesh)
    fine = np.zeros(mesh.var_stride, dtype=bool)
    for pt in mesh.patches:
        if pt["level"] == 1:
            fine[int(pt["offset"]):int(pt["offset"]) + int(pt["p"]) ** 3] = True
    fine_first = fine & np.isclose(X[0], 0.25 + 1.0 / 128)
    assert fine_first.sum() == 32 * 32
    assert np.all(got[fine_first] == -1.5 * alpha)
    assert np.array_equal(got[m], ref[0][m])


def test_coupled_plan_rejections():
    torch = require_cuda()
    mesh = _mesh(3)
    q = torch.zeros((5, mesh.var_stride), dtype=torch.float64, device="cuda")
    d_dt = torch.tensor([1e-3], dtype=torch.float64, device="cuda")
    with dh.Plan(3, 3, mesh.patches, 2, mesh.var_stride) as plan:
        with pytest.raises(dh.DhError):   # second order on coupled levels is not provided
            dh.patch_update_fv_muscl(plan, q, None, torch.zeros_like(q), None, None, d_dt, 0, 1, 1, 0)
    with dh.Plan(synth.PDE_ADV_NCP, 3, mesh.patches, 1, mesh.var_stride) as plan:
        qq = torch.zeros((1, mesh.var_stride), dtype=torch.float64, device="cuda")
        mat = torch.zeros((3, mesh.var_stride), dtype=torch.float64, device="cuda")
        with pytest.raises(dh.DhError):   # non-conservative system
            dh.patch_update_fv(plan, qq, None, torch.zeros_like(qq), None, mat, d_dt, 0, 1, 1, 0)
    bad = mesh.patches.copy()
    first_fine = mesh.level_ranges[1][0]
    bad["dx"][first_fine] *= 2.0     # a fine patch whose coarse neighbour is not exactly twice as coarse
    with pytest.raises(dh.DhError):
        dh.Plan(3, 3, bad, 1, mesh.var_stride)


@pytest.mark.parametrize("dim", [3, 2])
def test_coupled_ssprk3_stage_sum_form(orc, dim):
    """SSP-RK3 steps in the stage-sum form (acc given: raw face-flux sums, reflux corrections added
    to them) on coupled levels against the oracle's Shu-Osher steps, eager and from a graph."""
    torch = require_cuda()
    mesh = _mesh(dim)
    pde, q = _cons(orc, mesh, 110 + dim)
    ref = q.copy()
    dts = orc.rk_steps(FV, pde, dim, mesh.patches, 1, mesh.var_stride, ref, rk=3, steps=3, cfl=0.4)
    outs = []
    for use_graph in (False, True):
        with dh.Plan(pde, dim, mesh.patches, 1, mesh.var_stride) as plan:
            Q = dev(torch, q)
            U1, U2, R = torch.zeros_like(Q), torch.zeros_like(Q), torch.zeros_like(Q)
            lam = torch.zeros(1, dtype=torch.float64, device="cuda")
            dt = torch.zeros(1, dtype=torch.float64, device="cuda")
            dh.max_wave_speed(plan, Q, None, lam)
            if use_graph:
                torch.cuda.synchronize()
                s = torch.cuda.Stream()
                dh.dh_rk_step(plan, FV, 3, Q.clone(), U1, U2, R, None, dt.clone(), lam.clone(), 0.4, 0.0, s)
                s.synchronize()
                dh.dh_graph_capture(plan, FV, 3, 3, Q, U1, U2, R, None, dt, lam, 0.4, 0.0, 0, s)
                dh.dh_graph_launch(plan, s)
                s.synchronize()
            else:
                for _ in range(3):
                    dh.dh_rk_step(plan, FV, 3, Q, U1, U2, R, None, dt, lam, 0.4, 0.0)
            outs.append((host(Q), float(host(dt)[0])))
    m = _mask(mesh)
    assert_parity(outs[0][0], ref, m, what=f"coupled {dim}D SSP-RK3 stage-sum form")
    assert abs(outs[0][1] - dts[-1]) <= 1e-14 * dts[-1]
    assert np.array_equal(outs[0][0][:, m], outs[1][0][:, m])


def test_coupled_ssprk3_stage_sum_form_free_stream_bitwise():
    """With the stage-sum form, SSP-RK3 steps keep a constant state bitwise constant on coupled
    levels (each stage adds multiples of exactly zero sums and corrections to q)."""
    torch = require_cuda()
    mesh = _mesh(3)
    q = np.zeros((5, mesh.var_stride))
    for v, c in enumerate([1.3, 0.37, -0.21, 0.11, 2.9]):
        q[v, :] = c
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        Q = dev(torch, q)
        U1, U2, R = torch.zeros_like(Q), torch.zeros_like(Q), torch.zeros_like(Q)
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        dh.max_wave_speed(plan, Q, None, lam)
        for _ in range(2):
            dh.dh_rk_step(plan, FV, 3, Q, U1, U2, R, None, dt, lam, 0.4, 0.0)
        got = host(Q)
    m = _mask(mesh)
    assert np.array_equal(got[:, m], q[:, m])


@pytest.mark.parametrize("coef", [(0.0, 1.0, 1.0), (0.75, 0.25, 0.25)])
def test_coupled_srhd_stage(orc, coef):
    """SRHD (primitives in the material slots) on coupled levels: the fine halos take the coarse
    voxel's conserved state and primitives, reflux uses both sides' primitives."""
    torch = require_cuda()
    mesh = _mesh(3)
    rng = np.random.default_rng(121)
    specs = [(1.0, 0.5), (0.0, 0.3), (0.0, 0.3), (0.0, 0.3), (1.0, 0.5)]
    prim = synth.coupled_fields(mesh, rng, specs)
    cons = orc.prim2con(synth.PDE_SRHD3D, prim, mesh.var_stride)
    q0 = orc.prim2con(synth.PDE_SRHD3D, synth.coupled_fields(mesh, rng, specs), mesh.var_stride)
    a, b, g = coef
    dt = 1e-3
    ref = np.zeros_like(cons)
    orc.stage(FV, synth.PDE_SRHD3D, 3, mesh.patches, 1, mesh.var_stride, cons, q0=q0 if a else None, out=ref,
              mat=prim, dt=dt, a=a, b=b, g=g)
    with dh.Plan(synth.PDE_SRHD3D, 3, mesh.patches, 1, mesh.var_stride) as plan:
        out = torch.zeros(cons.shape, dtype=torch.float64, device="cuda")
        d_dt = torch.tensor([dt], dtype=torch.float64, device="cuda")
        dh.patch_update_fv(plan, dev(torch, cons), dev(torch, q0) if a else None, out, None, dev(torch, prim), d_dt,
                           a, b, g, 0)
        got = host(out)
    assert_parity(got, ref, _mask(mesh), what=f"coupled SRHD stage {coef}")
