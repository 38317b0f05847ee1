"""GPU parity of the first-order FV stage on plans whose patch sizes are not multiples of 8 (the
generic kernel: 2x2x2 blocks of 3^3 patches as 6^3 boxes, other small patches whole, boxes of
larger ones with ragged ends) against the FP64 oracle: the paper's typical 3^3 and 6^3 cells,
sizes that leave partial boxes (7, 12, 20), 2D, the advection forms with a material field, SRHD, mixed sizes, whole SSP-RK3
steps with the derived-quantity hand-over and the device-side CFL step, and the refusal of the
paths that need multiples of 8.

Tolerance: 1e-12 relative per voxel, relative to max(|r|, s_v) (values that cross zero)."""
import numpy as np
import pytest

from gpu_util import assert_parity, dev, host, require_cuda
from helpers import arena, single_level, voxel_mask
from paper_2608_19273_gb300 import dh, synth

pytestmark = pytest.mark.gpu
FV = 0

# 3^3: 2x2x2 blocks as 6^3 boxes (4x4x4), one block whose members are each other's periodic
# neighbours (2x2x2), and patches that form no block (2x2x1: the z neighbour is the patch itself)
SIZES_3D = [((4, 4, 4), 3), ((2, 2, 2), 3), ((2, 2, 1), 3), ((4, 4, 2), 2), ((3, 2, 2), 4), ((3, 3, 3), 6),
            ((2, 2, 2), 5), ((2, 2, 2), 12), ((2, 1, 1), 20), ((2, 2, 2), 7)]


def _stage(torch, orc, mesh, pde, dim, qs, q0, mat, coef, params=None, lam=True):
    a, b, g = coef
    dt = 1.3e-3
    ref = np.zeros_like(qs)
    lam_ref = orc.stage(FV, pde, dim, mesh.patches, 1, mesh.var_stride, qs, q0=q0 if a else None, out=ref,
                        mat=mat, dt=dt, a=a, b=b, g=g, want_lam=lam, params=params)
    with dh.Plan(pde, dim, mesh.patches, 1, mesh.var_stride, params) as plan:
        d_qs, d_q0 = dev(torch, qs), dev(torch, q0)
        d_mat = dev(torch, mat) if mat is not None else None
        d_out = torch.zeros_like(d_qs)
        d_dt = torch.tensor([dt], dtype=torch.float64, device="cuda")
        d_lam = torch.zeros(1, dtype=torch.float64, device="cuda") if lam else None
        dh.patch_update_fv(plan, d_qs, d_q0 if a else None, d_out, None, d_mat, d_dt, a, b, g, 0.0, d_lam)
        torch.cuda.synchronize()
        out = host(d_out)
        got_lam = float(host(d_lam)[0]) if lam else None
    return out, ref, got_lam, lam_ref


@pytest.mark.parametrize("n,p", SIZES_3D)
@pytest.mark.parametrize("coef", [(0.0, 1.0, 1.0), (0.75, 0.25, 0.25)])
def test_euler3d_odd_patch_sizes(orc, n, p, coef):
    torch = require_cuda()
    mesh = single_level(n, p, 1.0 / 64)
    pde = synth.PDE_EULER3D
    q0 = orc.prim2con(pde, synth.euler_prims(mesh, 41), mesh.var_stride)
    qs = orc.prim2con(pde, synth.euler_prims(mesh, 42), mesh.var_stride)
    out, ref, lam, lam_ref = _stage(torch, orc, mesh, pde, 3, qs, q0, None, coef)
    worst = assert_parity(out, ref, voxel_mask(mesh), what=f"euler3d p={p}")
    assert abs(lam - lam_ref) <= 1e-14 * lam_ref
    print(f"p = {p}: max relative error {worst:.2e}")


@pytest.mark.parametrize("n,p", [((3, 3), 5), ((2, 2), 20), ((4, 2), 3), ((2, 2), 12)])
def test_euler2d_odd_patch_sizes(orc, n, p):
    torch = require_cuda()
    mesh = single_level(n, p, 1.0 / 64, dim=2)
    pde = synth.PDE_EULER2D
    qs = orc.prim2con(pde, synth.euler_prims(mesh, 43), mesh.var_stride)
    params = np.array([1.3])
    out, ref, lam, lam_ref = _stage(torch, orc, mesh, pde, 2, qs, qs, None, (1 / 3, 2 / 3, 2 / 3), params)
    assert_parity(out, ref, voxel_mask(mesh), what=f"euler2d p={p}")
    assert abs(lam - lam_ref) <= 1e-14 * lam_ref


@pytest.mark.parametrize("pde", [synth.PDE_ADV_FLUX, synth.PDE_ADV_NCP])
@pytest.mark.parametrize("n,p", [((3, 3, 3), 3), ((2, 2, 2), 6), ((1, 2, 1), 10)])
def test_advection_with_material_odd_sizes(orc, pde, n, p):
    torch = require_cuda()
    mesh = single_level(n, p, 1.0 / 32)
    rng = np.random.default_rng(44)
    qs = rng.uniform(0.5, 1.5, (1, mesh.var_stride))
    mat = rng.uniform(-1.0, 1.0, (3, mesh.var_stride))
    out, ref, lam, lam_ref = _stage(torch, orc, mesh, pde, 3, qs, qs, mat, (0.0, 1.0, 1.0))
    assert_parity(out, ref, voxel_mask(mesh), what=f"advection pde {pde} p={p}")
    assert abs(lam - lam_ref) <= 1e-14 * lam_ref


def test_srhd_odd_patch_size(orc):
    torch = require_cuda()
    mesh = single_level((3, 3, 3), 6, 1.0 / 64)
    n = mesh.var_stride
    w = synth.srhd_iid_prims(n, 45, wmax=3.0)
    q = orc.prim2con(synth.PDE_SRHD3D, w, n)
    out, ref, _, _ = _stage(torch, orc, mesh, synth.PDE_SRHD3D, 3, q, q, w, (0.0, 1.0, 1.0),
                            params=np.array([5.0 / 3.0]), lam=False)
    assert_parity(out, ref, voxel_mask(mesh), what="srhd p=6")


def test_mixed_patch_sizes_one_plan(orc):
    """Two levels, 3^3 and 16^3 patches: the plan is generic, so both run the generic kernel."""
    torch = require_cuda()
    mesh = synth.make_mesh([synth.Level((4, 4, 4), 3, 1.0 / 48, 0), synth.Level((2, 1, 1), 16, 1.0 / 32, 1)], dim=3)
    pde = synth.PDE_EULER3D
    qs = orc.prim2con(pde, synth.euler_prims(mesh, 46), mesh.var_stride)
    out, ref, lam, lam_ref = _stage(torch, orc, mesh, pde, 3, qs, qs, None, (0.75, 0.25, 0.25))
    assert_parity(out, ref, voxel_mask(mesh), what="mixed 3^3 + 16^3")
    assert abs(lam - lam_ref) <= 1e-14 * lam_ref


@pytest.mark.parametrize("n,p", [((3, 3, 3), 6), ((2, 2, 2), 12)])
def test_ssprk3_steps_and_graph_odd_sizes(orc, n, p):
    """Whole SSP-RK3 steps with the device-side CFL step, eagerly (stage-sum form) and as a captured
    multi-step graph (derived quantities handed from stage to stage, dt written by each step's
    last stage), against the oracle's Shu-Osher steps; graph and eager bitwise equal."""
    torch = require_cuda()
    mesh = single_level(n, p, 1.0 / 64)
    pde = synth.PDE_EULER3D
    q = orc.prim2con(pde, synth.euler_prims(mesh, 47), mesh.var_stride)
    ref = q.copy()
    orc.rk_steps(FV, pde, 3, mesh.patches, 1, mesh.var_stride, ref, rk=3, steps=3, cfl=0.4)
    res = []
    for graph in (False, True):
        with dh.Plan(pde, 3, mesh.patches, 1, mesh.var_stride) as plan:
            Q = dev(torch, q)
            U1, U2, R = torch.zeros_like(Q), torch.zeros_like(Q), torch.zeros_like(Q)
            lam = torch.zeros(1, dtype=torch.float64, device="cuda")
            dt = torch.zeros(1, dtype=torch.float64, device="cuda")
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                dh.max_wave_speed(plan, Q, None, lam)
                if graph:
                    dh.dh_rk_step(plan, FV, 3, Q.clone(), U1, U2, R, None, dt.clone(), lam.clone(), 0.4, 0.0, s)
                    s.synchronize()
                    dh.dh_graph_capture(plan, FV, 3, 3, Q, U1, U2, R, None, dt, lam, 0.4, 0.0, 0, s)
                    dh.dh_graph_launch(plan, s)
                else:
                    for _ in range(3):
                        dh.dh_rk_step(plan, FV, 3, Q, U1, U2, R, None, dt, lam, 0.4, 0.0, s)
            s.synchronize()
            res.append(host(Q))
    m = voxel_mask(mesh)
    assert_parity(res[0], ref, m, what=f"SSP-RK3 p={p}")
    assert np.array_equal(res[0][:, m], res[1][:, m])


def test_paths_needing_multiples_of_8_refuse(orc):
    torch = require_cuda()
    mesh = single_level((2, 2, 2), 6, 1.0 / 64)
    with dh.Plan(synth.PDE_WAVE3D, 3, mesh.patches, 3, mesh.var_stride) as plan:
        q = torch.zeros((5, mesh.var_stride), dtype=torch.float64, device="cuda")
        c = torch.ones((1, mesh.var_stride), dtype=torch.float64, device="cuda")
        dt = torch.tensor([1e-3], dtype=torch.float64, device="cuda")
        with pytest.raises(dh.DhError) as e:
            dh.patch_update_fd_ko(plan, q, None, torch.zeros_like(q), None, c, dt, 0, 1, 1, 0, 0.1)
        assert e.value.status == dh.DH_EUNSUPPORTED
    with dh.Plan(synth.PDE_EULER3D, 3, mesh.patches, 2, mesh.var_stride) as plan:
        q = torch.ones((5, mesh.var_stride), dtype=torch.float64, device="cuda")
        dt = torch.tensor([1e-3], dtype=torch.float64, device="cuda")
        with pytest.raises(dh.DhError) as e:
            dh.patch_update_fv_muscl(plan, q, None, torch.zeros_like(q), None, None, dt, 0, 1, 1, 0)
        assert e.value.status == dh.DH_EUNSUPPORTED
