"""GPU parity of the second-order FV stage (patch_update_fv_muscl: MUSCL-minmod
reconstruction feeding the Rusanov flux, the reading of the reconstruction step
of Sec. II-A Eq. 3) against the oracle's scheme 2.  Tolerance: 1e-12 relative
per voxel, relative to max(|r|, s_v)."""
import numpy as np
import pytest

from gpu_util import assert_parity, dev, host, require_cuda
from helpers import arena, single_level, voxel_mask
from paper_2608_19273_gb300 import dh, synth

pytestmark = pytest.mark.gpu
FV2 = 2


@pytest.mark.parametrize("fv2_var", [0, 1, 2])
@pytest.mark.parametrize("scale", [8, 4])
@pytest.mark.parametrize("coef", [(0.0, 1.0, 1.0), (0.75, 0.25, 0.25), (1 / 3, 2 / 3, 2 / 3)])
def test_euler3d_muscl_stage(orc, scale, coef, fv2_var):
    """Every variant of the stage (z-march of whole patches / of 16-plane chunks, 8x8x4 tiles)."""
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=scale)
    q0 = orc.prim2con(3, synth.euler_prims(mesh, 61), mesh.var_stride)
    qs = orc.prim2con(3, synth.euler_prims(mesh, 62), mesh.var_stride)
    a, b, g = coef
    dt = 1.3e-3
    ref = np.zeros_like(qs)
    lam_ref = orc.stage(FV2, 3, 3, mesh.patches, 2, mesh.var_stride, qs, q0=q0 if a else None, out=ref, dt=dt,
                        a=a, b=b, g=g, want_lam=True)
    with dh.Plan(3, 3, mesh.patches, 2, mesh.var_stride) as plan:
        dh.dh_plan_set_variant_muscl(plan, fv2_var)
        out = torch.zeros(qs.shape, dtype=torch.float64, device="cuda")
        d_dt = torch.tensor([dt], dtype=torch.float64, device="cuda")
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dh.patch_update_fv_muscl(plan, dev(torch, qs), dev(torch, q0) if a else None, out, None, None, d_dt, a, b, g,
                                 0, lam)
        got = host(out)
        assert abs(float(host(lam)[0]) - lam_ref) <= 1e-14 * lam_ref
    assert_parity(got, ref, voxel_mask(mesh), what=f"muscl stage {coef}")


@pytest.mark.parametrize("fv2_var", [0, 2])
def test_advection_muscl_stage_with_material_field(orc, fv2_var):
    """ADV_FLUX with a velocity field that varies in space (material M = 3) and rough data."""
    torch = require_cuda()
    mesh = single_level((2, 3, 2), 8, 1.0 / 32)
    rng = np.random.default_rng(63)
    m = voxel_mask(mesh)
    q = arena(mesh, 1)
    q[:, m] = rng.normal(size=(1, int(m.sum())))
    mat = arena(mesh, 3)
    X = synth.voxel_centres(mesh)
    for a in range(3):
        mat[a] = synth.fourier_field(rng, X, [1, 1, 1], 3, 0.2 * (a - 1), 1.0)
    acc0 = rng.normal(size=q.shape)
    ref_out, ref_acc = np.zeros_like(q), acc0.copy()
    orc.stage(FV2, synth.PDE_ADV_FLUX, 3, mesh.patches, 2, mesh.var_stride, q, out=ref_out, acc=ref_acc, mat=mat,
              dt=2e-3, a=0, b=1, g=0.5, d=1 / 6)
    with dh.Plan(synth.PDE_ADV_FLUX, 3, mesh.patches, 2, mesh.var_stride) as plan:
        dh.dh_plan_set_variant_muscl(plan, fv2_var)
        out = torch.zeros(q.shape, dtype=torch.float64, device="cuda")
        acc = dev(torch, acc0)
        d_dt = torch.tensor([2e-3], dtype=torch.float64, device="cuda")
        dh.patch_update_fv_muscl(plan, dev(torch, q), None, out, acc, dev(torch, mat), d_dt, 0, 1, 0.5, 1 / 6)
        assert_parity(host(out), ref_out, m, what="muscl advection out")
        assert_parity(host(acc), ref_acc, m, what="muscl advection acc")


def test_euler3d_muscl_ssprk3_steps(orc):
    """Three SSP-RK3 steps with device-computed dt through dh_rk_step (scheme 2)."""
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=4)
    q = orc.prim2con(3, synth.euler_prims(mesh, 64), mesh.var_stride)
    ref = q.copy()
    dts = orc.rk_steps(FV2, 3, 3, mesh.patches, 2, mesh.var_stride, ref, rk=3, steps=3, cfl=0.4)
    with dh.Plan(3, 3, mesh.patches, 2, mesh.var_stride) as plan:
        Q = dev(torch, q)
        U1, U2 = torch.zeros_like(Q), torch.zeros_like(Q)
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        dh.max_wave_speed(plan, Q, None, lam)
        for _ in range(3):
            dh.dh_rk_step(plan, FV2, 3, Q, U1, U2, None, None, dt, lam, 0.4, 0.0)
        out = host(Q)
        dt_last = float(host(dt)[0])
    assert_parity(out, ref, voxel_mask(mesh), what="muscl 3 SSP-RK3 steps")
    assert abs(dt_last - dts[-1]) <= 1e-14 * dts[-1]


def test_muscl_free_stream_bitwise_gpu():
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=8)
    q = arena(mesh, 5)
    for v, c in enumerate([1.3, 0.37, -0.21, 0.11, 2.9]):
        q[v, :] = c
    with dh.Plan(3, 3, mesh.patches, 2, mesh.var_stride) as plan:
        out = torch.zeros(q.shape, dtype=torch.float64, device="cuda")
        d_dt = torch.tensor([0.123], dtype=torch.float64, device="cuda")
        dh.patch_update_fv_muscl(plan, dev(torch, q), None, out, None, None, d_dt, 0, 1, 1, 0)
        got = host(out)
    m = voxel_mask(mesh)
    assert np.array_equal(got[:, m], q[:, m])


def test_muscl_rejects_bad_plans():
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=8)
    q = torch.zeros((5, mesh.var_stride), dtype=torch.float64, device="cuda")
    out = torch.zeros_like(q)
    d_dt = torch.tensor([1e-3], dtype=torch.float64, device="cuda")
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:   # halo 1 is too narrow
        with pytest.raises(dh.DhError):
            dh.patch_update_fv_muscl(plan, q, None, out, None, None, d_dt, 0, 1, 1, 0)
    m2 = synth.euler2d_mesh(n=2, p=8)
    q2 = torch.zeros((4, m2.var_stride), dtype=torch.float64, device="cuda")
    with dh.Plan(2, 2, m2.patches, 2, m2.var_stride) as plan:        # 2D is not supported
        with pytest.raises(dh.DhError):
            dh.patch_update_fv_muscl(plan, q2, None, torch.zeros_like(q2), None, None, d_dt, 0, 1, 1, 0)


def test_muscl_variants_agree_bitwise(orc):
    """The z-march and the tile kernel perform the same operations in the same order: their
    results (and lambda) are bitwise equal on rough data."""
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=4)
    rng = np.random.default_rng(64)
    prim = synth.euler_prims(mesh, 65)
    prim[0] *= np.exp(0.3 * rng.normal(size=prim[0].shape))
    prim[4] *= np.exp(0.3 * rng.normal(size=prim[4].shape))
    q = orc.prim2con(3, prim, mesh.var_stride)
    outs = []
    with dh.Plan(3, 3, mesh.patches, 2, mesh.var_stride) as plan:
        for v in (0, 1, 2):
            dh.dh_plan_set_variant_muscl(plan, v)
            out = torch.zeros(q.shape, dtype=torch.float64, device="cuda")
            lam = torch.zeros(1, dtype=torch.float64, device="cuda")
            d_dt = torch.tensor([1e-3], dtype=torch.float64, device="cuda")
            dh.patch_update_fv_muscl(plan, dev(torch, q), None, out, None, None, d_dt, 0, 1, 1, 0, lam)
            outs.append((host(out), float(host(lam)[0])))
    m = voxel_mask(mesh)
    for o, l in outs[1:]:
        assert np.array_equal(o[:, m], outs[0][0][:, m]) and l == outs[0][1]
