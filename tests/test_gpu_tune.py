"""Every compiled kernel variant gives the oracle's result, and the autotuner
picks one of them and caches its choice."""
import numpy as np
import pytest

from gpu_util import assert_parity, dev, host, require_cuda
from helpers import voxel_mask
from paper_2608_19273_gb300 import dh, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fv_var", [0, 1, 2, 3])
@pytest.mark.parametrize("fv_zs", [0, 1])
def test_fv_variants_match_oracle(orc, fv_var, fv_zs):
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=4)
    qs = orc.prim2con(3, synth.euler_prims(mesh, 91), mesh.var_stride)
    q0 = orc.prim2con(3, synth.euler_prims(mesh, 92), mesh.var_stride)
    ref = np.zeros_like(qs)
    lam_ref = orc.stage(0, 3, 3, mesh.patches, 1, mesh.var_stride, qs, q0=q0, out=ref, dt=1e-3, a=0.75, b=0.25,
                        g=0.25, want_lam=True)
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        dh.dh_plan_set_variant(plan, fv_var, fv_zs, 0)
        out = torch.zeros(qs.shape, dtype=torch.float64, device="cuda")
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        d_dt = torch.tensor([1e-3], dtype=torch.float64, device="cuda")
        dh.patch_update_fv(plan, dev(torch, qs), dev(torch, q0), out, None, None, d_dt, 0.75, 0.25, 0.25, 0, lam)
        got = host(out)
        assert abs(float(host(lam)[0]) - lam_ref) <= 1e-14 * lam_ref
    assert_parity(got, ref, voxel_mask(mesh), what=f"variant {fv_var}/{fv_zs}")


@pytest.mark.parametrize("fd_var", [0, 2, 4, 6, 12, 20])
@pytest.mark.parametrize("pde", [synth.PDE_WAVE3D, synth.PDE_GW59])
def test_fd_variants_match_oracle(orc, fd_var, pde):
    torch = require_cuda()
    if pde == synth.PDE_GW59 and fd_var in (12, 20):
        with dh.Plan(pde, 3, synth.workload("gw59", scale=8).mesh.patches, 3,
                     synth.workload("gw59", scale=8).mesh.var_stride, synth.workload("gw59", scale=8).params) as plan:
            with pytest.raises(dh.DhError):
                dh.dh_plan_set_variant(plan, 2, 0, fd_var)
        return
    name = "wave3d" if pde == synth.PDE_WAVE3D else "gw59"
    w = synth.workload(name, scale=8)
    mesh = w.mesh
    if pde == synth.PDE_WAVE3D:
        q, mat = synth.wave_initial(mesh, w.seed)
    else:
        q, mat = synth.gw59_initial(mesh, w.seed, amp=1e-3, noise=0.05), None
    ref = np.zeros_like(q)
    orc.stage(1, pde, 3, mesh.patches, 3, mesh.var_stride, q, out=ref, mat=mat, dt=2e-3, sigma=0.1, params=w.params)
    with dh.Plan(pde, 3, mesh.patches, 3, mesh.var_stride, w.params) as plan:
        dh.dh_plan_set_variant(plan, 2, 0, fd_var)
        out = torch.zeros(q.shape, dtype=torch.float64, device="cuda")
        d_dt = torch.tensor([2e-3], dtype=torch.float64, device="cuda")
        dh.patch_update_fd_ko(plan, dev(torch, q), None, out, None, dev(torch, mat) if mat is not None else None, d_dt,
                              0, 1, 1, 0, 0.1)
        got = host(out)
    assert_parity(got, ref, voxel_mask(mesh), what=f"fd variant {fd_var}")


def test_autotune_picks_and_caches(orc, tmp_path):
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=4)
    qs = dev(torch, orc.prim2con(3, synth.euler_prims(mesh, 93), mesh.var_stride))
    out = torch.zeros_like(qs)
    d_dt = torch.tensor([1e-3], dtype=torch.float64, device="cuda")
    cache = str(tmp_path / "tune.jsonl")
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        v, z, f, cached, times = dh.dh_autotune(plan, 0, qs, out, None, d_dt, reps=2, cache_path=cache)
        assert not cached and 0 <= v <= 3 and z in (0, 1)
        assert all(t > 0 for t in times) and min(times) == times[z * 4 + v]
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        v2, z2, f2, cached2, _ = dh.dh_autotune(plan, 0, qs, out, None, d_dt, reps=2, cache_path=cache)
        assert cached2 and (v2, z2, f2) == (v, z, f)


def test_fd_tma_on_single_self_periodic_patch(orc):
    """TMA staging when every face neighbour is the patch itself (all slabs wrap around)."""
    torch = require_cuda()
    mesh = synth.make_mesh([synth.Level((1, 1, 1), 16, 1.0 / 16, 0)], dim=3)
    q, mat = synth.wave_initial(mesh, 3)
    ref = np.zeros_like(q)
    orc.stage(1, synth.PDE_WAVE3D, 3, mesh.patches, 3, mesh.var_stride, q, out=ref, mat=mat, dt=1e-3, sigma=0.1,
              params=[0.1])
    with dh.Plan(synth.PDE_WAVE3D, 3, mesh.patches, 3, mesh.var_stride, [0.1]) as plan:
        dh.dh_plan_set_variant(plan, 2, 0, 6)
        out = torch.zeros(q.shape, dtype=torch.float64, device="cuda")
        d_dt = torch.tensor([1e-3], dtype=torch.float64, device="cuda")
        dh.patch_update_fd_ko(plan, dev(torch, q), None, out, None, dev(torch, mat), d_dt, 0, 1, 1, 0, 0.1)
        got = host(out)
        assert dh.dh_plan_errors(plan) == 0
    assert_parity(got, ref, voxel_mask(mesh), what="tma self-periodic")


def test_fd_tma_bounded_wait_reports_timeout(orc):
    """With the test hook that arms the TMA barriers but issues no copy, every wait runs out:
    the kernel skips its tiles, raises the error flag and the context stays usable."""
    torch = require_cuda()
    mesh = synth.make_mesh([synth.Level((1, 1, 1), 16, 1.0 / 16, 0)], dim=3)
    q, mat = synth.wave_initial(mesh, 4)
    with dh.Plan(synth.PDE_WAVE3D, 3, mesh.patches, 3, mesh.var_stride, [0.1]) as plan:
        dh.dh_plan_set_variant(plan, 2, 0, 6)
        dh.dh_plan_set_debug(plan, 1)
        out = torch.full(q.shape, float("nan"), dtype=torch.float64, device="cuda")
        d_dt = torch.tensor([1e-3], dtype=torch.float64, device="cuda")
        dh.patch_update_fd_ko(plan, dev(torch, q), None, out, None, dev(torch, mat), d_dt, 0, 1, 1, 0, 0.1)
        torch.cuda.synchronize()
        assert dh.dh_plan_errors(plan) & 1
        assert torch.isnan(out).all()          # every tile was skipped
        dh.dh_plan_set_debug(plan, 0)
        dh.patch_update_fd_ko(plan, dev(torch, q), None, out, None, dev(torch, mat), d_dt, 0, 1, 1, 0, 0.1)
        torch.cuda.synchronize()
        assert dh.dh_plan_errors(plan) == 0
        assert torch.isfinite(out[:, :16 ** 3]).all()
