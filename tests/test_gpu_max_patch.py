"""GPU parity at the largest patch the plans accept: one self-periodic patch of 256^3 voxels
(16.8 M voxels, 134 MB per quantity), against the oracle after one stage, for the first-order FV
stage (the z-marching kernel), the generic FV stage on 255^3 (ragged boxes at the patch's upper
ends), the MUSCL stage and the FD4 + Kreiss-Oliger stage.  These exercise the index arithmetic of
every kernel at the top of its range (256 planes per column, 2^24 voxels per quantity).

Tolerance: 1e-12 relative per voxel, relative to max(|r|, s_v)."""
import numpy as np
import pytest

from gpu_util import assert_parity, dev, host, require_cuda
from helpers import single_level, voxel_mask
from paper_2608_19273_gb300 import dh, synth

pytestmark = pytest.mark.gpu
FV, FD, FV2 = 0, 1, 2


def _euler_stage(torch, orc, scheme, p, seed):
    mesh = single_level((1, 1, 1), p, 1.0 / p)
    qs = orc.prim2con(3, synth.euler_prims(mesh, seed), mesh.var_stride)
    halo = 2 if scheme == FV2 else 1
    dt = 0.2 / p
    ref = np.zeros_like(qs)
    lam_ref = orc.stage(scheme, 3, 3, mesh.patches, halo, mesh.var_stride, qs, out=ref, dt=dt, a=0.0, b=1.0, g=1.0,
                        want_lam=True)
    with dh.Plan(3, 3, mesh.patches, halo, mesh.var_stride) as plan:
        d_out = torch.zeros(qs.shape, dtype=torch.float64, device="cuda")
        d_dt = torch.tensor([dt], dtype=torch.float64, device="cuda")
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        update = dh.patch_update_fv_muscl if scheme == FV2 else dh.patch_update_fv
        update(plan, dev(torch, qs), None, d_out, None, None, d_dt, 0.0, 1.0, 1.0, 0.0, lam)
        torch.cuda.synchronize()
        got, got_lam = host(d_out), float(host(lam)[0])
    assert abs(got_lam - lam_ref) <= 1e-14 * lam_ref
    return got, ref, mesh


@pytest.mark.parametrize("p", [256, 255])
def test_euler3d_fv_stage_largest_patch(orc, p):
    """p = 256 runs the z-marching stage (16x16 columns, 256 planes); p = 255 the generic stage."""
    torch = require_cuda()
    got, ref, mesh = _euler_stage(torch, orc, FV, p, 81)
    assert_parity(got, ref, voxel_mask(mesh), what=f"FV stage p={p}")


def test_euler3d_muscl_stage_largest_patch(orc):
    torch = require_cuda()
    got, ref, mesh = _euler_stage(torch, orc, FV2, 256, 82)
    assert_parity(got, ref, voxel_mask(mesh), what="MUSCL stage p=256")


def test_wave_fd_stage_largest_patch(orc):
    torch = require_cuda()
    mesh = single_level((1, 1, 1), 256, 1.0 / 256)
    q, mat = synth.wave_initial(mesh, 83)
    params = np.array([0.1])
    dt = 0.05 / 256
    ref, acc_ref = np.zeros_like(q), q.copy()
    lam_ref = orc.stage(FD, synth.PDE_WAVE3D, 3, mesh.patches, 3, mesh.var_stride, q, out=ref, acc=acc_ref, mat=mat,
                        dt=dt, a=0.0, b=1.0, g=0.5, d=1 / 6, sigma=0.1, params=params, want_lam=True)
    with dh.Plan(synth.PDE_WAVE3D, 3, mesh.patches, 3, mesh.var_stride, params) as plan:
        d_out = torch.zeros(q.shape, dtype=torch.float64, device="cuda")
        d_acc = dev(torch, q)
        d_dt = torch.tensor([dt], dtype=torch.float64, device="cuda")
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dh.patch_update_fd_ko(plan, dev(torch, q), None, d_out, d_acc, dev(torch, mat), d_dt, 0.0, 1.0, 0.5, 1 / 6,
                              0.1, lam)
        torch.cuda.synchronize()
        got, got_acc, got_lam = host(d_out), host(d_acc), float(host(lam)[0])
    m = voxel_mask(mesh)
    assert_parity(got, ref, m, what="FD stage p=256 out")
    assert_parity(got_acc, acc_ref, m, what="FD stage p=256 acc")
    assert got_lam == lam_ref
