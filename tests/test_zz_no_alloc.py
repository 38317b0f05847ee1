"""patch_update_fv_noalloc: the FV stage for callers that cannot allocate device
memory (their framework's pool owns the GPU, or allocation is forbidden after
start-up).  It must give the same result as the plan-based patch_update_fv on
two calls in a row: the second call reuses, and must fully reset, the static
device scratch that the first call left behind.

This file is collected last on purpose, and it also passes on its own in a
fresh process."""
import numpy as np
import pytest

from gpu_util import assert_parity, dev, host, require_cuda
from helpers import voxel_mask
from paper_2608_19273_gb300 import dh, synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_plan_path_twice(orc):
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=4)
    m = voxel_mask(mesh)
    states = [orc.prim2con(3, synth.euler_prims(mesh, s), mesh.var_stride) for s in (71, 72)]
    coefs = [(0.0, 1.0, 1.0), (0.75, 0.25, 0.25)]
    d_dt = torch.tensor([1.3e-3], dtype=torch.float64, device="cuda")
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        for call in range(2):
            qs, q0 = dev(torch, states[call]), dev(torch, states[1 - call])
            a, b, g = coefs[call]
            ref, got = torch.zeros_like(qs), torch.full_like(qs, np.nan)
            lam_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
            lam_got = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
            dh.patch_update_fv(plan, qs, q0 if a else None, ref, None, None, d_dt, a, b, g, 0.0, lam_ref)
            dh.patch_update_fv_noalloc(3, 3, mesh.patches, mesh.var_stride, None, qs, q0 if a else None, got, None,
                                       None, d_dt, a, b, g, 0.0, lam_got)
            torch.cuda.synchronize()
            assert_parity(host(got), host(ref), m, what=f"noalloc call {call}")
            assert abs(float(host(lam_got)[0]) - float(host(lam_ref)[0])) <= 1e-14 * float(host(lam_ref)[0])


def test_noalloc_rejects_oversize(orc):
    require_cuda()
    mesh = synth.make_mesh([synth.Level((1, 1, 1), 8, 1.0 / 8, 0)], dim=3)
    big = np.repeat(mesh.patches, 8193)
    big["nbr"] = 0
    big["offset"] = 0
    with pytest.raises(dh.DhError) as ei:
        dh.patch_update_fv_noalloc(3, 3, big, mesh.var_stride, None, 1, None, 1, None, None, 1, 0, 1, 1, 0)
    assert ei.value.status == dh.DH_EINVAL


def test_noalloc_rejects_patch_sizes_not_multiples_of_8(orc):
    """6^3 patches, which a plan accepts (generic stage), are refused here before any launch."""
    require_cuda()
    mesh = synth.make_mesh([synth.Level((2, 2, 2), 6, 1.0 / 12, 0)], dim=3)
    with pytest.raises(dh.DhError) as ei:
        dh.patch_update_fv_noalloc(3, 3, mesh.patches, mesh.var_stride, None, 1, None, 1, None, None, 1, 0, 1, 1, 0)
    assert ei.value.status == dh.DH_EINVAL


def test_noalloc_euler2d_gamma_matches_plan_path(orc):
    """2D Euler with a non-default ratio of specific heats (gamma = 5/3, passed in params) on two
    calls in a row, against the plan path with the same parameter."""
    torch = require_cuda()
    w = synth.workload("euler2d")
    mesh = w.mesh
    m = voxel_mask(mesh)
    params = np.array([5.0 / 3.0])
    d_dt = torch.tensor([2.1e-3], dtype=torch.float64, device="cuda")
    with dh.Plan(2, 2, mesh.patches, 1, mesh.var_stride, params) as plan:
        for call, seed in enumerate((81, 82)):
            qs = dev(torch, orc.prim2con(2, synth.euler_prims(mesh, seed), mesh.var_stride, params=params))
            ref, got = torch.zeros_like(qs), torch.full_like(qs, np.nan)
            lam_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
            lam_got = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
            dh.patch_update_fv(plan, qs, None, ref, None, None, d_dt, 0.0, 1.0, 1.0, 0.0, lam_ref)
            dh.patch_update_fv_noalloc(2, 2, mesh.patches, mesh.var_stride, params, qs, None, got, None, None, d_dt,
                                       0.0, 1.0, 1.0, 0.0, lam_got)
            torch.cuda.synchronize()
            assert_parity(host(got), host(ref), m, what=f"noalloc euler2d call {call}")
            assert abs(float(host(lam_got)[0]) - float(host(lam_ref)[0])) <= 1e-14 * float(host(lam_ref)[0])
