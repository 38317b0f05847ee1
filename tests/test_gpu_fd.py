"""GPU parity of the FD4 + Kreiss-Oliger stage (patch_update_fd_ko) against the FP64 oracle."""
import math

import numpy as np
import pytest

from gpu_util import assert_parity, dev, host, require_cuda
from helpers import arena, from_grid, single_level, to_grid, voxel_mask
from paper_2608_19273_gb300 import dh, synth

pytestmark = pytest.mark.gpu
FD = 1


def _run_stage(torch, plan, q, q0, acc, mat, dt, coef, sigma=0.1, lam=False):
    a, b, g, d = coef
    d_qs = dev(torch, q)
    d_out = torch.zeros_like(d_qs)
    d_acc = dev(torch, acc) if acc is not None else None
    d_lam = torch.zeros(1, dtype=torch.float64, device="cuda") if lam else None
    d_dt = torch.tensor([dt], dtype=torch.float64, device="cuda")
    dh.patch_update_fd_ko(plan, d_qs, dev(torch, q0) if q0 is not None else None, d_out, d_acc,
                          dev(torch, mat) if mat is not None else None, d_dt, a, b, g, d, sigma, d_lam)
    torch.cuda.synchronize()
    return host(d_out), (host(d_acc) if acc is not None else None), (float(host(d_lam)[0]) if lam else None)


@pytest.mark.parametrize("coef", [(0.0, 1.0, 0.5, 1 / 6), (1.0, 0.0, 1.0, 1 / 3)])
def test_wave_stage(orc, coef):
    torch = require_cuda()
    w = synth.workload("wave3d", scale=8)
    mesh = w.mesh
    q, mat = synth.wave_initial(mesh, w.seed)
    q0, _ = synth.wave_initial(mesh, w.seed + 1)
    acc = q0.copy()
    dt = 2e-3
    a, b, g, d = coef
    ref, ref_acc = np.zeros_like(q), acc.copy()
    lam_ref = orc.stage(FD, synth.PDE_WAVE3D, 3, mesh.patches, 3, mesh.var_stride, q, q0=q0 if a else None,
                        out=ref, acc=ref_acc, mat=mat, dt=dt, a=a, b=b, g=g, d=d, sigma=0.1, params=w.params,
                        want_lam=True)
    with dh.Plan(synth.PDE_WAVE3D, 3, mesh.patches, 3, mesh.var_stride, w.params) as plan:
        out, gacc, lam = _run_stage(torch, plan, q, q0 if a else None, acc, mat, dt, coef, lam=True)
    m = voxel_mask(mesh)
    assert_parity(out, ref, m, what="wave stage out")
    assert_parity(gacc, ref_acc, m, what="wave stage acc")
    assert lam == lam_ref


def test_wave_rk4_steps(orc):
    torch = require_cuda()
    w = synth.workload("wave3d", scale=8)
    mesh = w.mesh
    q, mat = synth.wave_initial(mesh, w.seed)
    ref = q.copy()
    dts = orc.rk_steps(FD, synth.PDE_WAVE3D, 3, mesh.patches, 3, mesh.var_stride, ref, mat=mat, rk=4, steps=3,
                       cfl=w.cfl, sigma=0.1, params=w.params)
    with dh.Plan(synth.PDE_WAVE3D, 3, mesh.patches, 3, mesh.var_stride, w.params) as plan:
        Q, M = dev(torch, q), dev(torch, mat)
        U1, U2, ACC = torch.empty_like(Q), torch.empty_like(Q), torch.empty_like(Q)
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        dh.max_wave_speed(plan, Q, M, lam)
        for _ in range(3):
            dh.dh_rk_step(plan, FD, 4, Q, U1, U2, ACC, M, dt, lam, w.cfl, 0.1)
        out = host(Q)
        dt_last = float(host(dt)[0])
    assert_parity(out, ref, voxel_mask(mesh), what="wave 3 RK4 steps")
    assert abs(dt_last - dts[-1]) <= 1e-15 * dts[-1]


@pytest.mark.parametrize("noise", [0.0, 0.05])
def test_gw59_stage(orc, noise):
    torch = require_cuda()
    w = synth.workload("gw59", scale=8)
    mesh = w.mesh
    q = synth.gw59_initial(mesh, w.seed, amp=1e-3, noise=noise)
    q0 = synth.gw59_initial(mesh, w.seed + 5, amp=1e-3, noise=noise)
    acc = q0.copy()
    coef = (1.0, 0.0, 0.5, 1 / 3)
    ref, ref_acc = np.zeros_like(q), acc.copy()
    lam_ref = orc.stage(FD, synth.PDE_GW59, 3, mesh.patches, 3, mesh.var_stride, q, q0=q0, out=ref, acc=ref_acc,
                        dt=1e-3, a=1.0, b=0.0, g=0.5, d=1 / 3, sigma=0.1, params=w.params, want_lam=True)
    with dh.Plan(synth.PDE_GW59, 3, mesh.patches, 3, mesh.var_stride, w.params) as plan:
        out, gacc, lam = _run_stage(torch, plan, q, q0, acc, None, 1e-3, coef, lam=True)
    m = voxel_mask(mesh)
    assert_parity(out, ref, m, what="gw59 out")
    assert_parity(gacc, ref_acc, m, what="gw59 acc")
    assert abs(lam - lam_ref) <= 1e-15 * lam_ref


def test_gw59_rk4_steps(orc):
    torch = require_cuda()
    w = synth.workload("gw59", scale=8)
    mesh = w.mesh
    q = synth.gw59_initial(mesh, w.seed, amp=1e-6)
    ref = q.copy()
    dts = orc.rk_steps(FD, synth.PDE_GW59, 3, mesh.patches, 3, mesh.var_stride, ref, rk=4, steps=2, cfl=w.cfl,
                       sigma=0.1, params=w.params)
    with dh.Plan(synth.PDE_GW59, 3, mesh.patches, 3, mesh.var_stride, w.params) as plan:
        Q = dev(torch, q)
        U1, U2, ACC = torch.empty_like(Q), torch.empty_like(Q), torch.empty_like(Q)
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        dh.max_wave_speed(plan, Q, None, lam)
        for _ in range(2):
            dh.dh_rk_step(plan, FD, 4, Q, U1, U2, ACC, None, dt, lam, w.cfl, 0.1)
        out = host(Q)
    assert_parity(out, ref, voxel_mask(mesh), what="gw59 2 RK4 steps")


def test_ko_checkerboard_gpu(orc):
    torch = require_cuda()
    mesh = single_level((2, 2, 2), 8, 1.0 / 16)
    z, y, x = np.meshgrid(np.arange(16), np.arange(16), np.arange(16), indexing="ij")
    G = (-1.0) ** (x + y + z)
    q = from_grid(mesh, G, arena(mesh, 1)[0])[None].copy()
    mat = arena(mesh, 3)
    with dh.Plan(synth.PDE_ADV_NCP, 3, mesh.patches, 3, mesh.var_stride) as plan:
        out, _, _ = _run_stage(torch, plan, q, None, None, mat, 1.0, (0, 0, 1, 0), sigma=0.1)
    assert np.array_equal(to_grid(mesh, out[0]), -3 * 0.1 * 16 * G)


@pytest.mark.parametrize("pde", [synth.PDE_WAVE3D, synth.PDE_GW59])
def test_fd_free_stream_gpu(orc, pde):
    torch = require_cuda()
    mesh = single_level((2, 1, 2), 16, 1.0 / 32)
    nq = synth.PDE_NQ[pde]
    q = arena(mesh, nq)
    mat = None
    if pde == synth.PDE_WAVE3D:
        q[0] = 0.7
        mat = arena(mesh, 1)
        mat[0] = 1.25 + 0.75 * np.sin(2 * math.pi * synth.voxel_centres(mesh)[0])
        params = [0.1]
    else:
        q[55] = 1.0
        params = synth.workload("gw59", scale=8).params
    with dh.Plan(pde, 3, mesh.patches, 3, mesh.var_stride, params) as plan:
        out, _, _ = _run_stage(torch, plan, q, None, None, mat, 0.3, (0, 1, 1, 0))
    m = voxel_mask(mesh)
    assert np.array_equal(out[:, m], q[:, m])
