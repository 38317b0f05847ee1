"""GPU parity of offload mode (dh_offload_bind / dh_offload_run): AoAoS patch
blocks in page-locked host memory are gathered in place, advanced on the
device and scattered back (paper Sec. III-C/D, Sec. IV).  Reference: the
oracle's gather, Runge-Kutta steps and scatter on the same blocks."""
import numpy as np
import pytest

from gpu_util import assert_parity, require_cuda
from helpers import voxel_mask
from oracle import aoas
from paper_2608_19273_gb300 import dh, synth

pytestmark = pytest.mark.gpu
FV, FD = 0, 1


def pinned_blocks(torch, mesh, nq, halo, host_blocks, seed):
    """Copy numpy blocks into one page-locked buffer, blocks in shuffled order with gaps."""
    lens = [len(b) for b in host_blocks]
    order = np.random.default_rng(seed).permutation(len(lens))
    starts = np.zeros(len(lens), dtype=np.int64)
    pos = 0
    for k in order:
        starts[k] = pos
        pos += lens[k] + 5
    buf = torch.zeros(pos, dtype=torch.float64).pin_memory()   # the gaps too: buffers compare whole
    views = []
    for k, b in enumerate(host_blocks):
        v = buf[int(starts[k]):int(starts[k]) + lens[k]]
        v.copy_(torch.from_numpy(b))
        views.append(v)
    return buf, views


def blocks_from_arena(mesh, arena_rows, nq, halo, seed):
    """AoS blocks whose interior is the given arena and whose halo holds seeded junk."""
    rng = np.random.default_rng(seed)
    blocks = [rng.standard_normal(aoas.block_len(int(pt["p"]), mesh.dim, nq, halo)) for pt in mesh.patches]
    aoas.scatter_aoas(mesh.patches, np.ascontiguousarray(arena_rows).ravel(), blocks, nq, halo, mesh.var_stride,
                      mesh.dim)
    return blocks


def run_offload(torch, plan, mesh, views, nq, halo, n_q, scheme, rk, steps, cfl, nq_back, staged=False):
    (dh.dh_offload_bind_staged if staged else dh.dh_offload_bind)(plan, views, nq, halo)
    arena = torch.zeros(nq * mesh.var_stride, dtype=torch.float64, device="cuda")
    u1 = torch.zeros(n_q * mesh.var_stride, dtype=torch.float64, device="cuda")
    u2 = torch.zeros_like(u1) if rk >= 3 else None
    acc = torch.zeros_like(u1) if rk == 4 else None
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    lam = torch.zeros(1, dtype=torch.float64, device="cuda")
    dh.dh_offload_run(plan, scheme, rk, steps, arena, u1, u2, acc, dt, lam, cfl, 0.1, nq_back)
    torch.cuda.synchronize()
    return float(dt.item())


@pytest.mark.parametrize("staged", [False, True])
@pytest.mark.parametrize("mesh_kind", ["amr_mix", "p6"])
def test_offload_euler3d_ssprk3(orc, staged, mesh_kind):
    torch = require_cuda()
    # the AMR mix, or 6^3 patches (the paper's typical cells; the generic FV stage)
    mesh = (synth.euler3d_amr_mesh(scale=4) if mesh_kind == "amr_mix"
            else synth.make_mesh([synth.Level((4, 4, 3), 6, 1.0 / 24, 0)], dim=3))
    q = orc.prim2con(3, synth.euler_prims(mesh, 41), mesh.var_stride)
    halo = 1
    blocks = blocks_from_arena(mesh, q, 5, halo, 7)
    ref_q = q.copy()
    dts = orc.rk_steps(FV, 3, 3, mesh.patches, 1, mesh.var_stride, ref_q, rk=3, steps=3, cfl=0.4)
    ref_blocks = [b.copy() for b in blocks]
    aoas.scatter_aoas(mesh.patches, ref_q.ravel(), ref_blocks, 5, halo, mesh.var_stride, 3)
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        buf, views = pinned_blocks(torch, mesh, 5, halo, blocks, 3)
        dt = run_offload(torch, plan, mesh, views, 5, halo, 5, FV, 3, 3, 0.4, 5, staged)
    # compare through the oracle gather (interior) and bitwise on the halo entries
    got_arena = aoas.gather_aoas(mesh.patches, [v.numpy() for v in views], 5, halo, mesh.var_stride, 3)
    assert_parity(got_arena.reshape(5, -1), ref_q, voxel_mask(mesh), what="offload euler3d")
    for k, v in enumerate(views):
        g, r = v.numpy(), ref_blocks[k]
        inner = np.zeros(len(g), dtype=bool)
        aoas._interior(inner, int(mesh.patches[k]["p"]), 3, 5, halo)[...] = True
        assert np.array_equal(g[~inner], r[~inner]), f"halo of block {k} changed"
    assert abs(dt - dts[-1]) <= 1e-14 * dts[-1]


@pytest.mark.parametrize("staged", [False, True])
def test_offload_wave_rk4_with_material(orc, staged):
    """Wave system: 6 quantities per voxel (5 evolved + c); only the 5 evolved ones are written back
    (staged: the whole span goes back, the material and halos as they were read)."""
    torch = require_cuda()
    w = synth.workload("wave3d", scale=8)
    mesh = w.mesh
    q, mat = synth.wave_initial(mesh, w.seed)
    full = np.concatenate([q, mat], axis=0)
    halo = 3
    blocks = blocks_from_arena(mesh, full, 6, halo, 11)
    ref_q = q.copy()
    orc.rk_steps(FD, synth.PDE_WAVE3D, 3, mesh.patches, 3, mesh.var_stride, ref_q, mat=mat, rk=4, steps=2,
                 cfl=w.cfl, sigma=0.1, params=w.params)
    with dh.Plan(synth.PDE_WAVE3D, 3, mesh.patches, 3, mesh.var_stride, w.params) as plan:
        buf, views = pinned_blocks(torch, mesh, 6, halo, blocks, 4)
        run_offload(torch, plan, mesh, views, 6, halo, 5, FD, 4, 2, w.cfl, 5, staged)
    got = aoas.gather_aoas(mesh.patches, [v.numpy() for v in views], 6, halo, mesh.var_stride, 3).reshape(6, -1)
    assert_parity(got[:5], ref_q, voxel_mask(mesh), what="offload wave")
    assert np.array_equal(got[5][voxel_mask(mesh)], mat[0][voxel_mask(mesh)]), "material must come back unchanged"


@pytest.mark.parametrize("staged", [False, True])
def test_offload_zero_steps_round_trip(staged):
    torch = require_cuda()
    mesh = synth.make_mesh([synth.Level((2, 2, 2), 8, 1.0 / 16, 0)], dim=3)
    rng = np.random.default_rng(5)
    blocks = [rng.standard_normal(aoas.block_len(8, 3, 5, 2)) for _ in mesh.patches]
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        buf, views = pinned_blocks(torch, mesh, 5, 2, blocks, 6)
        run_offload(torch, plan, mesh, views, 5, 2, 5, FV, 3, 0, 0.0, 5, staged)
        for k, v in enumerate(views):
            assert np.array_equal(v.numpy(), blocks[k])


def test_offload_bind_rejects_pageable_memory():
    torch = require_cuda()
    mesh = synth.make_mesh([synth.Level((2, 2, 2), 8, 1.0 / 16, 0)], dim=3)
    pageable = [np.zeros(aoas.block_len(8, 3, 5, 0)) for _ in mesh.patches]
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        with pytest.raises(dh.DhError):
            dh.dh_offload_bind(plan, [int(b.ctypes.data) for b in pageable], 5, 0)
        with pytest.raises(dh.DhError):   # nq below N + M
            dh.dh_offload_bind(plan, [int(b.ctypes.data) for b in pageable], 4, 0)
        arena = torch.zeros(5 * mesh.var_stride, dtype=torch.float64, device="cuda")
        with pytest.raises(dh.DhError):   # nothing bound
            dh.dh_offload_run(plan, FV, 3, 1, arena, None, None, None, None, None, 0.0, 0.1, 5)


@pytest.mark.parametrize("staged", [False, True])
def test_two_offload_problems_on_two_streams(orc, staged):
    """Two independent problems (own plans, host blocks and device buffers) enqueued on two streams,
    so that one's host transfers can overlap the other's compute: each ends bitwise equal to the
    same problem advanced alone, and agrees with the oracle."""
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=4)
    qs = [orc.prim2con(3, synth.euler_prims(mesh, 51 + i), mesh.var_stride) for i in range(2)]
    halo, steps = 1, 2
    res = {}
    for mode in ("alone", "together"):
        plans = [dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) for _ in range(2)]
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        bufs, views, dev = [], [], []
        for i in range(2):
            b, v = pinned_blocks(torch, mesh, 5, halo, blocks_from_arena(mesh, qs[i], 5, halo, 60 + i), 70 + i)
            bufs.append(b)
            views.append(v)
            (dh.dh_offload_bind_staged if staged else dh.dh_offload_bind)(plans[i], v, 5, halo)
            z = lambda: torch.zeros(5 * mesh.var_stride, dtype=torch.float64, device="cuda")
            dev.append((z(), z(), z(), z(), torch.zeros(1, dtype=torch.float64, device="cuda"),
                        torch.zeros(1, dtype=torch.float64, device="cuda")))
        torch.cuda.synchronize()
        for i in range(2):
            arena, u1, u2, acc, dt, lam = dev[i]
            s = streams[0] if mode == "alone" else streams[i]
            dh.dh_offload_run(plans[i], FV, 3, steps, arena, u1, u2, acc, dt, lam, 0.4, 0.1, 5, s)
            if mode == "alone":
                s.synchronize()
        torch.cuda.synchronize()
        res[mode] = (bufs, views)
        for p in plans:
            p.close()
    for i in range(2):
        for k, (a, b) in enumerate(zip(res["alone"][1][i], res["together"][1][i])):
            assert torch.equal(a, b), f"problem {i}, block {k} differs when overlapped"
    ref = qs[0].copy()
    orc.rk_steps(FV, 3, 3, mesh.patches, 1, mesh.var_stride, ref, rk=3, steps=steps, cfl=0.4)
    got = aoas.gather_aoas(mesh.patches, [v.numpy() for v in res["together"][1][0]], 5, halo, mesh.var_stride, 3)
    assert_parity(got.reshape(5, -1), ref, voxel_mask(mesh), what="overlapped offload problem 0")


def test_staged_bind_rejections():
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=8)
    lens = [aoas.block_len(int(pt["p"]), 3, 5, 1) for pt in mesh.patches]
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        dev_blocks = [torch.zeros(n, dtype=torch.float64, device="cuda") for n in lens]
        with pytest.raises(dh.DhError):          # device memory, not host blocks
            dh.dh_offload_bind_staged(plan, dev_blocks, 5, 1)
        # page-locked blocks 9x the largest block apart: the span is more than 4x the blocks
        gap = 9 * max(lens)
        buf = torch.zeros(gap * len(lens), dtype=torch.float64).pin_memory()
        views = [buf[k * gap:k * gap + n] for k, n in enumerate(lens)]
        with pytest.raises(dh.DhError):
            dh.dh_offload_bind_staged(plan, views, 5, 1)
        # a failed bind leaves the plan unbound: a run is refused
        z = lambda: torch.zeros(5 * mesh.var_stride, dtype=torch.float64, device="cuda")
        one = lambda: torch.zeros(1, dtype=torch.float64, device="cuda")
        with pytest.raises(dh.DhError):
            dh.dh_offload_run(plan, FV, 3, 1, z(), z(), z(), None, one(), one(), 0.0, 0.1, 5)
        dense = [buf[int(a):int(a) + n] for a, n in zip(np.concatenate([[0], np.cumsum(lens)[:-1]]), lens)]
        dh.dh_offload_bind_staged(plan, dense, 5, 1)   # back to back: accepted
