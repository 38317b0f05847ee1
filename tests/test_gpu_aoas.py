"""GPU parity of the AoAoS <-> SoA arena gather/scatter (paper Sec. III-C Eq. 4
prologue and epilogue) against the CPU oracle: bit-exact, halo entries of the
blocks and arena padding untouched."""
import numpy as np
import pytest

from gpu_util import dev, host, require_cuda
from oracle import aoas
from paper_2608_19273_gb300 import synth

pytestmark = pytest.mark.gpu

SENT_ARENA = -123.25
SENT_BLOCK = 777.5


def mesh_for(case):
    if case == "euler3d_s4":
        return synth.workload("euler3d", scale=4).mesh
    if case == "gw59_s8":
        return synth.workload("gw59", scale=8).mesh
    if case == "euler2d":
        return synth.workload("euler2d").mesh
    if case == "p8_cube":
        return synth.make_mesh([synth.Level((2, 2, 2), 8, 1.0 / 16, 0)], dim=3)
    if case == "p24_cube":
        return synth.make_mesh([synth.Level((2, 2, 2), 24, 1.0 / 48, 0)], dim=3)
    if case == "p256_2d":
        return synth.make_mesh([synth.Level((2, 1, 1), 256, 1.0 / 512, 0)], dim=2)
    if case == "p3_cube":    # patch sizes that are not multiples of 8 (the paper's 3^3 and 6^3 cells)
        return synth.make_mesh([synth.Level((4, 4, 4), 3, 1.0 / 12, 0)], dim=3)
    if case == "p6_p13_mix":
        return synth.make_mesh([synth.Level((3, 3, 3), 6, 1.0 / 18, 0), synth.Level((2, 1, 1), 13, 1.0 / 26, 1)],
                               dim=3)
    if case == "p5_2d":
        return synth.make_mesh([synth.Level((3, 3, 1), 5, 1.0 / 15, 0)], dim=2)
    raise KeyError(case)


def make_blocks(torch, mesh, nq, halo, seed, separate=True):
    """Seeded AoS blocks (one CUDA tensor per patch, or views of one shuffled buffer)."""
    rng = np.random.default_rng(seed)
    lens = [aoas.block_len(int(pt["p"]), mesh.dim, nq, halo) for pt in mesh.patches]
    host_blocks = [rng.standard_normal(n) for n in lens]
    if separate:
        return host_blocks, [dev(torch, b) for b in host_blocks]
    order = rng.permutation(len(lens))
    starts = np.zeros(len(lens), dtype=np.int64)
    pos = 0
    for k in order:                      # blocks in shuffled order with small gaps
        starts[k] = pos
        pos += lens[k] + 3
    buf = torch.empty(pos, dtype=torch.float64, device="cuda")
    views = []
    for k, b in enumerate(host_blocks):
        v = buf[int(starts[k]):int(starts[k]) + lens[k]]
        v.copy_(torch.from_numpy(b))
        views.append(v)
    return host_blocks, views


def run_case(torch, mesh, nq, halo, seed, separate=True):
    from paper_2608_19273_gb300 import dh
    pde = synth.PDE_EULER2D if mesh.dim == 2 else synth.PDE_EULER3D
    plan = dh.Plan(pde, mesh.dim, mesh.patches, 1, mesh.var_stride)
    hb, db = make_blocks(torch, mesh, nq, halo, seed, separate)
    ptrs = dh.block_pointer_table(db)
    arena_d = torch.full((nq * mesh.var_stride,), SENT_ARENA, dtype=torch.float64, device="cuda")
    dh.dh_gather_aoas(plan, ptrs, nq, halo, arena_d)
    ref = aoas.gather_aoas(mesh.patches, hb, nq, halo, mesh.var_stride, mesh.dim,
                           arena=np.full(nq * mesh.var_stride, SENT_ARENA))
    got = host(arena_d)
    assert np.array_equal(got, ref), f"gather: {np.count_nonzero(got != ref)} elements differ"
    # scatter back into sentinel-filled blocks
    for b in db:
        b.fill_(SENT_BLOCK)
    dh.dh_scatter_aoas(plan, arena_d, ptrs, nq, halo)
    out_ref = aoas.scatter_aoas(mesh.patches, ref, [np.full_like(b, SENT_BLOCK) for b in hb], nq, halo,
                                mesh.var_stride, mesh.dim)
    torch.cuda.synchronize()
    for k, b in enumerate(db):
        g = host(b)
        assert np.array_equal(g, out_ref[k]), f"scatter: patch {k} differs"
    plan.close()


@pytest.mark.parametrize("case,nq,halo", [("euler3d_s4", 5, 0), ("euler3d_s4", 5, 1), ("gw59_s8", 59, 3),
                                          ("euler2d", 4, 1), ("p8_cube", 256, 2), ("p24_cube", 1, 0),
                                          ("p24_cube", 10, 1), ("p8_cube", 23, 8), ("p256_2d", 3, 8),
                                          ("p3_cube", 5, 1), ("p3_cube", 7, 3), ("p6_p13_mix", 5, 1),
                                          ("p6_p13_mix", 59, 2), ("p5_2d", 4, 1)])
def test_gather_scatter_bit_exact(case, nq, halo):
    torch = require_cuda()
    run_case(torch, mesh_for(case), nq, halo, seed=2608 + nq + 17 * halo)


def test_gather_scatter_full_mix_one_buffer():
    """The full 3D Euler AMR mix (4096 x 8^3 + 1024 x 16^3 + 128 x 32^3, 10,485,760 voxels),
    5 quantities, halo 1, blocks as shuffled views of one buffer."""
    torch = require_cuda()
    run_case(torch, synth.workload("euler3d").mesh, 5, 1, seed=26081, separate=False)


def test_gather_rejects_bad_arguments():
    torch = require_cuda()
    from paper_2608_19273_gb300 import dh
    mesh = mesh_for("p8_cube")
    plan = dh.Plan(synth.PDE_EULER3D, 3, mesh.patches, 1, mesh.var_stride)
    _, db = make_blocks(torch, mesh, 5, 0, 1)
    ptrs = dh.block_pointer_table(db)
    arena_d = torch.zeros(5 * mesh.var_stride, dtype=torch.float64, device="cuda")
    for nq, h in ((0, 0), (257, 0), (5, -1), (5, 9)):
        with pytest.raises(dh.DhError):
            dh.dh_gather_aoas(plan, ptrs, nq, h, arena_d)
        with pytest.raises(dh.DhError):
            dh.dh_scatter_aoas(plan, arena_d, ptrs, nq, h)
    with pytest.raises(dh.DhError):
        dh.dh_gather_aoas(plan, None, 5, 0, arena_d)
    with pytest.raises(dh.DhError):
        dh.dh_gather_aoas(plan, ptrs, 5, 0, None)
    plan.close()
