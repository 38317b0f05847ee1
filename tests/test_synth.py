"""The seeded synthetic inputs: workload sizes, patch tables and field ranges (CPU only).

The patch tables are shared by the CUDA path and the oracle, so a mistake in
them would not show up as a parity failure; these tests check them against
their geometric definition instead (periodic boxes tiled by patches, x
fastest, one box per refinement level; a finer level covering a block of
coarse patches with ratio 2)."""
import numpy as np
import pytest

from paper_2608_19273_gb300 import synth

# name -> ({p: patches of that size}, voxels)
SIZES = {
    "euler2d": ({16: 64}, 64 * 16 ** 2),
    "euler3d": ({8: 4096, 16: 1024, 32: 128}, 10_485_760),
    "euler3d_muscl": ({8: 4096, 16: 1024, 32: 128}, 10_485_760),
    "euler3d_amr2": ({16: 512 + 512}, 1024 * 16 ** 3),
    "wave3d": ({16: 2048}, 2048 * 16 ** 3),
    "srhd3d": ({16: 4096}, 16_777_216),
    "gw59": ({24: 512, 16: 1728 + 4096}, 512 * 24 ** 3 + 5824 * 16 ** 3),
}


@pytest.mark.parametrize("name", sorted(SIZES))
def test_workload_sizes(name):
    w = synth.workload(name)
    mix, nvox = SIZES[name]
    ps, counts = np.unique(w.mesh.patches["p"], return_counts=True)
    assert dict(zip(ps.tolist(), counts.tolist())) == mix
    assert w.mesh.nvox == nvox


def _check_arena(mesh):
    off = mesh.patches["offset"].astype(np.int64)
    n = mesh.patches["p"].astype(np.int64) ** mesh.dim
    assert np.all(off % 16 == 0)
    order = np.argsort(off)
    assert np.all(off[order][1:] >= (off + n)[order][:-1])  # no two patches overlap
    assert mesh.var_stride % 32 == 0 and mesh.var_stride >= int((off + n).max())


def _check_periodic_level(mesh, li):
    """Face neighbours on one periodic level: mutual, and displaced by one patch width."""
    a, b = mesh.level_ranges[li]
    P = mesh.patches
    lev = mesh.levels[li]
    ext = np.array([lev.n[0], lev.n[1], lev.n[2] if mesh.dim == 3 else 1]) * lev.p * lev.dx
    for k in range(a, b):
        for axis in range(mesh.dim):
            for side, sgn in ((0, -1), (1, 1)):
                nb = int(P["nbr"][k][2 * axis + side])
                assert a <= nb < b
                assert int(P["nbr"][nb][2 * axis + 1 - side]) == k
                d = (P["x0"][nb][axis] - P["x0"][k][axis] - sgn * lev.p * lev.dx) % ext[axis]
                assert min(d, ext[axis] - d) < 1e-12
                for other in range(mesh.dim):
                    if other != axis:
                        assert P["x0"][nb][other] == P["x0"][k][other]
    if mesh.dim == 2:
        assert np.all(P["nbr"][a:b, 4:] == -1)


@pytest.mark.parametrize("name", ["euler2d", "euler3d", "wave3d", "gw59"])
def test_periodic_tables(name):
    mesh = synth.workload(name, scale=1 if name == "euler2d" else 4).mesh
    _check_arena(mesh)
    for li in range(len(mesh.levels)):
        _check_periodic_level(mesh, li)


@pytest.mark.parametrize("dim", [2, 3])
def test_coupled_table(dim):
    """Fine patches: half the coarse dx, inside the refined block; a neighbour outside the block is
    the coarse patch that contains the point just across the fine face."""
    nc, p, dxc, lo, m = 4, 4, 1.0 / 16, 1, 2
    mesh = synth.coupled_mesh(nc, p, dxc, lo, m, dim=dim)
    _check_arena(mesh)
    _check_periodic_level(mesh, 0)
    a, b = mesh.level_ranges[1]
    P = mesh.patches
    assert b - a == (2 * m) ** dim
    for k in range(a, b):
        assert P["dx"][k] == dxc / 2 and P["level"][k] == 1
        x0 = P["x0"][k]
        for axis in range(dim):
            assert lo * p * dxc <= x0[axis] < (lo + m) * p * dxc
            for side, sgn in ((0, -1), (1, 1)):
                nb = int(P["nbr"][k][2 * axis + side])
                pt = np.array([x0[i] + 0.5 * p * dxc / 2 for i in range(3)])
                pt[axis] = x0[axis] + (p * dxc / 2 if sgn > 0 else 0.0) + sgn * 0.25 * dxc / 2
                L = nc * p * dxc
                pt[:dim] %= L
                e = p * P["dx"][nb]
                inside = all(P["x0"][nb][i] <= pt[i] < P["x0"][nb][i] + e for i in range(dim))
                assert inside, (k, axis, side, nb)
                if P["level"][nb] == 0:  # a coarse neighbour only across the border of the block
                    c = int(pt[axis] // (p * dxc))
                    assert not (lo <= c < lo + m)


def test_fields_ranges_and_seeds():
    mesh = synth.euler3d_amr_mesh(scale=4)
    a = synth.euler_prims(mesh, 7)
    assert np.array_equal(a, synth.euler_prims(mesh, 7))
    assert not np.array_equal(a, synth.euler_prims(mesh, 8))
    vox = np.zeros(mesh.var_stride, dtype=bool)
    for pt in mesh.patches:
        vox[int(pt["offset"]):int(pt["offset"]) + int(pt["p"]) ** 3] = True
    assert a[0, vox].min() >= 0.5 and a[0, vox].max() <= 1.5
    assert a[4, vox].min() >= 0.5 and a[4, vox].max() <= 1.5
    assert np.abs(a[1:4, vox]).max() <= 0.5
    s = synth.srhd_initial(synth.workload("srhd3d", scale=4).mesh, 3)
    n = 4 ** 3 * 16 ** 3
    rho, v, p = s[0, :n], s[1:4, :n], s[4, :n]
    assert rho.min() >= 0.1 - 1e-12 and rho.max() <= 10 + 1e-12
    assert p.min() >= 0.1 - 1e-12 and p.max() <= 10 + 1e-12
    W = 1 / np.sqrt(1 - (v ** 2).sum(0))
    assert W.min() >= 1.0 and W.max() <= 10.0 + 1e-9
    wm = synth.workload("wave3d", scale=8).mesh
    q, mat = synth.wave_initial(wm, 2)
    c = mat[0, :wm.nvox]  # equal 16^3 patches: the arena holds no padding
    assert c.min() >= 0.5 and c.max() <= 2.0
