"""Pins of the oracle's second-order FV stage (MUSCL reconstruction with the
minmod limiter feeding the Rusanov flux; the reading of the face-state
stencil of Sec. II-A Eq. 3) against
facts fixed by the mathematics.  CPU only."""
import numpy as np
import pytest

from helpers import arena, from_grid, single_level, to_grid, voxel_mask
from paper_2608_19273_gb300 import synth

FV, FV2 = 0, 2


def test_free_stream_bitwise(orc):
    """A constant Euler state on the AMR-like mix is a fixed point (slopes are exactly zero)."""
    mesh = synth.euler3d_amr_mesh(scale=8)
    q = arena(mesh, 5)
    for v, c in enumerate([1.3, 0.37, -0.21, 0.11, 2.9]):
        q[v, :] = c
    out = np.zeros_like(q)
    orc.stage(FV2, 3, 3, mesh.patches, 2, mesh.var_stride, q, out=out, dt=0.123)
    m = voxel_mask(mesh)
    assert np.array_equal(out[:, m], q[:, m])


def _adv_1d(orc, G, dx, a=1.0, scheme=FV2, dt=0.0):
    """L(q) (dt = 0: via out = q + 1 * L with g = 1/ (dt-free form)) for ADV_FLUX on a 16x8x8 box."""
    mesh = single_level((2, 1, 1), 8, dx)
    q = from_grid(mesh, G, arena(mesh, 1)[0])[None].copy()
    mat = arena(mesh, 3)
    mat[0, :] = a
    out = np.zeros_like(q)
    orc.stage(scheme, synth.PDE_ADV_FLUX, 3, mesh.patches, 2, mesh.var_stride, q, out=out, mat=mat, dt=1.0,
              a=0, b=0, g=1)       # out = dt L with dt = 1
    return to_grid(mesh, out[0])


@pytest.mark.parametrize("a", [1.0, -1.0])
def test_quadratic_profile_exact(orc, a):
    """On q = x^2 (monotone and convex away from the periodic wrap) minmod picks the upwind
    one-sided slope, and MUSCL + upwind Rusanov reproduces dq/dx = 2x exactly: L = -a 2x.
    First-order upwind is off by a dx there (checked as a contrast)."""
    dx = 1.0 / 16
    x = (np.arange(16) + 0.5) * dx
    G = np.broadcast_to((x * x)[None, None, :], (8, 8, 16)).copy()
    L = _adv_1d(orc, G, dx, a)
    L1 = _adv_1d(orc, G, dx, a, scheme=FV)
    for i in range(3, 13):
        assert np.all(L[:, :, i] == -a * 2 * x[i]), i
        assert np.all(L1[:, :, i] != -a * 2 * x[i])


def test_linear_profile_exact(orc):
    """On a linear profile both one-sided differences are equal; the reconstruction is exact."""
    dx = 1.0 / 16
    x = (np.arange(16) + 0.5) * dx
    G = np.broadcast_to((3.0 * x)[None, None, :], (8, 8, 16)).copy()
    L = _adv_1d(orc, G, dx, 1.0)
    for i in range(3, 14):
        assert np.all(L[:, :, i] == -3.0)


def _advect_sine(orc, n, steps_per_unit, t_end):
    """ADV_FLUX with a = (1, 0, 0) on a periodic box of n x 8 x 8 voxels (patches of 8),
    SSP-RK3 at fixed dt; returns the L1 error against the exact translate."""
    dx = 1.0 / n
    mesh = single_level((n // 8, 1, 1), 8, dx)
    x = (np.arange(n) + 0.5) * dx
    G = np.broadcast_to(np.sin(2 * np.pi * x)[None, None, :], (8, 8, n)).copy()
    q = from_grid(mesh, G, arena(mesh, 1)[0])[None].copy()
    mat = arena(mesh, 3)
    mat[0, :] = 1.0
    steps = int(round(t_end * steps_per_unit * n))
    dt = t_end / steps
    orc.rk_steps(FV2, synth.PDE_ADV_FLUX, 3, mesh.patches, 2, mesh.var_stride, q, mat=mat, rk=3, steps=steps,
                 dt_fixed=dt)
    exact = np.sin(2 * np.pi * (x - t_end))
    got = to_grid(mesh, q[0])[4, 4, :]
    return np.mean(np.abs(got - exact))


def test_second_order_convergence(orc):
    """L1 error of a translated sine wave falls by about 4x per halving of dx (minmod clips the
    extrema, so the observed L1 order is a little below 2); first order would give about 2x."""
    errs = [_advect_sine(orc, n, 2.5, 0.25) for n in (32, 64, 128)]
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 1.6, orders


def test_total_variation_diminishing(orc):
    """Scalar advection of a square wave with minmod MUSCL and SSP-RK3 at CFL 0.4 never
    increases the total variation (no new extrema)."""
    n, dx = 32, 1.0 / 32
    mesh = single_level((4, 1, 1), 8, dx)
    G = np.zeros((8, 8, n))
    G[:, :, 8:20] = 1.0
    q = from_grid(mesh, G, arena(mesh, 1)[0])[None].copy()
    mat = arena(mesh, 3)
    mat[0, :] = 1.0
    tv = [np.sum(np.abs(np.diff(np.r_[G[4, 4], G[4, 4, :1]])))]
    for _ in range(20):
        orc.rk_steps(FV2, synth.PDE_ADV_FLUX, 3, mesh.patches, 2, mesh.var_stride, q, mat=mat, rk=3, steps=1,
                     dt_fixed=0.4 * dx)
        line = to_grid(mesh, q[0])[4, 4]
        tv.append(np.sum(np.abs(np.diff(np.r_[line, line[:1]]))))
        assert line.max() <= 1.0 + 1e-14 and line.min() >= -1e-14
    assert all(tv[i + 1] <= tv[i] + 1e-12 for i in range(len(tv) - 1)), tv


def test_periodic_conservation(orc):
    mesh = synth.euler3d_amr_mesh(scale=4)
    q = orc.prim2con(3, synth.euler_prims(mesh, 51), mesh.var_stride)
    m = voxel_mask(mesh)
    before = q[:, m].sum(axis=1)
    scale = np.abs(q[:, m]).sum(axis=1)
    orc.rk_steps(FV2, 3, 3, mesh.patches, 2, mesh.var_stride, q, rk=3, steps=1, cfl=0.4)
    after = q[:, m].sum(axis=1)
    assert np.all(np.abs(after - before) <= 1e-13 * scale)


def test_mirror_symmetry_bitwise(orc):
    """x -> -x with the x momentum negated commutes with the stage."""
    mesh = single_level((2, 2, 2), 8, 1.0 / 16)
    q = orc.prim2con(3, synth.euler_prims(mesh, 52), mesh.var_stride)
    grids = [to_grid(mesh, q[v]) for v in range(5)]
    qm = arena(mesh, 5)
    for v in range(5):
        g = grids[v][:, :, ::-1] * (-1.0 if v == 1 else 1.0)
        from_grid(mesh, g, qm[v])
    out, outm = np.zeros_like(q), np.zeros_like(qm)
    orc.stage(FV2, 3, 3, mesh.patches, 2, mesh.var_stride, q, out=out, dt=1e-3)
    orc.stage(FV2, 3, 3, mesh.patches, 2, mesh.var_stride, qm, out=outm, dt=1e-3)
    for v in range(5):
        a = to_grid(mesh, out[v])[:, :, ::-1] * (-1.0 if v == 1 else 1.0)
        assert np.array_equal(a, to_grid(mesh, outm[v])), v


def test_patch_decomposition_invariance(orc):
    """27 patches of 4^3 tiling a periodic 12^3 box update bitwise like one 12^3 patch (halo 2)."""
    many = single_level((3, 3, 3), 4, 1.0 / 12)
    one = single_level((1, 1, 1), 12, 1.0 / 12)
    cons_one = orc.prim2con(3, synth.euler_prims(one, 53), one.var_stride)
    cons_many = arena(many, 5)
    for v in range(5):
        from_grid(many, to_grid(one, cons_one[v]), cons_many[v])
    o1, o2 = np.zeros_like(cons_one), np.zeros_like(cons_many)
    orc.stage(FV2, 3, 3, one.patches, 2, one.var_stride, cons_one, out=o1, dt=1e-3)
    orc.stage(FV2, 3, 3, many.patches, 2, many.var_stride, cons_many, out=o2, dt=1e-3)
    for v in range(5):
        assert np.array_equal(to_grid(one, o1[v]), to_grid(many, o2[v]))
