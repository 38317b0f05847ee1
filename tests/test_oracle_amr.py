"""Pins of the oracle's coarse-fine coupling (two refinement levels, ratio 2):
piecewise-constant prolongation into fine halos, reflux of the coarse voxels
next to the finer level, restriction of the covered coarse voxels.  The paper's
meshes are Peano spacetrees (Sec. IV); the coupling is the reading documented
with the oracle.  CPU only."""
import numpy as np
import pytest

from paper_2608_19273_gb300 import synth

FV = 0


def _mesh(dim=3, nc=4, p=8, lo=1, m=2):
    return synth.coupled_mesh(nc, p, 1.0 / (nc * p), lo, m, dim=dim)


def _active(mesh, lo=1, m=2):
    """Mask of voxels that represent the solution: fine voxels and coarse voxels outside the block."""
    act = np.zeros(mesh.var_stride, dtype=bool)
    vol = np.zeros(mesh.var_stride)
    for pt in mesh.patches:
        p, o = int(pt["p"]), int(pt["offset"])
        n = p ** mesh.dim
        if pt["level"] == 0:
            lat = [int(round(pt["x0"][a] / (p * pt["dx"]))) for a in range(mesh.dim)]
            if all(lo <= c < lo + m for c in lat):
                continue
        act[o:o + n] = True
        vol[o:o + n] = float(pt["dx"]) ** mesh.dim
    return act, vol


def _cons(orc, mesh, seed):
    rng = np.random.default_rng(seed)
    specs = [(1.0, 0.5)] + [(0.0, 0.5)] * mesh.dim + [(1.0, 0.5)]
    prim = synth.coupled_fields(mesh, rng, specs)
    pde = synth.PDE_EULER3D if mesh.dim == 3 else synth.PDE_EULER2D
    return pde, orc.prim2con(pde, prim, mesh.var_stride)


@pytest.mark.parametrize("dim", [3, 2])
def test_free_stream_bitwise(orc, dim):
    """A constant state stays bitwise constant on both levels: prolongation copies it, the fine face
    fluxes equal the coarse one (reflux adds exactly zero), restriction averages equal values."""
    mesh = _mesh(dim)
    pde = synth.PDE_EULER3D if dim == 3 else synth.PDE_EULER2D
    nq = synth.PDE_NQ[pde]
    q = np.zeros((nq, mesh.var_stride))
    for v, c in enumerate([1.3, 0.37, -0.21, 0.11, 2.9][:nq] if dim == 3 else [1.3, 0.37, -0.21, 2.9]):
        q[v, :] = c
    ref = q.copy()
    # forward-Euler steps (the SSP-RK3 combination 3/4 q0 + 1/4 u is not exact in floating point)
    orc.rk_steps(FV, pde, dim, mesh.patches, 1, mesh.var_stride, q, rk=1, steps=2, cfl=0.4)
    m = np.zeros(mesh.var_stride, dtype=bool)
    for pt in mesh.patches:
        m[int(pt["offset"]):int(pt["offset"]) + int(pt["p"]) ** dim] = True
    assert np.array_equal(q[:, m], ref[:, m])


@pytest.mark.parametrize("dim", [3, 2])
def test_conservation_across_levels(orc, dim):
    """Volume-weighted totals over the active voxels are conserved (reflux makes the coarse face
    flux equal to the mean of the fine face fluxes)."""
    mesh = _mesh(dim)
    pde, q = _cons(orc, mesh, 71 + dim)
    act, vol = _active(mesh)
    before = (q[:, act] * vol[act]).sum(axis=1)
    scale = (np.abs(q[:, act]) * vol[act]).sum(axis=1)
    orc.rk_steps(FV, pde, dim, mesh.patches, 1, mesh.var_stride, q, rk=3, steps=2, cfl=0.4)
    after = (q[:, act] * vol[act]).sum(axis=1)
    assert np.all(np.abs(after - before) <= 1e-13 * scale), (after - before) / scale


def _linear_advection_L(orc, dim, alpha=0.5):
    """L(q) (out with a = b = 0, g = dt = 1) for ADV_FLUX, a = (1, 0, 0), q = alpha x."""
    mesh = _mesh(dim)
    X = synth.voxel_centres_any(mesh)
    q = (alpha * X[0])[None].copy()
    mat = np.zeros((3, mesh.var_stride))
    mat[0, :] = 1.0
    out = np.zeros_like(q)
    if dim == 2:
        pytest.skip("ADV_FLUX is a 3D system")
    orc.stage(FV, synth.PDE_ADV_FLUX, dim, mesh.patches, 1, mesh.var_stride, q, out=out, mat=mat, dt=1.0, a=0,
              b=0, g=1)
    return mesh, X, out[0]


def test_prolongation_and_reflux_on_a_linear_profile(orc):
    """Upwind flux a q with q = alpha x: away from the level border L = -alpha exactly.  The first fine
    voxels of the refined block see a halo that is the containing coarse voxel's value (centre one and
    a half fine spacings upwind): L = -1.5 alpha.  The coarse voxel right after the block takes the mean
    of the fine fluxes on its face (the fine voxels' values, centre a half fine spacing upwind of the
    face) instead of the covered coarse voxel's value: L = -0.75 alpha.  The coarse voxel before the
    block is unchanged by reflux (the fine fluxes there carry its own value): L = -alpha."""
    alpha = 0.5
    mesh, X, L = _linear_advection_L(orc, 3, alpha)
    nc, p, dxc = 4, 8, 1.0 / 32
    dxf = dxc / 2
    lo_x, hi_x = 1 * p * dxc, 3 * p * dxc  # block [0.25, 0.75) along every axis
    yz_in = (X[1] > lo_x) & (X[1] < hi_x) & (X[2] > lo_x) & (X[2] < hi_x)
    fine = np.zeros(mesh.var_stride, dtype=bool)
    coarse_active = np.zeros(mesh.var_stride, dtype=bool)
    act, _ = _active(mesh)
    for pt in mesh.patches:
        o, n = int(pt["offset"]), int(pt["p"]) ** 3
        (fine if pt["level"] == 1 else coarse_active)[o:o + n] = True
    coarse_active &= act
    x = X[0]
    first_fine = fine & np.isclose(x, lo_x + dxf / 2)
    after_block = coarse_active & yz_in & np.isclose(x, hi_x + dxc / 2)
    before_block = coarse_active & yz_in & np.isclose(x, lo_x - dxc / 2)
    away = (coarse_active & (x > 2 * dxc) & (x < 1 - 2 * dxc) & ~after_block) | (fine & ~first_fine)
    assert first_fine.sum() == 32 * 32 and after_block.sum() == 16 * 16 and before_block.sum() == 16 * 16
    assert np.all(L[first_fine] == -1.5 * alpha)
    assert np.all(L[after_block] == -0.75 * alpha)
    assert np.all(L[before_block] == -alpha)
    assert np.all(L[away] == -alpha)


@pytest.mark.parametrize("dim", [3, 2])
def test_restriction_is_the_mean_of_the_fine_voxels(orc, dim):
    mesh = _mesh(dim)
    pde, q = _cons(orc, mesh, 81 + dim)
    out = np.zeros_like(q)
    orc.stage(FV, pde, dim, mesh.patches, 1, mesh.var_stride, q, out=out, dt=1e-3)
    p = 8
    first_fine = mesh.level_ranges[1][0]
    for pt in mesh.patches[first_fine:]:
        lat = [int(round(pt["x0"][a] / (p * pt["dx"]))) for a in range(dim)]
        par_lat = [c // 2 for c in lat]
        oc = [c % 2 for c in lat]
        par = ((par_lat[2] if dim == 3 else 0) * 4 + par_lat[1]) * 4 + par_lat[0]
        pc = mesh.patches[par]
        for v in range(q.shape[0]):
            f = out[v, int(pt["offset"]):int(pt["offset"]) + p ** dim].reshape((p,) * dim)
            c = out[v, int(pc["offset"]):int(pc["offset"]) + p ** dim].reshape((p,) * dim)
            if dim == 3:
                mean = f.reshape(4, 2, 4, 2, 4, 2).mean(axis=(1, 3, 5))
                sub = c[oc[2] * 4:oc[2] * 4 + 4, oc[1] * 4:oc[1] * 4 + 4, oc[0] * 4:oc[0] * 4 + 4]
            else:
                mean = f.reshape(4, 2, 4, 2).mean(axis=(1, 3))
                sub = c[oc[1] * 4:oc[1] * 4 + 4, oc[0] * 4:oc[0] * 4 + 4]
            assert np.allclose(sub, mean, rtol=1e-15, atol=1e-15 * np.abs(mean).max())
