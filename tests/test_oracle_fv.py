"""Pins of the FV oracle against facts fixed by the mathematics (CPU only).

Finite-volume Rusanov + non-conservative product scheme (Sec. II-A Eq. 3;
Rusanov and the path-conservative midpoint product are the readings used where
the paper is silent)."""
import math

import numpy as np
import pytest

from helpers import arena, from_grid, single_level, to_grid, voxel_mask
from paper_2608_19273_gb300 import synth

FV = 0


def _adv_mesh(n=(3, 2, 2), p=4, dx=1.0 / 128):
    return single_level(n, p, dx)


@pytest.mark.parametrize("pde", [synth.PDE_ADV_FLUX, synth.PDE_ADV_NCP])
@pytest.mark.parametrize("axis,sign", [(0, 1), (1, 1), (2, 1), (0, -1), (2, -1)])
def test_exact_shift_at_cfl_one(orc, pde, axis, sign):
    """Upwind Rusanov on linear advection with |a| dt/dx = 1 moves data by exactly one voxel."""
    mesh = _adv_mesh()
    rng = np.random.default_rng(1)
    G = synth.dyadic_field(rng, (2 * 4, 2 * 4, 3 * 4))
    q = from_grid(mesh, G, arena(mesh, 1)[0])[None].copy()
    mat = arena(mesh, 3)
    mat[axis, :] = sign * 1.0
    out = np.zeros_like(q)
    dx = 1.0 / 128
    orc.stage(FV, pde, 3, mesh.patches, 1, mesh.var_stride, q, out=out, mat=mat, dt=dx, a=0, b=1, g=1)
    expect = np.roll(G, sign, axis=2 - axis)
    assert np.array_equal(to_grid(mesh, out[0]), expect)


@pytest.mark.parametrize("pde,dim", [(synth.PDE_EULER3D, 3), (synth.PDE_EULER2D, 2),
                                     (synth.PDE_ADV_FLUX, 3), (synth.PDE_ADV_NCP, 3)])
def test_free_stream_bitwise(orc, pde, dim):
    """A constant state is a fixed point of the scheme for any dt (forward Euler stage)."""
    if dim == 3:
        mesh = synth.euler3d_amr_mesh(scale=8)
    else:
        mesh = synth.euler2d_mesh(n=3, p=5)
    nq, nm = synth.PDE_NQ[pde], synth.PDE_NM[pde]
    q = arena(mesh, nq)
    const = [1.3, 0.37, -0.21, 0.11, 2.9][:nq] if pde in (2, 3) else [0.7]
    for v in range(nq):
        q[v, :] = const[v]
    mat = arena(mesh, nm) if nm else None
    if nm:
        mat[:] = np.array([0.3, -0.2, 0.7])[:, None]
    out = np.zeros_like(q)
    orc.stage(FV, pde, dim, mesh.patches, 1, mesh.var_stride, q, out=out, mat=mat, dt=0.123)
    m = voxel_mask(mesh)
    assert np.array_equal(out[:, m], q[:, m])


def test_patch_decomposition_invariance(orc):
    """27 patches of 3^3 tiling a periodic 9^3 box (the p=3, h=1 patches of Fig. 1) give
    bitwise the same update as one self-periodic 9^3 patch: halo gather is exact."""
    many = single_level((3, 3, 3), 3, 1.0 / 9)
    one = single_level((1, 1, 1), 9, 1.0 / 9)
    prim_one = synth.euler_prims(one, 7)
    cons_one = orc.prim2con(synth.PDE_EULER3D, prim_one, one.var_stride)
    cons_many = arena(many, 5)
    for v in range(5):
        from_grid(many, to_grid(one, cons_one[v]), cons_many[v])
    out_one = np.zeros_like(cons_one)
    out_many = np.zeros_like(cons_many)
    lam1 = orc.stage(FV, 3, 3, one.patches, 1, one.var_stride, cons_one, out=out_one, dt=1e-3, want_lam=True)
    lam2 = orc.stage(FV, 3, 3, many.patches, 1, many.var_stride, cons_many, out=out_many, dt=1e-3,
                     want_lam=True)
    for v in range(5):
        assert np.array_equal(to_grid(one, out_one[v]), to_grid(many, out_many[v]))
    assert lam1 == lam2


def _euler_state(orc, mesh, seed, dim=3):
    prim = synth.euler_prims(mesh, seed)
    return orc.prim2con(synth.PDE_EULER3D if dim == 3 else synth.PDE_EULER2D, prim, mesh.var_stride)


@pytest.mark.parametrize("dim", [2, 3])
def test_periodic_conservation(orc, dim):
    """Zero-source flux form on a periodic box: sum of each conserved variable is unchanged."""
    mesh = single_level((3, 2, 2), 6, 1.0 / 32, dim=dim) if dim == 3 else synth.euler2d_mesh(n=3, p=6)
    pde = synth.PDE_EULER3D if dim == 3 else synth.PDE_EULER2D
    q = _euler_state(orc, mesh, 11, dim)
    out = np.zeros_like(q)
    orc.stage(FV, pde, dim, mesh.patches, 1, mesh.var_stride, q, out=out, dt=2e-3)
    for v in range(q.shape[0]):
        assert abs(out[v].sum() - q[v].sum()) <= 1e-13 * np.abs(q[v]).sum()
    assert not np.array_equal(out, q)


def test_mirror_symmetry_x(orc):
    """Reflecting x -> -x (and negating x-momentum) commutes with the update, bitwise."""
    mesh = single_level((2, 2, 2), 5, 1.0 / 10)
    q = _euler_state(orc, mesh, 5)
    qm = np.zeros_like(q)
    for v in range(5):
        G = to_grid(mesh, q[v])[:, :, ::-1]
        from_grid(mesh, -G if v == 1 else G, qm[v])
    out = np.zeros_like(q)
    outm = np.zeros_like(q)
    orc.stage(FV, 3, 3, mesh.patches, 1, mesh.var_stride, q, out=out, dt=1e-3)
    orc.stage(FV, 3, 3, mesh.patches, 1, mesh.var_stride, qm, out=outm, dt=1e-3)
    for v in range(5):
        G = to_grid(mesh, out[v])[:, :, ::-1]
        assert np.array_equal(to_grid(mesh, outm[v]), -G if v == 1 else G)


def test_contact_preserves_velocity_and_pressure(orc):
    """A density wave with constant u, p: Rusanov keeps u and p constant (exact up to rounding)."""
    mesh = single_level((2, 2, 2), 6, 1.0 / 12)
    rng = np.random.default_rng(3)
    prim = arena(mesh, 5)
    X = synth.voxel_centres(mesh)
    prim[0] = synth.fourier_field(rng, X, [1, 1, 1], 3, 1.0, 0.5)
    prim[1], prim[2], prim[3], prim[4] = 0.3, -0.2, 0.1, 0.8
    q = orc.prim2con(3, prim, mesh.var_stride)
    out = np.zeros_like(q)
    orc.stage(FV, 3, 3, mesh.patches, 1, mesh.var_stride, q, out=out, dt=2e-3)
    m = voxel_mask(mesh)
    out, prim = out[:, m], prim[:, m]
    rho = out[0]
    u = out[1:4] / rho
    p = 0.4 * (out[4] - 0.5 * (out[1:4] ** 2).sum(0) / rho)
    assert np.max(np.abs(u - prim[1:4])) < 1e-14
    assert np.max(np.abs(p - 0.8)) < 1e-13
    assert np.max(np.abs(rho - prim[0])) > 1e-4  # density did move


def test_lambda_max_closed_form(orc):
    """lambda_max = |u| + sqrt(gamma p / rho) for a constant Euler state; dt = CFL dx/(d lambda)."""
    mesh = single_level((1, 1, 2), 4, 1.0 / 8)
    prim = arena(mesh, 5)
    prim[0], prim[1], prim[2], prim[3], prim[4] = 2.0, 0.1, -0.45, 0.2, 3.0
    q = orc.prim2con(3, prim, mesh.var_stride)
    lam = orc.max_wave_speed(3, 3, mesh.patches, mesh.var_stride, q)
    assert abs(lam - (0.45 + math.sqrt(1.4 * 3.0 / 2.0))) < 1e-15
    out = np.zeros_like(q)
    lam2 = orc.stage(FV, 3, 3, mesh.patches, 1, mesh.var_stride, q, out=out, dt=0.01, want_lam=True)
    assert lam2 == lam
    assert orc.cfl_dt(0.4, 1.0 / 128, 3, 2.0) == 0.4 / 128 / 6.0


@pytest.mark.parametrize("rk,R", [
    (1, lambda z: 1 + z),
    (3, lambda z: 1 + z + z * z / 2 + z ** 3 / 6),
    (4, lambda z: 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24),
])
def test_rk_amplification_factor(orc, rk, R):
    """On one Fourier mode, upwind advection is diagonal: L e^{ikx} = -(a/dx)(1 - e^{-ik dx}) e^{ikx}.
    One RK step must multiply the mode by the scheme's stability polynomial R(z)."""
    n, p = 4, 4
    mesh = single_level((n, 1, 1), p, 1.0 / 16)
    N = n * p
    dx = 1.0 / 16
    kk = 3
    x = np.arange(N)
    G = np.cos(2 * math.pi * kk * x / N)[None, None, :].repeat(p, 0).repeat(p, 1)
    q = from_grid(mesh, G, arena(mesh, 1)[0])[None].copy()
    mat = arena(mesh, 3)
    mat[0] = 0.75
    dt = 0.6 * dx / 0.75
    orc.rk_steps(FV, synth.PDE_ADV_FLUX, 3, mesh.patches, 1, mesh.var_stride, q, mat=mat, rk=rk, steps=1,
                 dt_fixed=dt)
    th = 2 * math.pi * kk / N
    z = -(0.75 * dt / dx) * (1 - complex(math.cos(th), -math.sin(th)))
    expect = (R(z) * np.exp(1j * th * x)).real
    got = to_grid(mesh, q[0])[0, 0]
    assert np.max(np.abs(got - expect)) < 1e-13


def test_euler2d_runs_and_conserves(orc):
    """The 2D workload: 10 forward-Euler steps at CFL 0.4 conserve mass/momentum/energy."""
    w = synth.workload("euler2d")
    mesh = w.mesh
    q = orc.prim2con(2, synth.euler_prims(mesh, w.seed), mesh.var_stride)
    s0 = q.sum(axis=1)
    dts = orc.rk_steps(FV, 2, 2, mesh.patches, 1, mesh.var_stride, q, rk=1, steps=10, cfl=0.4)
    assert np.all(dts > 0) and np.all(np.isfinite(q))
    assert np.max(np.abs(q.sum(axis=1) - s0) / np.abs(q).sum(axis=1)) < 1e-13


def test_ssprk3_stage_sum_form_is_the_shu_osher_step(orc):
    """The SSP-RK3 step in the Butcher ("stage-sum") form the GPU path evaluates when given acc,
    u1 = q + k0, u2 = q + (k0 + k1)/4, q' = q + (k0 + k1)/6 + 2 k2/3 with k_i = dt L(u_i), built here
    from the oracle's own L, equals the oracle's Shu-Osher step to rounding."""
    mesh = single_level((2, 2, 2), 8, 1.0 / 16)
    q = _euler_state(orc, mesh, 23)
    dt = 2e-3
    ref = q.copy()
    orc.rk_steps(FV, synth.PDE_EULER3D, 3, mesh.patches, 1, mesh.var_stride, ref, rk=3, steps=1, dt_fixed=dt)

    def k(u):  # dt L(u): a stage with a = b = 0, g = 1
        out = np.zeros_like(u)
        orc.stage(FV, synth.PDE_EULER3D, 3, mesh.patches, 1, mesh.var_stride, u, out=out, dt=dt, a=0, b=0, g=1)
        return out
    k0 = k(q)
    u1 = q + k0
    k1 = k(u1)
    u2 = q + (k0 + k1) / 4
    k2 = k(u2)
    got = q + (k0 + k1) / 6 + 2 * k2 / 3
    m = voxel_mask(mesh)
    scale = np.abs(ref[:, m]).max(axis=1, keepdims=True)
    assert np.max(np.abs(got[:, m] - ref[:, m]) / scale) < 1e-14
    assert not np.allclose(ref[:, m], q[:, m])   # the step changed the state


def test_brute_force_on_fig1_sized_patches(orc):
    """K = 3 patches of 3^3 voxels (Fig. 1 sizes, halo 1) in a periodic 9x3x3 box against a
    brute-force evaluation of the same first-order Rusanov stage written directly on the global
    grid (periodic shifts, no patches, no halos): the patch gather and the per-patch update
    change nothing but the summation order."""
    mesh = single_level((3, 1, 1), 3, 1.0 / 9)
    q = _euler_state(orc, mesh, 5)
    dt, dx, gam = 2e-3, 1.0 / 9, 1.4
    out = np.zeros_like(q)
    orc.stage(FV, synth.PDE_EULER3D, 3, mesh.patches, 1, mesh.var_stride, q, out=out, dt=dt)
    Q = np.stack([to_grid(mesh, q[v]) for v in range(5)])  # (5, z, y, x)
    rho, m, E = Q[0], Q[1:4], Q[4]
    u = m / rho
    p = (gam - 1.0) * (E - 0.5 * (m * u).sum(0))
    c = np.sqrt(gam * p / rho)
    L = np.zeros_like(Q)
    for a in range(3):
        ax = 3 - a  # grid axis of direction a in (var, z, y, x)
        F = np.stack([m[a]] + [m[k] * u[a] + (p if k == a else 0.0) for k in range(3)] + [(E + p) * u[a]])
        lam = np.abs(u[a]) + c
        QR, FR, lamR = np.roll(Q, -1, ax), np.roll(F, -1, ax), np.roll(lam, -1, ax - 1)
        Fs = 0.5 * (F + FR) - 0.5 * np.maximum(lam, lamR) * (QR - Q)  # face i + 1/2
        L -= (Fs - np.roll(Fs, 1, ax)) / dx
    ref = Q + dt * L
    got = np.stack([to_grid(mesh, out[v]) for v in range(5)])
    scale = np.abs(ref).max(axis=(1, 2, 3), keepdims=True)
    assert np.max(np.abs(got - ref) / scale) < 1e-14
