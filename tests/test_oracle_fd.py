"""Pins of the FD4 + Kreiss-Oliger oracle (CPU only).

4th-order centred differences and 6th-difference KO dissipation (Sec. I,
Sec. IV: FD4 with KO; the KO normalisation sigma/(64 dx) delta^6 is the
reading used since the paper only cites it)."""
import math

import numpy as np
import pytest

from helpers import arena, from_grid, single_level, to_grid, voxel_mask
from paper_2608_19273_gb300 import synth

FD = 1
WAVE, GW = synth.PDE_WAVE3D, synth.PDE_GW59


def _wave_state(mesh, k, c=1.0):
    X = synth.voxel_centres(mesh)
    ph = 2 * math.pi * (k[0] * X[0] + k[1] * X[1] + k[2] * X[2])
    q = arena(mesh, 5)
    q[0] = np.sin(ph)
    q[1] = np.cos(ph)
    for i in range(3):
        q[2 + i] = 2 * math.pi * k[i] * np.cos(ph)
    mat = arena(mesh, 1)
    mat[0] = c
    return q, mat, ph


def _operator(orc, pde, mesh, q, mat=None, sigma=0.1, params=None):
    """L(q) exactly: out = 0 * q + 1 * 1 * L(q)."""
    L = np.zeros_like(q)
    orc.stage(FD, pde, 3, mesh.patches, 3, mesh.var_stride, q, out=L, mat=mat, dt=1.0, a=0, b=0, g=1,
              sigma=sigma, params=params)
    return L


def test_fd4_operator_fourth_order(orc):
    """Wave system with constant c on sin(k.x): ||L_h(Q) - L(Q)|| falls like dx^4."""
    k = (1, 2, 1)
    c, gam = 1.3, 0.1
    errs = []
    for n in (2, 4):
        mesh = single_level((n, n, n), 8, 1.0 / (8 * n))
        q, mat, ph = _wave_state(mesh, k, c)
        L = _operator(orc, WAVE, mesh, q, mat, params=[gam])
        k2 = 4 * math.pi ** 2 * sum(x * x for x in k)
        exact = np.zeros_like(q)
        exact[0] = q[1]
        exact[1] = -c * c * k2 * np.sin(ph) - gam * np.cos(ph)
        for i in range(3):
            exact[2 + i] = -2 * math.pi * k[i] * np.sin(ph)
        m = voxel_mask(mesh)
        errs.append(np.max(np.abs(L[:, m] - exact[:, m])))
    order = math.log2(errs[0] / errs[1])
    assert 3.8 < order < 4.3, (errs, order)


def test_ko_on_checkerboard_exact(orc):
    """KO alone (zero-velocity advection: B = 0) on (-1)^(i+j+k) gives exactly -3 sigma/dx Q."""
    mesh = single_level((2, 2, 2), 8, 1.0 / 16)
    z, y, x = np.meshgrid(np.arange(16), np.arange(16), np.arange(16), indexing="ij")
    G = ((-1.0) ** (x + y + z))
    q = from_grid(mesh, G, arena(mesh, 1)[0])[None].copy()
    mat = arena(mesh, 3)
    L = _operator(orc, synth.PDE_ADV_NCP, mesh, q, mat, sigma=0.1)
    assert np.array_equal(to_grid(mesh, L[0]), -3 * 0.1 * 16 * G)


@pytest.mark.parametrize("pde", [WAVE, GW])
def test_free_stream_bitwise(orc, pde):
    mesh = single_level((2, 1, 2), 8, 1.0 / 16)
    nq = synth.PDE_NQ[pde]
    q = arena(mesh, nq)
    if pde == WAVE:
        q[0] = 0.7
        mat = arena(mesh, 1)
        mat[0] = 1.25 + 0.75 * np.sin(2 * math.pi * synth.voxel_centres(mesh)[0])
        params = [0.1]
    else:
        q[55] = 1.0
        mat = None
        params = synth.workload("gw59", scale=8).params
    out = np.zeros_like(q)
    orc.stage(FD, pde, 3, mesh.patches, 3, mesh.var_stride, q, out=out, mat=mat, dt=0.3, params=params)
    m = voxel_mask(mesh)
    assert np.array_equal(out[:, m], q[:, m])


def _telegraph(X, t, k, c, gam):
    ph = 2 * math.pi * (k[0] * X[0] + k[1] * X[1] + k[2] * X[2])
    kk = [2 * math.pi * ki for ki in k]
    k2 = sum(x * x for x in kk)
    w = math.sqrt(c * c * k2 - gam * gam / 4)
    e = math.exp(-gam * t / 2)
    T = math.cos(w * t) + gam / (2 * w) * math.sin(w * t)
    q = np.zeros((5, X.shape[1]))
    q[0] = e * T * np.sin(ph)
    q[1] = -e * (c * c * k2 / w) * math.sin(w * t) * np.sin(ph)
    for i in range(3):
        q[2 + i] = e * T * kk[i] * np.cos(ph)
    return q


def test_rk4_telegraph_plane_wave_convergence(orc):
    """Full RK4 + FD4 + KO run of the damped wave against the exact telegraph solution: 4th order."""
    k, c, gam, T = (1, 1, 1), 1.0, 0.1, 0.05
    errs = []
    for n in (2, 4):
        mesh = single_level((n, n, n), 8, 1.0 / (8 * n))
        X = synth.voxel_centres(mesh)
        q = _telegraph(X, 0.0, k, c, gam)
        mat = arena(mesh, 1)
        mat[0] = c
        dx = 1.0 / (8 * n)
        nsteps = int(math.ceil(T / (0.25 * dx / 3)))
        orc.rk_steps(FD, WAVE, 3, mesh.patches, 3, mesh.var_stride, q, mat=mat, rk=4, steps=nsteps,
                     dt_fixed=T / nsteps, sigma=0.1, params=[gam])
        ex = _telegraph(X, T, k, c, gam)
        m = voxel_mask(mesh)
        errs.append(np.max(np.abs(q[:, m] - ex[:, m])))
    order = math.log2(errs[0] / errs[1])
    assert 3.7 < order < 4.4, (errs, order)


def test_gw59_linear_limit_is_unit_wave(orc):
    """Around the flat state (alpha = 1, beta = 0) each GW59 field triple (phi_a, Pi_a, psi_a) obeys the
    undamped unit-speed wave system up to O(amplitude^2)."""
    mesh = single_level((2, 2, 2), 8, 1.0 / 16)
    amp = 1e-6
    qw, _, _ = _wave_state(mesh, (1, 0, 2))
    qw *= amp
    params = synth.workload("gw59", scale=8).params
    for a in (0, 4, 10):
        q = arena(mesh, 59)
        q[55] = 1.0
        q[5 * a:5 * a + 5] = qw
        Lg = _operator(orc, GW, mesh, q, params=params)
        mat = arena(mesh, 1)
        mat[0] = 1.0
        Lw = _operator(orc, WAVE, mesh, qw, mat, params=[0.0])
        m = voxel_mask(mesh)
        scale = np.max(np.abs(Lw[:, m]))
        assert np.max(np.abs(Lg[5 * a:5 * a + 5][:, m] - Lw[:, m])) <= 1e-8 * scale
        others = np.delete(Lg[:, m], np.s_[5 * a:5 * a + 5], axis=0)
        assert np.max(np.abs(others)) <= 1e-6 * scale  # alpha, beta and other fields move at O(amp^2)


@pytest.mark.parametrize("pde", [WAVE, GW])
def test_mirror_symmetry_x(orc, pde):
    """x -> -x with the x-components (psi_x, beta^x) negated commutes with the FD operator, bitwise."""
    mesh = single_level((2, 2, 2), 8, 1.0 / 16)
    rng = np.random.default_rng(9)
    nq = synth.PDE_NQ[pde]
    X = synth.voxel_centres(mesh)
    q = arena(mesh, nq)
    for v in range(nq):
        q[v] = synth.fourier_field(rng, X, [1, 1, 1], 3, 0.0, 0.3)
    odd = {2} if pde == WAVE else {5 * a + 2 for a in range(11)} | {56}
    if pde == GW:
        q[55] += 1.0
    mat, params = None, synth.workload("gw59", scale=8).params
    if pde == WAVE:
        mat = arena(mesh, 1)
        mat[0] = 1.0 + 0.2 * np.cos(2 * math.pi * X[1])  # even in x
        params = [0.1]
    qm = np.zeros_like(q)
    for v in range(nq):
        G = to_grid(mesh, q[v])[:, :, ::-1]
        from_grid(mesh, -G if v in odd else G, qm[v])
    matm = None
    if mat is not None:
        matm = np.zeros_like(mat)
        from_grid(mesh, to_grid(mesh, mat[0])[:, :, ::-1], matm[0])
    L = _operator(orc, pde, mesh, q, mat, params=params)
    Lm = _operator(orc, pde, mesh, qm, matm, params=params)
    for v in range(nq):
        G = to_grid(mesh, L[v])[:, :, ::-1]
        assert np.array_equal(to_grid(mesh, Lm[v]), -G if v in odd else G), v


def _interior(mesh, h=3):
    """Voxels of a single self-periodic patch whose h-wide stencils do not wrap around."""
    p = int(mesh.patches[0]["p"])
    z, y, x = np.meshgrid(np.arange(p), np.arange(p), np.arange(p), indexing="ij")
    return ((x >= h) & (x < p - h) & (y >= h) & (y < p - h) & (z >= h) & (z < p - h)).ravel()


def test_fd4_exact_on_quartics(orc):
    """The centred 4th-order derivative is exact on polynomials of degree <= 4 and the 6th
    difference of the KO term vanishes on them, so on quartic data (away from the periodic
    seam) the wave operator equals its continuous value to rounding: L(phi) = Pi,
    L(Pi) = c^2 div psi - gamma Pi, L(psi_d) = d_d Pi."""
    mesh = single_level((1, 1, 1), 16, 1.0 / 16)
    X = synth.voxel_centres(mesh)
    x, y, z = X[0], X[1], X[2]
    q = arena(mesh, 5)
    q[0] = 0.3 * x ** 4 - 0.2 * x * y ** 3 + 0.5 * z * z * x - 0.1
    q[1] = 0.7 * y ** 4 + 0.4 * x * z - 0.3 * x * x * y + 0.25 * z ** 4
    q[2] = 0.2 * z ** 4 - x ** 3 * y + 0.6 * x ** 4
    q[3] = -0.5 * y ** 3 * z + 0.8 * y ** 4
    q[4] = 0.9 * x * y * z * z - 0.4 * z ** 4
    c, gam = 1.3, 0.1
    mat = arena(mesh, 1)
    mat[0] = c
    L = _operator(orc, WAVE, mesh, q, mat, sigma=0.1, params=[gam])
    dPi = [0.4 * z - 0.6 * x * y, 2.8 * y ** 3 - 0.3 * x * x, 0.4 * x + z ** 3]
    div_psi = (-3 * x * x * y + 2.4 * x ** 3) + (-1.5 * y * y * z + 3.2 * y ** 3) + (1.8 * x * y * z - 1.6 * z ** 3)
    exact = np.stack([q[1], c * c * div_psi - gam * q[1], dPi[0], dPi[1], dPi[2]])
    m = _interior(mesh)
    n = 16 ** 3
    err = np.abs(L[:, :n][:, m] - exact[:, :n][:, m])
    assert np.max(err) <= 1e-12 * np.max(np.abs(exact[:, :n][:, m])), np.max(err)


def test_ko_stencil_on_monomials(orc):
    """KO alone (zero-velocity advection: B = 0): sigma/(64 dx) delta^6 vanishes on x^k for
    k <= 5 and gives sigma/(64 dx) 720 dx^6 on x^6 (the 6th difference of x^6 is 6! dx^6);
    together with the checkerboard this fixes all seven stencil weights."""
    dx, sigma = 1.0 / 16, 0.1
    mesh = single_level((1, 1, 1), 16, dx)
    X = synth.voxel_centres(mesh)
    mat = arena(mesh, 3)
    m = _interior(mesh)
    n = 16 ** 3
    for k in range(7):
        for axis in range(3):
            q = arena(mesh, 1)
            q[0] = (X[axis] - 0.5) ** k
            L = _operator(orc, synth.PDE_ADV_NCP, mesh, q, mat, sigma=sigma)[0, :n][m]
            expect = sigma / (64 * dx) * 720 * dx ** 6 if k == 6 else 0.0
            assert np.max(np.abs(L - expect)) <= 1e-13, (k, axis, np.max(np.abs(L - expect)))


def test_gw59_operator_on_quadratic_fields(orc):
    """Every GW59 field a quadratic polynomial in x, y, z (lapse near 1): the FD4 derivatives are
    exact and the KO term vanishes, so away from the periodic seam the discrete operator equals the
    system's right-hand side evaluated with the exact gradients, nonlinear products included:
      dphi_a = alpha Pi_a + beta^k psi_ak,
      dPi_a = alpha d_k psi_ak + beta^k d_k Pi_a + alpha sum_b C_ab phi_b Pi_b,
      dpsi_ai = alpha d_i Pi_a + Pi_a d_i alpha + beta^k d_k psi_ai,
      dalpha = -kappa alpha^2 sum_a Pi_a^2,  dbeta^i = 3/4 sum_a psi_ai Pi_a."""
    mesh = single_level((1, 1, 1), 16, 1.0 / 16)
    X = synth.voxel_centres(mesh)[:, :16 ** 3] - 0.5
    rng = np.random.default_rng(59)
    # f = c0 + c . x + x^T A x (A symmetric), gradient c + 2 A x
    c0 = rng.uniform(-0.2, 0.2, 59)
    c1 = rng.uniform(-0.3, 0.3, (59, 3))
    A = rng.uniform(-0.3, 0.3, (59, 3, 3))
    A = 0.5 * (A + A.transpose(0, 2, 1))
    c0[55] = 1.0
    val = c0[:, None] + c1 @ X + np.einsum("vij,in,jn->vn", A, X, X)
    grad = c1[:, :, None] + 2.0 * np.einsum("vij,jn->vin", A, X)  # (59, 3, n)
    q = arena(mesh, 59)
    q[:, :16 ** 3] = val
    params = synth.workload("gw59", scale=8).params
    kappa, C = params[0], params[1:].reshape(11, 11)
    L = _operator(orc, GW, mesh, q, sigma=0.1, params=params)[:, :16 ** 3]
    al, be = val[55], val[56:59]
    phi, Pi, psi = val[0:55:5], val[1:55:5], np.stack([val[2 + i:55:5] for i in range(3)], 1)  # psi (11, 3, n)
    dPi = np.stack([grad[1 + 5 * a] for a in range(11)])                                    # (11, 3, n)
    dpsi = np.stack([np.stack([grad[2 + i + 5 * a] for i in range(3)]) for a in range(11)])  # (11, i, k, n)
    ref = np.zeros_like(val)
    for a in range(11):
        o = 5 * a
        ref[o] = al * Pi[a] + (be * psi[a]).sum(0)
        ref[o + 1] = (al * np.einsum("kkn->n", dpsi[a]) + (be * dPi[a]).sum(0)
                      + al * (C[a][:, None] * phi * Pi).sum(0))
        for i in range(3):
            ref[o + 2 + i] = al * dPi[a][i] + Pi[a] * grad[55][i] + (be * dpsi[a][i]).sum(0)
    ref[55] = -kappa * al * al * (Pi * Pi).sum(0)
    ref[56:59] = 0.75 * (psi * Pi[:, None, :]).sum(0)
    m = _interior(mesh)
    err = np.abs(L[:, m] - ref[:, m]).max()
    assert err <= 1e-12 * np.abs(ref[:, m]).max(), err
