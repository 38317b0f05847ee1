"""Pins of the FV oracle against hand-worked examples (CPU only).

Each fixture under ``golden/`` is a two-state Riemann problem on a periodic
row of 16 voxels, worked out by hand in exact rational arithmetic: the
physical fluxes, the Rusanov face fluxes (Sec. II-A, Eq. 3 with the Rusanov
reading) and the four voxels next to the two faces after one forward-Euler
stage.  The oracle runs the same stage along every axis of a 2D or 3D
patch row and must reproduce those values to rounding, while every other
voxel stays bitwise unchanged.  A dropped flux term (the p u of the energy
flux, the p of the normal momentum flux), a wrong dissipation speed, a wrong
sign or a transposed velocity component moves at least one listed value.

Every stored number traces back to the primitive states: the tests first check,
in exact rational arithmetic, that each fixture line follows from the lines
before it (conserved states and fluxes from the primitives, face fluxes from
those, voxel values from the update rule)."""
import os
from fractions import Fraction

import numpy as np
import pytest

from helpers import arena, from_grid, single_level, to_grid

FV = 0
EULER2D, EULER3D, SRHD3D = 2, 3, 5
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    """Fixture -> {section: {key: [Fraction, ...]}}; section "" holds the global keys."""
    out, sec = {"": {}}, ""
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("[") and line.endswith("]"):
                sec = line[1:-1]
                out[sec] = {}
                continue
            key, val = (t.strip() for t in line.split("=", 1))
            out[sec][key] = [Fraction(t) for t in val.split()]
    return out


def _rusanov_lines_agree(g):
    """The fixture's Rusanov lines follow from its F, Q and s lines (exact)."""
    s = g["speed_max"][0]
    for a, b, ql, qr, lr, rl in zip(g["F_L"], g["F_R"], g["Q_L"], g["Q_R"], g["Fstar_LR"], g["Fstar_RL"]):
        assert (a + b) / 2 - s / 2 * (qr - ql) == lr
        assert (a + b) / 2 - s / 2 * (ql - qr) == rl


def _euler_lines_agree(g, gamma, dim):
    """The fixture's conserved and flux lines follow from its primitive lines (exact):
    E = p/(gamma-1) + rho |u|^2/2, F_n = (rho u_n, rho u u_n + p e_n, (E + p) u_n)."""
    for side in ("L", "R"):
        rho, u, p = g[f"prim_{side}"][0], g[f"prim_{side}"][1:1 + dim], g[f"prim_{side}"][1 + dim]
        E = p / (gamma - 1) + rho * sum(x * x for x in u) / 2
        assert g[f"Q_{side}"] == [rho] + [rho * x for x in u] + [E]
        F = [rho * u[0]] + [rho * x * u[0] for x in u] + [(E + p) * u[0]]
        F[1] += p
        assert g[f"F_{side}"] == F


def _exact_sqrt(x):
    import math
    a, b = math.isqrt(x.numerator), math.isqrt(x.denominator)
    assert a * a == x.numerator and b * b == x.denominator, x
    return Fraction(a, b)


def _srhd_lines_agree(g, Gamma):
    """The same for SRHD: W = 1/sqrt(1 - v^2), h = 1 + Gamma p/((Gamma - 1) rho), D = rho W,
    S = rho h W^2 v, tau = rho h W^2 - p - D, F_n = (D v_n, S v_n + p e_n, S_n - D v_n)."""
    for side in ("L", "R"):
        rho, v, p = g[f"prim_{side}"][0], g[f"prim_{side}"][1:4], g[f"prim_{side}"][4]
        W = 1 / _exact_sqrt(1 - sum(x * x for x in v))
        h = 1 + Gamma * p / ((Gamma - 1) * rho)
        D, S = rho * W, [rho * h * W * W * x for x in v]
        assert g[f"Q_{side}"] == [D] + S + [rho * h * W * W - p - D]
        F = [D * v[0]] + [x * v[0] for x in S] + [S[0] - D * v[0]]
        F[1] += p
        assert g[f"F_{side}"] == F


def _update_lines_agree(g, r):
    QL, QR, FL, FR, LR, RL = (g[k] for k in ("Q_L", "Q_R", "F_L", "F_R", "Fstar_LR", "Fstar_RL"))
    for v in range(len(QL)):
        assert g["voxel_7"][v] == QL[v] - r * (LR[v] - FL[v])
        assert g["voxel_8"][v] == QR[v] - r * (FR[v] - LR[v])
        assert g["voxel_15"][v] == QR[v] - r * (RL[v] - FR[v])
        assert g["voxel_0"][v] == QL[v] - r * (FL[v] - RL[v])


def _to_axes(vec_nt, axis, dim):
    """(normal, t1[, t2]) components -> physical axes (tangential axes in increasing order)."""
    out = [None] * dim
    out[axis] = vec_nt[0]
    others = [a for a in range(dim) if a != axis]
    for j, a in enumerate(others):
        out[a] = vec_nt[1 + j]
    return out


def _row_case(orc, pde, dim, axis, g, r, nq, nm, prim_to_mat=None):
    """Run one FE stage on a periodic row of 2 patches of 8 voxels along `axis`; return the
    oracle's 16 voxels of the row (per quantity, normal/tangential order) and the grids."""
    p = 8
    n = [1, 1, 1]
    n[axis] = 2
    dx = Fraction(1, 16)
    mesh = single_level(tuple(n), p, float(dx), dim=dim)
    shape = (16 if axis == 2 else p, 16 if axis == 1 else p, 16 if axis == 0 else p)[3 - dim:]
    grid_axis = dim - 1 - axis
    idx = np.arange(16)
    left = idx < 8

    def fill(vals_L, vals_R, rows):
        a = arena(mesh, rows)
        for v in range(rows):
            G = np.empty(shape)
            line = np.where(left, float(vals_L[v]), float(vals_R[v]))
            G[...] = np.expand_dims(line, tuple(k for k in range(dim) if k != grid_axis))
            from_grid(mesh, G, a[v])
        return a

    def phys(Q):  # conserved (scalar, vector n/t..., [scalar]) -> physical component order
        vec = _to_axes(Q[1:1 + dim], axis, dim)
        return [Q[0]] + vec + list(Q[1 + dim:])

    q = fill(phys(g["Q_L"]), phys(g["Q_R"]), nq)
    mat = None
    if nm:
        mL, mR = prim_to_mat(g["prim_L"]), prim_to_mat(g["prim_R"])
        mat = fill(mL, mR, nm)
    out = np.zeros_like(q)
    dt = float(r * dx)
    orc.stage(FV, pde, dim, mesh.patches, 1, mesh.var_stride, q, out=out, mat=mat, dt=dt, a=0, b=1, g=1)
    Gq = [to_grid(mesh, q[v]) for v in range(nq)]
    Go = [to_grid(mesh, out[v]) for v in range(nq)]
    return Gq, Go, phys, grid_axis


def _check_row(Gq, Go, phys, grid_axis, g, nq, tol=1e-14):
    for i in range(16):
        key = f"voxel_{i}"
        for v in range(nq):
            got = np.take(Go[v], i, axis=grid_axis)
            if key in g:
                exp = float(phys(g[key])[v])
                assert np.all(np.abs(got - exp) <= tol * max(1.0, abs(exp))), (key, v, got.ravel()[:3], exp)
            else:  # no face of voxel i carries a jump: bitwise unchanged
                assert np.array_equal(got, np.take(Gq[v], i, axis=grid_axis)), (key, v)


@pytest.mark.parametrize("dim,axis", [(2, 0), (2, 1), (3, 0), (3, 1), (3, 2)])
def test_euler_rusanov_riemann_worked_example(orc, dim, axis):
    fx = load("euler_rusanov_riemann.txt")
    r = fx[""]["dt_over_dx"][0]
    g = fx[f"{dim}d"]
    _euler_lines_agree(g, fx[""]["gamma"][0], dim)
    _rusanov_lines_agree(g)
    _update_lines_agree(g, r)
    pde = EULER2D if dim == 2 else EULER3D
    nq = dim + 2
    Gq, Go, phys, ga = _row_case(orc, pde, dim, axis, g, r, nq, 0)
    _check_row(Gq, Go, phys, ga, g, nq)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_srhd_rusanov_riemann_worked_example(orc, axis):
    fx = load("srhd_rusanov_riemann.txt")
    r = fx[""]["dt_over_dx"][0]
    g = fx["3d"]
    _srhd_lines_agree(g, fx[""]["Gamma"][0])
    _rusanov_lines_agree(g)
    _update_lines_agree(g, r)

    def prim_to_mat(prim):  # (rho, v_n, v_t1, v_t2, p) -> (rho, vx, vy, vz, p)
        return [prim[0]] + _to_axes(prim[1:4], axis, 3) + [prim[4]]

    Gq, Go, phys, ga = _row_case(orc, SRHD3D, 3, axis, g, r, 5, 5, prim_to_mat)
    _check_row(Gq, Go, phys, ga, g, 5)


def test_srhd_speed_along_the_flow_is_the_relativistic_sum():
    """The fixture's s = 17/19 is |(v - cs)/(1 - v cs)| for v = -4/5, cs = 1/3 (state R)."""
    g = load("srhd_rusanov_riemann.txt")["3d"]
    rho, v, p = g["prim_R"][0], g["prim_R"][1], g["prim_R"][4]
    Gm = Fraction(5, 3)
    h = 1 + Gm / (Gm - 1) * p / rho
    cs2 = Gm * p / (rho * h)
    assert cs2 == Fraction(1, 9)
    cs = Fraction(1, 3)
    assert max(abs((v + cs) / (1 + v * cs)), abs((v - cs) / (1 - v * cs))) == g["speed_max"][0]


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_ncp_advection_midpoint_worked_example(orc, axis):
    """Path-conservative midpoint fluctuation with Rusanov dissipation on a material jump:
    bitwise, since every value of the worked example is dyadic."""
    g = load("ncp_advection_midpoint.txt")[""]
    p, ADV_NCP = 8, 1
    n = [1, 1, 1]
    n[axis] = 2
    dx = Fraction(1, 16)
    mesh = single_level(tuple(n), p, float(dx), dim=3)
    shape = (16 if axis == 2 else p, 16 if axis == 1 else p, 16 if axis == 0 else p)
    ga = 2 - axis
    left = np.expand_dims(np.arange(16) < 8, tuple(k for k in range(3) if k != ga))
    q = arena(mesh, 1)
    from_grid(mesh, np.broadcast_to(np.where(left, float(g["Q_left"][0]), float(g["Q_right"][0])), shape).copy(),
              q[0])
    mat = arena(mesh, 3)
    from_grid(mesh, np.broadcast_to(np.where(left, float(g["a_left"][0]), float(g["a_right"][0])), shape).copy(),
              mat[axis])
    out = np.zeros_like(q)
    orc.stage(FV, ADV_NCP, 3, mesh.patches, 1, mesh.var_stride, q, out=out, mat=mat,
              dt=float(g["dt_over_dx"][0] * dx), a=0, b=1, g=1)
    got, before = to_grid(mesh, out[0]), to_grid(mesh, q[0])
    for i in range(16):
        row = np.take(got, i, axis=ga)
        if f"voxel_{i}" in g:
            assert np.all(row == float(g[f"voxel_{i}"][0])), (i, row.ravel()[:2])
        else:
            assert np.array_equal(row, np.take(before, i, axis=ga))


def test_srhd_conversions_on_the_worked_example_states(orc):
    """prim2con of the example's exact primitive states gives its exact conserved states, and
    con2prim (Newton on p, cold seed) recovers the primitives from them."""
    g = load("srhd_rusanov_riemann.txt")["3d"]
    prim = np.array([[float(x) for x in g["prim_L"]], [float(x) for x in g["prim_R"]]]).T.copy()
    cons = np.array([[float(x) for x in g["Q_L"]], [float(x) for x in g["Q_R"]]]).T.copy()
    got = orc.prim2con(SRHD3D, prim, 2)
    assert np.allclose(got, cons, rtol=4e-16, atol=4e-16), got - cons
    rec, status, iters, fails = orc.con2prim(cons, 2)
    assert fails == 0 and np.all(status == 0)
    assert np.allclose(rec, prim, rtol=1e-12, atol=1e-14), rec - prim


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_muscl_advection_kink_worked_example(orc, axis):
    """Second-order stage (MUSCL-minmod into Rusanov) on a ramp between plateaus: bitwise."""
    g = load("muscl_advection_kink.txt")[""]
    p, ADV_FLUX, FV2 = 8, 0, 2
    n = [1, 1, 1]
    n[axis] = 2
    dx = Fraction(1, 16)
    mesh = single_level(tuple(n), p, float(dx), dim=3)
    shape = (16 if axis == 2 else p, 16 if axis == 1 else p, 16 if axis == 0 else p)
    ga = 2 - axis
    other = tuple(k for k in range(3) if k != ga)
    line = np.array([float(x) for x in g["Q"]])
    q = arena(mesh, 1)
    from_grid(mesh, np.broadcast_to(np.expand_dims(line, other), shape).copy(), q[0])
    mat = arena(mesh, 3)
    mat[axis] = float(g["a"][0])
    out = np.zeros_like(q)
    orc.stage(FV2, ADV_FLUX, 3, mesh.patches, 2, mesh.var_stride, q, out=out, mat=mat,
              dt=float(g["dt_over_dx"][0] * dx), a=0, b=1, g=1)
    got = to_grid(mesh, out[0])
    expect = np.broadcast_to(np.expand_dims(np.array([float(x) for x in g["out"]]), other), shape)
    assert np.array_equal(got, expect), np.take(got, 0, axis=other[0]).ravel()[:16]
