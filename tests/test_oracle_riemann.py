"""The first-order FV oracle against the exact solution of the Sod shock tube (CPU only).

The exact solution of the Riemann problem for the Euler equations of an
ideal gas is a textbook construction: the star pressure is the root of
f_L(p) + f_R(p) + u_R - u_L = 0 (shock branch (p - p_K) sqrt(A_K / (p + B_K)),
rarefaction branch 2 c_K / (gamma - 1) ((p / p_K)^((gamma - 1) / (2 gamma)) - 1)),
and the solution at x/t is read off the wave pattern.  It is written out here
from those definitions, independent of the oracle, and itself pinned to the
published star state of Sod's problem (p* = 0.30313, u* = 0.92745).

The oracle's first-order Rusanov scheme (Sec. II-A, Eq. 3 with the Rusanov
reading; forward Euler) must converge to it: the L1 error of the density
falls with the mesh spacing at the rate of a first-order scheme on
discontinuous data (between 1/2, the rate at which a first-order scheme
smears a contact discontinuity, over O(sqrt(t dx)), and 1), and the density
never leaves the range of its initial values (the scheme is monotone on this
problem).  A scheme that converges to another solution (a wrong flux term)
stalls at a fixed error instead."""
import math

import numpy as np

from helpers import arena, from_grid, single_level, to_grid

FV, EULER2D = 0, 2
G = 1.4


def _f(p, rho, pk, ck):
    if p > pk:
        A, B = 2.0 / ((G + 1.0) * rho), (G - 1.0) / (G + 1.0) * pk
        return (p - pk) * math.sqrt(A / (p + B))
    return 2.0 * ck / (G - 1.0) * ((p / pk) ** ((G - 1.0) / (2.0 * G)) - 1.0)


def star_state(L, R):
    (rl, ul, pl), (rr, ur, pr) = L, R
    cl, cr = math.sqrt(G * pl / rl), math.sqrt(G * pr / rr)
    lo, hi = 1e-14, 100.0 * max(pl, pr)
    for _ in range(300):  # f is increasing in p: bisection to the last bit
        mid = 0.5 * (lo + hi)
        if _f(mid, rl, pl, cl) + _f(mid, rr, pr, cr) + ur - ul > 0.0:
            hi = mid
        else:
            lo = mid
    ps = 0.5 * (lo + hi)
    us = 0.5 * (ul + ur) + 0.5 * (_f(ps, rr, pr, cr) - _f(ps, rl, pl, cl))
    return ps, us


def sample(L, R, xi):
    """(rho, u, p) of the exact solution at x/t = xi (interface at x = 0)."""
    (rl, ul, pl), (rr, ur, pr) = L, R
    cl, cr = math.sqrt(G * pl / rl), math.sqrt(G * pr / rr)
    ps, us = star_state(L, R)
    g6 = (G - 1.0) / (G + 1.0)
    if xi <= us:  # left of the contact
        if ps > pl:
            s = ul - cl * math.sqrt((G + 1.0) / (2.0 * G) * ps / pl + (G - 1.0) / (2.0 * G))
            return (rl, ul, pl) if xi <= s else (rl * (ps / pl + g6) / (g6 * ps / pl + 1.0), us, ps)
        head, tail = ul - cl, us - cl * (ps / pl) ** ((G - 1.0) / (2.0 * G))
        if xi <= head:
            return rl, ul, pl
        if xi >= tail:
            return rl * (ps / pl) ** (1.0 / G), us, ps
        u = 2.0 / (G + 1.0) * (cl + 0.5 * (G - 1.0) * ul + xi)
        c = 2.0 / (G + 1.0) * (cl + 0.5 * (G - 1.0) * (ul - xi))
        return rl * (c / cl) ** (2.0 / (G - 1.0)), u, pl * (c / cl) ** (2.0 * G / (G - 1.0))
    if ps > pr:
        s = ur + cr * math.sqrt((G + 1.0) / (2.0 * G) * ps / pr + (G - 1.0) / (2.0 * G))
        return (rr, ur, pr) if xi >= s else (rr * (ps / pr + g6) / (g6 * ps / pr + 1.0), us, ps)
    head, tail = ur + cr, us + cr * (ps / pr) ** ((G - 1.0) / (2.0 * G))
    if xi >= head:
        return rr, ur, pr
    if xi <= tail:
        return rr * (ps / pr) ** (1.0 / G), us, ps
    u = 2.0 / (G + 1.0) * (-cr + 0.5 * (G - 1.0) * ur + xi)
    c = 2.0 / (G + 1.0) * (cr - 0.5 * (G - 1.0) * (ur - xi))
    return rr * (c / cr) ** (2.0 / (G - 1.0)), u, pr * (c / cr) ** (2.0 * G / (G - 1.0))


SOD_L, SOD_R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)


def test_exact_solver_reproduces_the_published_sod_star_state():
    ps, us = star_state(SOD_L, SOD_R)
    assert abs(ps - 0.30313) < 5e-6 and abs(us - 0.92745) < 5e-6
    # the solution is continuous across the rarefaction's edges and the contact keeps u and p
    for edge in (-math.sqrt(G), us - math.sqrt(G) * (ps / 1.0) ** ((G - 1) / (2 * G))):
        a, b = sample(SOD_L, SOD_R, edge - 1e-9), sample(SOD_L, SOD_R, edge + 1e-9)
        assert max(abs(x - y) for x, y in zip(a, b)) < 1e-7
    a, b = sample(SOD_L, SOD_R, us - 1e-9), sample(SOD_L, SOD_R, us + 1e-9)
    assert abs(a[1] - b[1]) < 1e-12 and abs(a[2] - b[2]) < 1e-12 and a[0] > b[0]


def _sod_run(orc, N, t_end=0.2):
    """Periodic row of length 2: state L on [0.5, 1.5), state R outside, so two Sod problems
    (the one at 0.5 mirrored) that do not meet before t = 0.2.  Returns x, rho, rho_exact."""
    nx, p = N // 8, 8
    dx = 2.0 / N
    mesh = single_level((nx, 1, 1), p, dx, dim=2)
    x = (np.arange(N) + 0.5) * dx
    inside = (x >= 0.5) & (x < 1.5)
    prim = arena(mesh, 4)
    for v, (a, b) in enumerate(zip((SOD_L[0], SOD_L[1], 0.0, SOD_L[2]), (SOD_R[0], SOD_R[1], 0.0, SOD_R[2]))):
        from_grid(mesh, np.repeat(np.where(inside, a, b)[None, :], p, axis=0), prim[v])
    q = orc.prim2con(EULER2D, prim, mesh.var_stride)
    steps = int(math.ceil(t_end / (0.2 * dx)))  # lambda_max dt / dx <= 0.39 (lambda_max < 1.93)
    orc.rk_steps(FV, EULER2D, 2, mesh.patches, 1, mesh.var_stride, q, rk=1, steps=steps, dt_fixed=t_end / steps)
    rho = to_grid(mesh, q[0])
    assert np.all(rho == rho[0:1, :])  # every row of the 2D patch row evolves identically
    exact = np.empty(N)
    for i, xi in enumerate(x):
        if xi >= 1.0:
            exact[i] = sample(SOD_L, SOD_R, (xi - 1.5) / t_end)[0]
        else:  # mirror image of the problem at 1.5
            exact[i] = sample(SOD_L, SOD_R, (0.5 - xi) / t_end)[0]
    return x, rho[0], exact


def test_first_order_scheme_converges_to_the_exact_sod_solution(orc):
    errs = []
    for N in (128, 256, 512):
        x, rho, exact = _sod_run(orc, N)
        assert rho.min() >= SOD_R[0] - 1e-12 and rho.max() <= SOD_L[0] + 1e-12
        errs.append(np.abs(rho - exact).sum() * (2.0 / N))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 0.05, errs
    assert all(0.4 < r < 1.1 for r in rates), (errs, rates)
