"""GPU parity of the first-order FV stage (patch_update_fv, Sec. II-A Eq. 3 with the Rusanov
reading) on discontinuous Euler data, against the FP64 oracle at the 1e-12 rule.

The smooth Fourier workloads never exercise the parts of the stage kernel where the two
implementations could part: the integer-pipe selection of the larger face speed, the refined
reciprocal of rho and the square root of the sound speed at extreme ratios, and the shared
symmetric momentum products at high Mach number.  Each case here is a two-state Riemann
problem laid out in slabs along one axis (so two jumps per periodic row, one of them across a
patch boundary, one inside a patch or on the wrap), run along every axis in 2D and 3D, with
both tile classes (16^2 / 16x16 columns and 8^3 patches in groups of four):

  * the worked example of tests/golden (exact rationals; the four face voxels match it to 1e-14);
  * Sod's shock tube (rho 1 | 0.125, p 1 | 0.1);
  * a strong pressure jump (p 1000 | 0.01, ratio 1e5);
  * near-vacuum: two streams at rho = 1e-6 moving apart at Mach ~3 (every value is small, so
    the per-variable floor of the rule is small too);
  * a Mach-3 stream running into gas at rest;
  * all of the above mixed in random 4^d blocks (jumps across every axis at once).

dt is the CFL step (0.4) of the state; lambda of the result is compared as well."""
import math
from fractions import Fraction

import numpy as np
import pytest

from gpu_util import assert_parity, dev, host, require_cuda
from helpers import arena, from_grid, single_level, to_grid, voxel_mask
from paper_2608_19273_gb300 import dh, synth
from test_oracle_golden import _to_axes, load

pytestmark = pytest.mark.gpu
FV = 0
GAMMA = 1.4
C3 = 3.0 * math.sqrt(GAMMA)  # Mach 3 at rho = 1, p = 1

# (rho, velocity along the slab axis, p); tangential velocities are given per case
RIEMANN = {
    "sod": ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1)),
    "strong_jump": ((1.0, 0.0, 1000.0), (1.0, 0.0, 0.01)),
    "near_vacuum": ((1e-6, -2.0, 4e-7), (1e-6, 2.0, 4e-7)),
    "mach3": ((1.0, C3, 1.0), (1.0, 0.0, 1.0)),
}
TANGENTIAL = (0.3, -0.2)


def _prim_field(mesh, dim, axis, states, nb=2):
    """Primitive arena of a slab pattern along `axis`: the first half of every row takes state 0."""
    G = to_grid(mesh, np.zeros(mesh.var_stride))
    ga = dim - 1 - axis
    n = G.shape[ga]
    left = np.arange(n) < n // 2
    shape = [1] * dim
    shape[ga] = n
    left = left.reshape(shape)
    prim = arena(mesh, dim + 2)
    for v in range(dim + 2):
        vals = []
        for (rho, un, p) in states:
            vel = _to_axes([un] + list(TANGENTIAL[:dim - 1]), axis, dim)
            vals.append([rho] + vel + [p])
        from_grid(mesh, np.broadcast_to(np.where(left, vals[0][v], vals[1][v]), G.shape).copy(), prim[v])
    return prim


def _run_stage(torch, orc, mesh, pde, q, dt, coef=(0.0, 1.0, 1.0)):
    a, b, g = coef
    q0 = q * 0.5 if a else None
    ref = np.zeros_like(q)
    lam_ref = orc.stage(FV, pde, mesh.dim, mesh.patches, 1, mesh.var_stride, q, q0=q0, out=ref, dt=dt, a=a, b=b,
                        g=g, want_lam=True)
    with dh.Plan(pde, mesh.dim, mesh.patches, 1, mesh.var_stride) as plan:
        d_q = dev(torch, q)
        out = torch.zeros_like(d_q)
        d_dt = torch.tensor([dt], dtype=torch.float64, device="cuda")
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dh.patch_update_fv(plan, d_q, dev(torch, q0) if a else None, out, None, None, d_dt, a, b, g, 0.0, lam)
        torch.cuda.synchronize()
        got, lam_got = host(out), float(host(lam)[0])
    return got, ref, lam_got, lam_ref


def _cfl_dt(orc, mesh, pde, q):
    lam = orc.max_wave_speed(pde, mesh.dim, mesh.patches, mesh.var_stride, q)
    return orc.cfl_dt(0.4, float(mesh.patches["dx"].min()), mesh.dim, lam)


CASES = [(2, 0), (2, 1), (3, 0), (3, 1), (3, 2)]


@pytest.mark.parametrize("problem", sorted(RIEMANN))
@pytest.mark.parametrize("dim,axis", CASES)
@pytest.mark.parametrize("p", [8, 16])
def test_riemann_slabs(orc, problem, dim, axis, p):
    torch = require_cuda()
    n = [2] * dim
    n[axis] = 4
    mesh = single_level(tuple(n) if dim == 3 else (n[0], n[1]), p, 1.0 / 64, dim=dim)
    pde = synth.PDE_EULER2D if dim == 2 else synth.PDE_EULER3D
    prim = _prim_field(mesh, dim, axis, RIEMANN[problem])
    q = orc.prim2con(pde, prim, mesh.var_stride)
    dt = _cfl_dt(orc, mesh, pde, q)
    got, ref, lam, lam_ref = _run_stage(torch, orc, mesh, pde, q, dt)
    m = voxel_mask(mesh)
    worst = assert_parity(got, ref, m, what=f"{problem} dim {dim} axis {axis} p {p}")
    assert abs(lam - lam_ref) <= 1e-14 * lam_ref, (lam, lam_ref)
    # the jump moved: the stage is not trivially the identity
    assert np.any(got[:, m] != q[:, m])
    print(f"{problem} dim {dim} axis {axis} p {p}: max relative error {worst:.3e}")


@pytest.mark.parametrize("dim,axis", CASES)
def test_golden_rows_on_the_gpu(orc, dim, axis):
    """The worked example of tests/golden on a periodic row of two 8-voxel patches: the GPU's four
    face voxels equal the exact rationals to 1e-14, every other voxel is bitwise unchanged, and
    the whole row matches the oracle at the 1e-12 rule."""
    torch = require_cuda()
    fx = load("euler_rusanov_riemann.txt")
    r = fx[""]["dt_over_dx"][0]
    g = fx[f"{dim}d"]
    pde = synth.PDE_EULER2D if dim == 2 else synth.PDE_EULER3D
    nq = dim + 2
    p = 8
    n = [1] * dim
    n[axis] = 2
    dx = Fraction(1, 16)
    mesh = single_level(tuple(n), p, float(dx), dim=dim)
    ga = dim - 1 - axis
    G0 = to_grid(mesh, np.zeros(mesh.var_stride))
    shape = [1] * dim
    shape[ga] = 16
    left = (np.arange(16) < 8).reshape(shape)

    def phys(Q):
        return [Q[0]] + _to_axes(Q[1:1 + dim], axis, dim) + list(Q[1 + dim:])

    q = arena(mesh, nq)
    QL, QR = phys(g["Q_L"]), phys(g["Q_R"])
    for v in range(nq):
        from_grid(mesh, np.broadcast_to(np.where(left, float(QL[v]), float(QR[v])), G0.shape).copy(), q[v])
    got, ref, _, _ = _run_stage(torch, orc, mesh, pde, q, float(r * dx))
    assert_parity(got, ref, voxel_mask(mesh), what=f"golden row dim {dim} axis {axis}")
    for i in range(16):
        for v in range(nq):
            row = np.take(to_grid(mesh, got[v]), i, axis=ga)
            key = f"voxel_{i}"
            if key in g:
                exp = float(phys(g[key])[v])
                assert np.all(np.abs(row - exp) <= 1e-14 * max(1.0, abs(exp))), (key, v, row.ravel()[:2], exp)
            else:
                assert np.array_equal(row, np.take(to_grid(mesh, q[v]), i, axis=ga)), (key, v)


@pytest.mark.parametrize("dim,p", [(2, 16), (3, 8), (3, 16)])
@pytest.mark.parametrize("coef", [(0.0, 1.0, 1.0), (1 / 3, 2 / 3, 2 / 3)])
def test_mixed_blocks_every_axis(orc, dim, p, coef):
    """All states of the Riemann cases (with random tangential velocities) in random 4^d blocks:
    jumps of every kind across every axis and every patch face at once."""
    torch = require_cuda()
    n = (2, 2, 2) if dim == 3 else (4, 4)
    mesh = single_level(n, p, 1.0 / 64, dim=dim)
    pde = synth.PDE_EULER2D if dim == 2 else synth.PDE_EULER3D
    states = [s for pair in RIEMANN.values() for s in pair]
    rng = np.random.default_rng(2608 + dim * 100 + p)
    G0 = to_grid(mesh, np.zeros(mesh.var_stride))
    nblk = [s // 4 for s in G0.shape]
    pick = rng.integers(0, len(states), size=nblk)
    axis_of = rng.integers(0, dim, size=nblk)
    tang = rng.uniform(-0.5, 0.5, size=(dim,) + tuple(nblk))
    idx = np.kron(pick, np.ones((4,) * dim, dtype=int))
    ax = np.kron(axis_of, np.ones((4,) * dim, dtype=int))
    prim = arena(mesh, dim + 2)
    Gs = [np.zeros(G0.shape) for _ in range(dim + 2)]
    for si, (rho, un, pr) in enumerate(states):
        sel = idx == si
        Gs[0][sel] = rho
        Gs[dim + 1][sel] = pr
        for a in range(dim):
            t = np.kron(tang[a], np.ones((4,) * dim))
            # the stream's own speed along its block's axis, random tangential components
            Gs[1 + a][sel] = np.where(ax[sel] == a, un, t[sel] * math.sqrt(GAMMA * pr / rho))
    for v in range(dim + 2):
        from_grid(mesh, Gs[v], prim[v])
    q = orc.prim2con(pde, prim, mesh.var_stride)
    dt = _cfl_dt(orc, mesh, pde, q)
    got, ref, lam, lam_ref = _run_stage(torch, orc, mesh, pde, q, dt, coef)
    worst = assert_parity(got, ref, voxel_mask(mesh), what=f"mixed blocks dim {dim} p {p}")
    assert abs(lam - lam_ref) <= 1e-14 * lam_ref, (lam, lam_ref)
    print(f"mixed blocks dim {dim} p {p} coef {coef}: max relative error {worst:.3e}")
