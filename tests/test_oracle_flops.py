"""Pins of the oracle's FP64 operation counts (CPU only).

The roofline's algorithmic FLOPs are the oracle's exact operation counts
(add, sub, mul, div and sqrt count one; min, max and abs are free), taken by
its counting build.  Here they are checked against a count by hand of the
formulas the first-order FV stage evaluates (Sec. II-A, Eq. 3 with the
Rusanov reading; Euler fluxes; the Runge-Kutta stage combination).

Euler 3D, per interior voxel of a forward-Euler stage:
  * derived quantities W: u_k = m_k / rho (3 div); kin = 0 + sum m_k u_k
    (3 mul, 3 add); p = (gamma - 1)(E - kin/2) (1 sub, 1 mul, 1 sub, 1 mul);
    c = sqrt(gamma p / rho) (1 mul, 1 div, 1 sqrt)                        = 16
  * per direction d (three of them):
      - physical flux: m_k u_d (3 mul), + p (1 add), (E + p) u_d (1 add, 1 mul) =  6
      - speed |u_d| + c                                                       =  1
      - the voxel's one face: s/2 (1 mul) and per quantity
        (F_L + F_R)/2 - (s/2)(Q_R - Q_L) (add, mul, sub, mul, sub)           = 26
      - accumulation per quantity: (F+ - F-) and sum + term                   = 10
    together 43 per direction                                               = 129
  * L = -(1/dx) sum: one mul per quantity                                   =   5
  * out = b qs + (g dt) L: mul, mul, add per quantity                       =  15
  total 165 per voxel.
Per patch and face layer (the p^2 term): the face-halo voxels' W (6 x 16),
the flux and speed of the two halo voxels of every line (3 x 2 x 7) and the
extra face of every line (3 x 26): 96 + 42 + 78 = 216.  Per stage: g dt,
d dt (2 mul) and 1/dx (1 div) = 3.

An SSP-RK3 step: stage 1 is that stage (165); stages 2 and 3 add a q0 term
(mul, add per quantity: 175 each); the wave speed of the result adds W and
three speeds (16 + 3): 165 + 175 + 175 + 19 = 534.

Euler 2D, forward-Euler step with the wave speed: W 13 (2 div, 2 mul, 2 add,
4 for p, 3 for c); per direction flux 5, speed 1, face 1 + 4 x 5, accumulation
8 (35, twice 70); L 4; stage 12; wave speed 13 + 2: 114.  Halo term:
4 x 13 + 2 x 2 x 6 + 2 x 21 = 118."""
import json
import os

import numpy as np
import pytest

FV = 0
EULER2D, EULER3D = 2, 3
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (pde, dim, rk, with_lam) -> (per voxel, per face layer, per patch), counted by hand above
HAND = {
    "fv/euler3d/stage_fe": (EULER3D, 3, 0, False, (165, 216, 3)),
    "fv/euler3d/ssprk3_step": (EULER3D, 3, 3, True, (534, 3 * 216, 3 * 3)),
    "fv/euler2d/fe_step": (EULER2D, 2, 1, True, (114, 118, 3)),
}


def _state(dim, p):
    """A smooth positive Euler state on one p^dim patch (the count does not depend on values)."""
    n = p ** dim
    i = np.arange(n)
    rho = 1.0 + 0.25 * np.sin(0.37 * i)
    u = [0.3 * np.cos(0.11 * (k + 1) * i) for k in range(dim)]
    pr = 1.0 + 0.2 * np.cos(0.23 * i)
    E = pr / 0.4 + 0.5 * rho * sum(x * x for x in u)
    return np.ascontiguousarray(np.stack([rho] + [rho * x for x in u] + [E]))


@pytest.mark.parametrize("key", sorted(HAND))
@pytest.mark.parametrize("p", [4, 8])
def test_counting_build_matches_the_hand_count(orc, key, p):
    pde, dim, rk, with_lam, (A, B, C) = HAND[key]
    got = orc.count_flops(FV, pde, dim, p, 1, _state(dim, p), rk=rk, with_lam=with_lam)
    assert got == A * p ** dim + B * p ** (dim - 1) + C


@pytest.mark.parametrize("key", sorted(HAND))
def test_stored_counts_are_the_hand_counts(key):
    """The benchmark reads its algorithmic FLOPs from the stored table."""
    with open(os.path.join(ROOT, "oracle", "flop_counts.json")) as f:
        table = json.load(f)
    A, B, C = HAND[key][4]
    assert table[key]["flops_per_voxel"] == A
    assert table[key]["halo_term"] == B
    assert table[key]["constant"] == C


def test_stored_table_is_what_the_oracle_counts_now():
    """The stored table (the benchmark's algorithmic FLOPs) equals a fresh count of the oracle."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("count_flops", os.path.join(ROOT, "oracle", "count_flops.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    table = mod.compute()
    table.update(mod.con2prim_counts())
    fresh = json.loads(json.dumps(table, sort_keys=True))
    with open(os.path.join(ROOT, "oracle", "flop_counts.json")) as f:
        assert json.load(f) == fresh


# SRHD con2prim, counted by hand from the oracle's formulas (add, sub, mul, div, sqrt = 1):
#   setup     E = tau + D (1); |S|^2 (3 mul + 2 add); |S| (1); |S| - E (1);
#             cold seed (1 + 1e-8) p_lo + 1e-300 and (Gamma - 1) tau (3)          = 11
#   recovery  E + p (1); v = S/(E + p) (3); v^2 (5); W = 1/sqrt(1 - v^2) (3); rho = D/W (1) = 13
#   iteration y = E + p (1); S^2/y^2 (2); sqrt(1 - .) (2); f (S^2/y, y - ., D rt, -, gf *, - p: 6);
#             f' (1 + ., D S^2, y^3 rt (3), /, -, gf *, - 1: 9); p - f/f' (2);
#             |p_new - p| <= tol p_new (2)                                             = 24
#   speeds    derived quantities: v^2 (5), rho h = rho + Gamma p/(Gamma - 1) (4),
#             cs^2 = Gamma p/(rho h) (2) = 11; per direction cs (1), 1 - v^2 cs^2 (2),
#             v_d (1 - cs^2) (2), cs sqrt((1 - v^2)(1 - v^2 cs^2 - v_d^2 (1 - cs^2))) (10),
#             (a +- r)/den (4) = 19                                                    = 11 + 3 x 19
#             (one direction, what the kernel evaluates: the largest |v_d|)           = 11 + 19
C2P_HAND = {"c2p/srhd3d/voxel": 11 + 13, "c2p/srhd3d/newton_iteration": 24, "speed/srhd3d/voxel": 11 + 3 * 19,
            "speed/srhd3d/voxel_one_direction": 11 + 19}


@pytest.mark.parametrize("key", sorted(C2P_HAND))
def test_con2prim_counts_are_the_hand_counts(key):
    with open(os.path.join(ROOT, "oracle", "flop_counts.json")) as f:
        assert json.load(f)[key]["flops_per_voxel"] == C2P_HAND[key]


def test_con2prim_count_of_known_iterations(orc):
    """At rest the cold seed (Gamma - 1) tau is the root, so Newton stops after one iteration:
    the counted work of n such voxels is n x (24 + 24)."""
    n = 64
    prim = np.zeros((5, n))
    prim[0] = np.linspace(0.2, 3.0, n)
    prim[4] = np.linspace(0.1, 5.0, n)
    cons = orc.prim2con(5, prim, n)
    fl, it = orc.count_con2prim(cons, n)
    assert it == n
    assert fl == n * (C2P_HAND["c2p/srhd3d/voxel"] + C2P_HAND["c2p/srhd3d/newton_iteration"])
