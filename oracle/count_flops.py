"""Write oracle/flop_counts.json: exact FP64 operations per voxel of each time-step kind.

Runs the oracle's counting build (scalar type that counts add, sub, mul, div
and sqrt; min, max and abs are free) on one self-periodic patch of size p for
two sizes and separates the per-voxel term from the halo term:
count(p) = A p^d + B p^(d-1)  =>  A = algorithmic operations per voxel.
Only this script (which calls nothing but the oracle) writes the file; the
benchmark reads it as data.
"""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import oracle  # noqa: E402
from paper_2608_19273_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "flop_counts.json")


def _state(pde, dim, p, seed=3):
    mesh = synth.make_mesh([synth.Level((1, 1, 1), p, 1.0 / 64, 0)], dim=dim)
    n = p ** dim
    if pde in (synth.PDE_EULER2D, synth.PDE_EULER3D):
        prim = synth.euler_prims(mesh, seed)
        q = oracle.prim2con(pde, prim, mesh.var_stride)[:, :n]
        return np.ascontiguousarray(q), None
    rng = np.random.default_rng(seed)
    if pde == synth.PDE_SRHD3D:
        prim = synth.srhd_iid_prims(n, seed, wmax=3.0)
        return oracle.prim2con(pde, prim, n), prim
    if pde == synth.PDE_WAVE3D:
        return rng.normal(size=(5, n)), np.full((1, n), 1.3)
    if pde == synth.PDE_GW59:
        q = 1e-3 * rng.normal(size=(59, n))
        q[55] += 1.0
        return q, None
    raise KeyError(pde)


PARAMS = {synth.PDE_GW59: synth.workload("gw59", scale=8).params, synth.PDE_WAVE3D: np.array([0.1])}


def per_voxel(scheme, pde, dim, halo, rk, with_lam, sizes=(8, 16, 24)):
    """Exact fit count(p) = A p^d + B p^(d-1) + C (C: per-stage and per-patch scalars)."""
    c = []
    for p in sizes:
        q, m = _state(pde, dim, p)
        c.append(oracle.count_flops(scheme, pde, dim, p, halo, q, m, rk=rk, with_lam=with_lam,
                                    params=PARAMS.get(pde)))
    M = np.array([[p ** dim, p ** (dim - 1), 1.0] for p in sizes])
    A, B, C = np.linalg.solve(M, np.array(c, dtype=float))
    return A, B, C, c


def compute():
    """The table: per time-step kind, exact FP64 operations per voxel, per face layer and per stage."""
    res = {}
    for key, args in {
        "fv/euler3d/ssprk3_step": (0, synth.PDE_EULER3D, 3, 1, 3, True),
        "fv/euler3d/stage_fe": (0, synth.PDE_EULER3D, 3, 1, 0, False),
        "fv2/euler3d/ssprk3_step": (2, synth.PDE_EULER3D, 3, 2, 3, True),
        "fv/euler2d/fe_step": (0, synth.PDE_EULER2D, 2, 1, 1, True),
        "fd/wave3d/rk4_step": (1, synth.PDE_WAVE3D, 3, 3, 4, True),
        "fv/srhd3d/ssprk3_step": (0, synth.PDE_SRHD3D, 3, 1, 3, False),
        "fd/gw59/rk4_step": (1, synth.PDE_GW59, 3, 3, 4, True),
    }.items():
        A, B, C, c = per_voxel(*args)
        A2, B2, C2, _ = per_voxel(*args, sizes=(8, 16, 32))
        assert abs(A - A2) < 1e-6 and abs(A - round(A)) < 1e-6, (key, A, A2)
        res[key] = {"flops_per_voxel": int(round(A)), "halo_term": round(B, 6), "constant": round(C, 6),
                    "raw_counts": c}
    return res


def con2prim_counts(n=20000, seed=5):
    """Exact split of the plain-seeded SRHD recovery into a per-voxel part (E, |S|^2, |S|, the
    bracket, the cold seed, the recovery of v and rho) and a per-Newton-iteration part:
    count = A n + B iterations, solved from two seeds of different quality on the same states and
    checked on a third (warm seeds: no safeguard step is taken)."""
    prim = synth.srhd_iid_prims(n, seed)
    cons = oracle.prim2con(synth.PDE_SRHD3D, prim, n)
    rows, rhs = [], []
    for rel in (1e-3, 1e-9, 1e-6):
        fl, it = oracle.count_con2prim(cons, n, p_prev=prim[4] * (1 + rel))
        rows.append([n, it])
        rhs.append(fl)
    A, B = np.linalg.solve(np.array(rows[:2], dtype=float), np.array(rhs[:2], dtype=float))
    assert abs(A - round(A)) < 1e-6 and abs(B - round(B)) < 1e-6, (A, B)
    assert round(A) * rows[2][0] + round(B) * rows[2][1] == rhs[2]
    speed = oracle.count_max_speed(synth.PDE_SRHD3D, 3, cons, prim, n)
    assert speed % n == 0
    # derived quantities and the speed of one direction: the kernel evaluates only the direction
    # of the largest |v_d|, whose speed is the largest (the speed increases with |v_d|)
    speed1 = oracle.count_max_speed(synth.PDE_SRHD3D, 1, cons, prim, n)
    assert speed1 % n == 0
    return {"c2p/srhd3d/voxel": {"flops_per_voxel": int(round(A)),
                                 "note": "setup and recovery of one voxel, plain seed, without the Newton iterations"},
            "c2p/srhd3d/newton_iteration": {"flops_per_voxel": int(round(B)),
                                            "note": "one Newton iteration on the pressure (no safeguard step)"},
            "speed/srhd3d/voxel": {"flops_per_voxel": speed // n,
                                   "note": "derived quantities and the speeds of all three directions, from the "
                                           "primitives"},
            "speed/srhd3d/voxel_one_direction": {"flops_per_voxel": speed1 // n,
                                                 "note": "derived quantities and the speed of one direction, "
                                                         "from the primitives"}}


def main():
    res = compute()
    res.update(con2prim_counts())
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1, sort_keys=True)
    print(json.dumps(res, indent=1, sort_keys=True))


if __name__ == "__main__":
    main()
