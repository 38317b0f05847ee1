"""Pins of the SRHD oracle: prim2con / con2prim (Newton on p) and the MLP seed maths (CPU only).

Special-relativistic hydro is not in the paper; the system, the Newton
iteration and the learned seed follow textbook definitions."""
import math

import numpy as np
import pytest

from helpers import arena, single_level, voxel_mask
from paper_2608_19273_gb300 import synth

G = 5.0 / 3.0


def iid_prims(n, seed, wmax=10.0):
    """rho, p log-uniform on [0.1, 10]; Lorentz factor uniform in [1, wmax]; random direction."""
    rng = np.random.default_rng(seed)
    rho = np.exp(rng.uniform(math.log(0.1), math.log(10), n))
    p = np.exp(rng.uniform(math.log(0.1), math.log(10), n))
    W = rng.uniform(1.0, wmax, n)
    v = np.sqrt(1 - 1 / W ** 2)
    nd = rng.normal(size=(3, n))
    nd /= np.linalg.norm(nd, axis=0)
    w = np.zeros((5, n))
    w[0], w[4] = rho, p
    w[1:4] = v * nd
    return w


def test_round_trip_iid(orc):
    w = iid_prims(20000, 1)
    n = w.shape[1]
    q = orc.prim2con(synth.PDE_SRHD3D, w, n)
    got, status, iters, fails = orc.con2prim(q, n)
    assert fails == 0 and np.all(status == 0)
    assert np.max(np.abs(got[4] - w[4]) / w[4]) < 1e-10
    assert np.max(np.abs(got[0] - w[0]) / w[0]) < 1e-10
    assert np.max(np.abs(got[1:4] - w[1:4])) < 1e-10
    assert iters.max() <= 50


def test_at_rest_closed_form(orc):
    """v = 0: p = (Gamma - 1) tau, which the cold seed hits, so Newton stops after one step."""
    w = np.zeros((5, 4))
    w[0] = [0.3, 1.0, 2.0, 7.0]
    w[4] = [0.1, 1.0, 3.0, 9.5]
    q = orc.prim2con(synth.PDE_SRHD3D, w, 4)
    assert np.allclose(q[0], w[0], rtol=0, atol=0)
    assert np.max(np.abs(q[4] - w[4] / (G - 1)) / q[4]) < 1e-15
    got, status, iters, _ = orc.con2prim(q, 4)
    assert np.max(np.abs(got[4] - w[4]) / w[4]) < 1e-15
    assert np.all(iters == 1)


def test_warm_seed_converges_fast(orc):
    w = iid_prims(5000, 2)
    n = w.shape[1]
    q = orc.prim2con(synth.PDE_SRHD3D, w, n)
    _, _, it_cold, _ = orc.con2prim(q, n)
    _, status, it_warm, _ = orc.con2prim(q, n, p_prev=w[4] * (1 + 1e-6))
    assert np.all(status == 0)
    assert it_warm.mean() < it_cold.mean()


def test_unphysical_state_reports_failure(orc):
    """|S| > E + large margin has no physical pressure: status 2, counted, no exception."""
    q = np.zeros((5, 3))
    q[:, 0] = [1.0, 50.0, 0.0, 0.0, 0.1]     # |S| >> tau + D
    q[:, 1] = [1.0, 0.1, 0.0, 0.0, 2.0]      # physical
    q[:, 2] = [1.0, 0.0, 0.0, 0.0, -5.0]     # negative energy
    prim, status, iters, fails = orc.con2prim(q, 3)
    assert status[1] == 0
    assert status[0] == 2 and status[2] == 2
    assert fails == 2


def test_sound_speed_at_rest(orc):
    """v = 0: the characteristic speeds are +-cs, cs^2 = Gamma p / (rho h)."""
    mesh = single_level((1, 1, 1), 8, 1.0 / 8)
    prim = arena(mesh, 5)
    prim[0], prim[4] = 2.0, 3.0
    q = orc.prim2con(synth.PDE_SRHD3D, prim, mesh.var_stride)
    lam = orc.max_wave_speed(synth.PDE_SRHD3D, 3, mesh.patches, mesh.var_stride, q, mat=prim)
    h = 1 + G * 3.0 / ((G - 1) * 2.0)
    assert abs(lam - math.sqrt(G * 3.0 / (2.0 * h))) < 1e-15


def test_light_speed_limit(orc):
    """Every characteristic speed stays below c = 1 even at W = 10."""
    mesh = single_level((1, 1, 1), 8, 1.0 / 8)
    w = iid_prims(512, 3)
    prim = arena(mesh, 5)
    prim[:, :512] = w
    q = orc.prim2con(synth.PDE_SRHD3D, prim, mesh.var_stride)
    lam = orc.max_wave_speed(synth.PDE_SRHD3D, 3, mesh.patches, mesh.var_stride, q, mat=prim)
    assert 0.5 < lam < 1.0


def test_srhd_fv_free_stream_and_conservation(orc):
    mesh = single_level((2, 2, 2), 8, 1.0 / 16)
    prim = arena(mesh, 5)
    prim[0], prim[1], prim[2], prim[3], prim[4] = 1.5, 0.3, -0.4, 0.2, 2.0
    q = orc.prim2con(synth.PDE_SRHD3D, prim, mesh.var_stride)
    out = np.zeros_like(q)
    orc.stage(0, synth.PDE_SRHD3D, 3, mesh.patches, 1, mesh.var_stride, q, out=out, mat=prim, dt=0.01)
    m = voxel_mask(mesh)
    assert np.array_equal(out[:, m], q[:, m])
    rng = np.random.default_rng(4)
    X = synth.voxel_centres(mesh)
    prim[0] = synth.fourier_field(rng, X, [1, 1, 1], 3, 1.0, 0.5)
    prim[4] = synth.fourier_field(rng, X, [1, 1, 1], 3, 1.0, 0.5)
    q = orc.prim2con(synth.PDE_SRHD3D, prim, mesh.var_stride)
    orc.stage(0, synth.PDE_SRHD3D, 3, mesh.patches, 1, mesh.var_stride, q, out=out, mat=prim, dt=0.005)
    for v in range(5):
        assert abs(out[v, m].sum() - q[v, m].sum()) <= 1e-13 * np.abs(q[v, m]).sum()


def test_mlp_gradient_matches_finite_differences(orc):
    rng = np.random.default_rng(5)
    w = rng.normal(scale=0.3, size=1217)
    x = rng.normal(size=(64, 3))
    t = rng.normal(size=64)
    loss, g = orc.mlp_loss_grad(w, x, t)
    h = 1e-6
    idx = rng.choice(1217, 60, replace=False).tolist() + [0, 95, 96, 127, 128, 1151, 1152, 1183, 1184, 1215, 1216]
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (orc.mlp_loss_grad(wp, x, t)[0] - orc.mlp_loss_grad(wm, x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])
    assert abs(loss - np.mean((orc.mlp_forward(w, x) - t) ** 2)) < 1e-14


def test_adam_first_step_closed_form(orc):
    """After one step from zero moments, Adam moves each weight by lr g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    w = np.zeros(4)
    m, v = np.zeros(4), np.zeros(4)
    orc.adam(w, m, v, g, 1, lr=1e-3)
    assert np.max(np.abs(w + 1e-3 * g / (np.abs(g) + 1e-8))) < 1e-18


def test_newton_step_forms_agree(orc):
    """The con2prim Newton step in the form the GPU evaluates (y f and y^2 f' with y = E + p and
    q = sqrt(y^2 - S^2), one reciprocal) equals the textbook step f / f' to rounding, on i.i.d.
    states and pressures around the solution; and the oracle's converged pressure is a root of it."""
    w = iid_prims(4000, 9)
    n = w.shape[1]
    cons = orc.prim2con(synth.PDE_SRHD3D, w, n)
    G = 5.0 / 3.0
    gf = (G - 1) / G
    D, E = cons[0], cons[4] + cons[0]
    S2 = cons[1] ** 2 + cons[2] ** 2 + cons[3] ** 2
    rng = np.random.default_rng(10)
    for rel in (1e-3, 3e-2, 0.3):
        p = w[4] * (1 + rel * rng.uniform(-1, 1, n))
        y = E + p
        a = S2 / y ** 2
        f = gf * (y - S2 / y - D * np.sqrt(1 - a)) - p
        fp = gf * (1 + a - D * S2 / (y ** 3 * np.sqrt(1 - a))) - 1
        q = np.sqrt(y * y - S2)
        num = y * (gf * q * (q - D) - p * y)
        den = gf * S2 * (q - D) / q + (gf - 1) * y * y
        step_text, step_gpu = f / fp, num / den
        # both forms cancel digits for ultra-relativistic states (S^2/y^2 near 1); the steps agree
        # far below the stopping tolerance 1e-12 p
        assert np.all(np.abs(step_gpu - step_text) <= 1e-9 * np.abs(step_text) + 1e-12 * p)
    prim, st, _, _ = orc.con2prim(cons, n)
    assert np.all(st == 0)
    ps = prim[4]
    y = E + ps
    q = np.sqrt(y * y - S2)
    assert np.all(np.abs(gf * q * (q - D) - ps * y) <= 1e-11 * y * ps)


def test_mlp_forward_layout_closed_form(orc):
    """With two isolated paths through the network (input 2 -> hidden-1 unit 5 -> hidden-2 unit 11,
    input 0 -> unit 20 -> unit 3) the forward pass is a closed form in tanh; this fixes the weight
    layout W1[32][3], b1, W2[32][32] (row = output unit), b2, W3, b3 that the GPU kernels share."""
    w = np.zeros(1217)
    W1, b1, W2, b2, W3, b3 = 0, 96, 128, 1152, 1184, 1216
    w[W1 + 3 * 5 + 2], w[b1 + 5], w[W2 + 32 * 11 + 5], w[b2 + 11], w[W3 + 11] = 0.7, 0.1, -1.3, 0.2, 0.9
    w[W1 + 3 * 20 + 0], w[W2 + 32 * 3 + 20], w[W3 + 3] = -0.45, 0.8, 1.7
    w[b3] = -0.4
    x = np.array([[0.3, -2.0, 0.5], [-1.1, 0.4, -0.25], [0.0, 0.0, 0.0]])
    y = orc.mlp_forward(w, x)
    for k in range(len(x)):
        a = 0.9 * math.tanh(-1.3 * math.tanh(0.7 * x[k, 2] + 0.1) + 0.2)
        b = 1.7 * math.tanh(0.8 * math.tanh(-0.45 * x[k, 0]))
        assert abs(y[k] - (a + b - 0.4)) <= 1e-15, (k, y[k], a + b - 0.4)


def test_invariants_closed_form(orc):
    """(|S|/E, D/E, ln(E/D)) with E = tau + D, on a state at rest and on a moving state whose
    conserved variables are exact: rho = 1, |v| = 3/5 (W = 5/4), p = 6/25 gives D = 5/4,
    S = 5/2 v, |S| = 3/2, tau = 101/100."""
    cons = np.zeros((5, 2))
    cons[:, 0] = [2.0, 0.0, 0.0, 0.0, 0.3 / (G - 1.0)]
    cons[:, 1] = [1.25, 0.9, 0.96, 0.72, 1.01]
    x = orc.srhd_invariants(cons, 2)
    E0, E1 = 2.0 + 0.45, 2.26
    assert np.allclose(x[0], [0.0, 2.0 / E0, math.log(E0 / 2.0)], rtol=1e-15, atol=1e-16)
    assert np.allclose(x[1], [1.5 / E1, 1.25 / E1, math.log(E1 / 1.25)], rtol=1e-15, atol=1e-16)


def test_learned_seed_converges_to_the_same_pressure(orc):
    """Whatever network seeds Newton (here an untrained one with random weights), the seeded solve
    converges to the same root as the cold-seeded one within the con2prim tolerance."""
    w = iid_prims(3000, 17, wmax=10.0)
    n = w.shape[1]
    cons = orc.prim2con(synth.PDE_SRHD3D, w, n)
    rng = np.random.default_rng(4)
    mlp = np.zeros(1217 + 6, dtype=np.float32)
    mlp[:1217] = rng.normal(scale=0.3, size=1217)
    mlp[1217:1220] = 0.0  # z-score mean
    mlp[1220:1223] = 1.0  # z-score std
    plain, st0, it0, f0 = orc.con2prim(cons, n)
    seeded, st1, it1, f1 = orc.con2prim(cons, n, mlp=mlp)
    assert f0 == 0 and f1 == 0
    assert np.max(np.abs(seeded[4] - plain[4]) / plain[4]) <= 1e-10
    assert np.max(np.abs(seeded[4] - w[4]) / w[4]) <= 1e-10


def test_oracle_training_reduces_the_seed_loss(orc):
    """A few hundred FP64 Adam steps of the oracle's loss and gradient on the seed's task
    (z-scored invariants -> ln(p/E)) cut the mean squared error by more than half."""
    w = iid_prims(2048, 21, wmax=10.0)
    n = w.shape[1]
    cons = orc.prim2con(synth.PDE_SRHD3D, w, n)
    x = orc.srhd_invariants(cons, n)
    x = (x - x.mean(0)) / x.std(0)
    t = np.log(w[4] / (cons[4] + cons[0]))
    rng = np.random.default_rng(8)
    wt = rng.normal(scale=0.3, size=1217)
    m, v = np.zeros(1217), np.zeros(1217)
    loss0 = orc.mlp_loss_grad(wt, x, t)[0]
    for step in range(1, 301):
        idx = rng.choice(n, 256, replace=False)
        _, g = orc.mlp_loss_grad(wt, x[idx], t[idx])
        orc.adam(wt, m, v, g, step, lr=3e-3)
    loss1 = orc.mlp_loss_grad(wt, x, t)[0]
    assert loss1 < 0.5 * loss0, (loss0, loss1)


def constant_seed_mlp(ln_p_over_E):
    """A network whose output is the constant ln(p/E) = c for every input (all weights zero,
    output bias c; unit z-score scales): its seed is p = E exp(c)."""
    w = np.zeros(1224, dtype=np.float32)
    w[1216] = ln_p_over_E
    w[1220:1223] = 1.0
    return w


def fallback_states(n, seed, min_iters=6):
    """i.i.d. states from which a seed at E e^30 needs at least `min_iters` Newton steps (so that a
    cap of 3 steps misses tolerance by a wide margin), with their exact primitives."""
    import oracle
    w = iid_prims(n, seed)
    cons = oracle.prim2con(synth.PDE_SRHD3D, w, n)
    _, st, it, _ = oracle.con2prim(cons, n, mlp=constant_seed_mlp(30.0), max_iter=50)
    # and from which Newton from the previous pressure (1e-7 off) stops after 2 steps even at a
    # tolerance 100x tighter, so the second step's decision has a wide margin too
    _, st2, it2, _ = oracle.con2prim(cons, n, p_prev=w[4] * (1 + 1e-7), tol=1e-14, max_iter=50)
    keep = (st == 0) & (it >= min_iters) & (st2 == 0) & (it2 == 2)
    w = np.ascontiguousarray(w[:, keep])
    return w, np.ascontiguousarray(cons[:, keep])


def test_seeded_solve_falls_back_to_the_previous_pressure(orc):
    """The learned seed misses tolerance within max_iter = 3 steps; Newton from the previous
    pressure (1e-7 off) then converges in 2: status 1 on every voxel, 3 + 2 iterations, and the
    recovered primitives are the ones the states were made from."""
    w, cons = fallback_states(20000, 41)
    n = w.shape[1]
    assert n > 5000
    prim, st, it, fails = orc.con2prim(cons, n, p_prev=w[4] * (1 + 1e-7), mlp=constant_seed_mlp(30.0),
                                       max_iter=3)
    assert fails == 0 and np.all(st == 1)
    assert np.all(it == 5)
    assert np.max(np.abs(prim[4] - w[4]) / w[4]) < 1e-10
    assert np.max(np.abs(prim[0] - w[0]) / w[0]) < 1e-10
    assert np.max(np.abs(prim[1:4] - w[1:4])) < 1e-10


def test_both_seeds_failing_keeps_the_previous_pressure(orc):
    """When the fallback seed misses tolerance too, status is 2, the pressure is the previous
    pressure itself, the voxel is counted, and v, rho follow from that pressure."""
    w, cons = fallback_states(4000, 42)
    n = w.shape[1]
    E = cons[4] + cons[0]
    p_prev = E * math.exp(30.0)
    prim, st, it, fails = orc.con2prim(cons, n, p_prev=p_prev, mlp=constant_seed_mlp(30.0), max_iter=3)
    assert fails == n and np.all(st == 2) and np.all(it == 6)
    assert np.array_equal(prim[4], p_prev)
    v = cons[1:4] / (E + p_prev)
    assert np.allclose(prim[1:4], v, rtol=1e-15, atol=0)
    assert np.allclose(prim[0], cons[0] * np.sqrt(1 - np.sum(v * v, axis=0)), rtol=1e-15, atol=0)


def test_refinement_off_is_the_plain_recovery(orc):
    """refine = 0 leaves the recovery bitwise as without the option (cold, warm, learned seeds)."""
    w = iid_prims(5000, 51)
    n = w.shape[1]
    q = orc.prim2con(synth.PDE_SRHD3D, w, n)
    mlp = constant_seed_mlp(-1.0)
    for kw in (dict(), dict(p_prev=w[4] * 1.01), dict(mlp=mlp, p_prev=w[4] * 1.01)):
        a = orc.con2prim(q, n, **kw)
        b = orc.con2prim(q, n, refine=0, **kw)
        assert all(np.array_equal(x, y) for x, y in zip(a[:3], b[:3])) and a[3] == b[3]


def test_refinement_at_rest_is_exact_in_one_step(orc):
    """At rest f(p) = (G-1)/G (E + p - D) - p is linear, so one FP32 Newton step from any seed lands
    on its root (G-1) tau to float rounding (q = sqrt(E^2 + p (2 E + p)) is E + p, q - D is formed
    as (B + t)/(q + D) without cancellation)."""
    w = np.zeros((5, 6))
    w[0] = [0.2, 0.5, 1.0, 2.0, 4.0, 9.0]
    w[4] = [0.1, 3.0, 0.7, 6.0, 0.3, 2.0]
    q = orc.prim2con(synth.PDE_SRHD3D, w, 6)
    seeds = np.array([1e-3, 50.0, 0.2, 1e2, 1e-2, 7.0])
    got = orc.refine_seed(q, seeds, 1)
    assert np.all(np.abs(got / w[4] - 1) < 2e-6), got / w[4] - 1
    assert np.all(np.abs(seeds / w[4] - 1) > 0.7)  # every seed far from the root


def test_refinement_converges_quadratically_to_float_precision(orc):
    """Seeds 3% off converge like a Newton iteration: the error after one step is of the order of
    the square of the error before it, down to the floor of the FP32 evaluation (about 1e-6: the
    step is formed from FP64 invariants in which nothing cancels), which three steps reach (W <= 3)."""
    w = iid_prims(20000, 52, wmax=3.0)
    n = w.shape[1]
    q = orc.prim2con(synth.PDE_SRHD3D, w, n)
    rng = np.random.default_rng(53)
    seed = w[4] * np.exp(rng.uniform(-0.03, 0.03, n))
    e0 = np.abs(seed / w[4] - 1)
    e1 = np.abs(orc.refine_seed(q, seed, 1) / w[4] - 1)
    e3 = np.abs(orc.refine_seed(q, seed, 3) / w[4] - 1)
    assert np.all(e1 <= 10 * e0 ** 2 + 1e-6)
    assert np.median(e1[e0 > 1e-2]) < 1e-4
    assert np.max(e3) < 2e-6 and np.median(e3) < 3e-7


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_refined_seeds_reach_the_same_root(orc, k):
    """With the refinement on, cold and learned seeds still converge to the generating pressure
    (1e-10), with no failures, and in fewer FP64 iterations than without it."""
    w = iid_prims(20000, 54)
    n = w.shape[1]
    q = orc.prim2con(synth.PDE_SRHD3D, w, n)
    for kw in (dict(), dict(mlp=constant_seed_mlp(-1.0))):
        prim, st, it, f = orc.con2prim(q, n, refine=k, **kw)
        _, _, it0, _ = orc.con2prim(q, n, **kw)
        assert f == 0 and np.all(st == 0)
        assert np.max(np.abs(prim[4] - w[4]) / w[4]) < 1e-10
        assert it.mean() < it0.mean()


def test_refined_warm_seeds_need_two_fp64_steps(orc):
    """The property the FP32 refinement is for: at Lorentz factors up to 10, where the textbook f
    cancels in FP32, one FP32 step from a previous pressure 0.1% off (two from 1% off) lands within
    2e-6 of the generating pressure, so the FP64 iteration meets the 1e-12 rule after two steps
    (the first corrects the float error, the second confirms) for practically every voxel."""
    w = iid_prims(50000, 55, wmax=10.0)
    n = w.shape[1]
    q = orc.prim2con(synth.PDE_SRHD3D, w, n)
    rng = np.random.default_rng(56)
    for eps, k in ((1e-3, 1), (1e-2, 2)):
        p_prev = w[4] * np.exp(rng.uniform(-eps, eps, n))
        seed = orc.refine_seed(q, p_prev, k)
        assert np.max(np.abs(seed / w[4] - 1)) < 2e-6
        prim, st, it, f = orc.con2prim(q, n, p_prev=p_prev, refine=k)
        assert f == 0 and np.all(st == 0)
        assert np.mean(it == 2) > 0.999, np.bincount(it)
        assert np.max(np.abs(prim[4] - w[4]) / w[4]) < 1e-10
