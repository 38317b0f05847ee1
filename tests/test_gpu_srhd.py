"""GPU parity of the SRHD path: prim2con, con2prim (plain and MLP-seeded Newton),
the FV stage with SRHD fluxes, and the MLP forward/backward/Adam kernels, against
the FP64 oracle.  con2prim tolerance: 1e-10 relative; status arrays bit-exact."""
import math

import numpy as np
import pytest

from gpu_util import assert_parity, dev, host, require_cuda
from helpers import arena, single_level, voxel_mask
from paper_2608_19273_gb300 import dh, synth
from test_oracle_srhd import constant_seed_mlp, fallback_states, iid_prims

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0


def _flat_c2p(torch, cons, p_prev=None, mlp=None, refine=0):
    n = cons.shape[1]
    d_cons = dev(torch, cons)
    prim = torch.zeros_like(d_cons)
    status = torch.zeros(n, dtype=torch.uint8, device="cuda")
    iters = torch.zeros(n, dtype=torch.int32, device="cuda")
    fails = torch.zeros(1, dtype=torch.int32, device="cuda")
    dh.con2prim_flat(d_cons, prim, n, n, dev(torch, p_prev) if p_prev is not None else None,
                     dev(torch, mlp) if mlp is not None else None, G, 1e-12, 50, status, iters, fails,
                     seed_refine=refine)
    torch.cuda.synchronize()
    return host(prim), host(status), host(iters), int(host(fails)[0])


def test_prim2con_gpu_matches_oracle(orc):
    torch = require_cuda()
    for pde, mesh in ((synth.PDE_SRHD3D, single_level((2, 2, 2), 8, 1 / 16)),
                      (synth.PDE_EULER3D, synth.euler3d_amr_mesh(scale=8))):
        if pde == synth.PDE_SRHD3D:
            prim = arena(mesh, 5)
            m = voxel_mask(mesh)
            prim[:, m] = iid_prims(int(m.sum()), 11)
        else:
            prim = synth.euler_prims(mesh, 3)
        ref = orc.prim2con(pde, prim, mesh.var_stride)
        with dh.Plan(pde, 3, mesh.patches, 1, mesh.var_stride) as plan:
            out = torch.zeros(ref.shape, dtype=torch.float64, device="cuda")
            dh.dh_prim2con(plan, dev(torch, prim), out)
            got = host(out)
        assert_parity(got, ref, voxel_mask(mesh), tol=1e-14, what=f"prim2con pde {pde}")


@pytest.mark.parametrize("warm", [False, True])
def test_con2prim_plain(orc, warm):
    torch = require_cuda()
    w = iid_prims(50000, 21)
    n = w.shape[1]
    cons = orc.prim2con(synth.PDE_SRHD3D, w, n)
    p_prev = w[4] * (1 + 1e-6) if warm else None
    ref, st_ref, it_ref, f_ref = orc.con2prim(cons, n, p_prev=p_prev)
    got, st, it, f = _flat_c2p(torch, cons, p_prev)
    assert np.array_equal(st, st_ref) and f == f_ref == 0
    assert_parity(got, ref, np.ones(n, dtype=bool), tol=1e-10, what="con2prim")
    assert_parity(got, w, np.ones(n, dtype=bool), tol=1e-10, what="round trip")
    assert abs(it.mean() - it_ref.mean()) < 0.05 * it_ref.mean()


def test_con2prim_unphysical_reports(orc):
    torch = require_cuda()
    cons = np.zeros((5, 4))
    cons[:, 0] = [1.0, 50.0, 0.0, 0.0, 0.1]
    cons[:, 1] = [1.0, 0.1, 0.0, 0.0, 2.0]
    cons[:, 2] = [1.0, 0.0, 0.0, 0.0, -5.0]
    cons[:, 3] = [1.0, 0.0, 0.0, 0.0, float("nan")]
    _, st_ref, _, f_ref = orc.con2prim(cons, 4)
    _, st, _, f = _flat_c2p(torch, cons)
    assert np.array_equal(st, st_ref)
    assert f == f_ref and f >= 2 and st[1] == 0


def _random_mlp(rng):
    w = np.zeros(1224, dtype=np.float32)
    w[:1217] = rng.normal(scale=0.4, size=1217)
    w[1217:1220] = [0.3, 0.4, 0.8]
    w[1220:1223] = [0.2, 0.25, 0.6]
    return w


def test_mlp_forward_and_gradient_vs_oracle(orc):
    torch = require_cuda()
    rng = np.random.default_rng(7)
    w = _random_mlp(rng)
    n = 4000
    xraw = rng.uniform([0.0, 0.05, 0.0], [1.0, 1.0, 2.5], size=(n, 3)).astype(np.float32)
    t = rng.normal(size=n).astype(np.float32)
    xn = (xraw.astype(np.float64) - w[1217:1220].astype(np.float64)) / w[1220:1223].astype(np.float64)
    xn = xn.astype(np.float32).astype(np.float64)
    y_ref = orc.mlp_forward(w[:1217].astype(np.float64), xn)
    d_w, d_x, d_t = dev(torch, w), dev(torch, xraw), dev(torch, t)
    y = torch.zeros(n, dtype=torch.float32, device="cuda")
    dh.dh_mlp_forward(d_w, d_x, n, y)
    assert np.max(np.abs(host(y) - y_ref)) < 2e-5 * max(1.0, np.max(np.abs(y_ref)))
    loss_ref, g_ref = orc.mlp_loss_grad(w[:1217].astype(np.float64), xn, t.astype(np.float64))
    part = torch.zeros(((n + 63) // 64) * 1224, dtype=torch.float32, device="cuda")
    grad = torch.zeros(1224, dtype=torch.float32, device="cuda")
    dh.dh_mlp_grad(d_w, d_x, d_t, 0, n, part, grad)
    g = host(grad)
    assert abs(g[1217] - loss_ref) <= 1e-5 * loss_ref
    for lo, hi in ((0, 96), (96, 128), (128, 1152), (1152, 1184), (1184, 1216), (1216, 1217)):
        err = np.linalg.norm(g[lo:hi] - g_ref[lo:hi]) / max(np.linalg.norm(g_ref[lo:hi]), 1e-30)
        assert err <= 1e-4, (lo, hi, err)
    # determinism: the same call gives bitwise the same gradient
    grad2 = torch.zeros_like(grad)
    dh.dh_mlp_grad(d_w, d_x, d_t, 0, n, part, grad2)
    assert torch.equal(grad, grad2)


def test_mlp_adam_vs_oracle(orc):
    torch = require_cuda()
    rng = np.random.default_rng(8)
    w = rng.normal(size=1224).astype(np.float32)
    g = rng.normal(size=1224).astype(np.float32)
    m = (0.1 * rng.normal(size=1224)).astype(np.float32)
    v = np.abs(0.1 * rng.normal(size=1224)).astype(np.float32)
    wr, mr, vr = w[:1217].astype(np.float64), m[:1217].astype(np.float64), v[:1217].astype(np.float64)
    orc.adam(wr, mr, vr, g[:1217].astype(np.float64), 5)
    d_w, d_m, d_v = dev(torch, w), dev(torch, m), dev(torch, v)
    dh.dh_mlp_adam(d_w, d_m, d_v, dev(torch, g), 5)
    assert np.max(np.abs(host(d_w)[:1217] - wr)) < 1e-6
    assert np.max(np.abs(host(d_m)[:1217] - mr)) < 1e-6


def train_seed_mlp(torch, orc, n=1_000_000, steps=6000, seed=260819276):
    """Train the seed network on n oracle prim2con pairs with the library kernels."""
    w_prim = iid_prims(n, seed)
    cons = orc.prim2con(synth.PDE_SRHD3D, w_prim, n)
    d_cons = dev(torch, cons)
    d_p = dev(torch, np.ascontiguousarray(w_prim[4]))
    x = torch.zeros(n * 3, dtype=torch.float32, device="cuda")
    y = torch.zeros(n, dtype=torch.float32, device="cuda")
    dh.dh_mlp_features(d_cons, d_p, n, n, x, y)
    rng = np.random.default_rng(seed)
    w = np.zeros(1224, dtype=np.float32)
    # Xavier (Glorot) uniform initial weights, zero biases
    for off, fan_in, fan_out in ((0, 3, 32), (128, 32, 32), (1184, 32, 1)):
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        w[off:off + fan_in * fan_out] = rng.uniform(-lim, lim, fan_in * fan_out)
    d_w = dev(torch, w)
    scratch = torch.zeros(6 * 1024, dtype=torch.float64, device="cuda")
    dh.dh_mlp_standardize(x, n, d_w, scratch)
    m = torch.zeros(1224, dtype=torch.float32, device="cuda")
    v = torch.zeros(1224, dtype=torch.float32, device="cuda")
    B = 4096
    part = torch.zeros((B // 64) * 1224, dtype=torch.float32, device="cuda")
    grad = torch.zeros(1224, dtype=torch.float32, device="cuda")
    loss = torch.zeros(steps, dtype=torch.float32, device="cuda")
    dh.dh_mlp_train(d_w, m, v, x, y, n, B, steps, 0, 1e-3, part, grad, loss)
    torch.cuda.synchronize()
    return host(d_w), host(loss)


def _warp_cost(it):
    """Mean over warps of 32 consecutive voxels of their largest iteration count (what a warp pays)."""
    m = len(it) // 32 * 32
    return it[:m].reshape(-1, 32).max(axis=1).mean()


def test_mlp_training_and_seeded_newton(orc):
    """Train on oracle pairs.  The learned seed (refined by 3 FP32 Newton steps) converges to the
    oracle's answer (held-out i.i.d. states), and on the full-size SRHD workload after one FV stage
    it beats plain Newton from the previous pressure -- the method without the network -- in FP64
    Newton iterations per warp (a warp runs until its slowest lane converges) and in device time."""
    torch = require_cuda()
    w, loss = train_seed_mlp(torch, orc, n=200_000, steps=3000)
    assert loss[-100:].mean() < 0.1 * loss[:20].mean()
    held = iid_prims(20000, 99)
    n = held.shape[1]
    cons = orc.prim2con(synth.PDE_SRHD3D, held, n)
    for refine in (0, 3):
        ref, st_ref, it_ref, _ = orc.con2prim(cons, n, mlp=w, refine=refine)
        got, st, it, f = _flat_c2p(torch, cons, mlp=w, refine=refine)
        assert f == 0
        assert np.array_equal(st, st_ref)
        assert_parity(got, ref, np.ones(n, dtype=bool), tol=1e-10, what=f"mlp-seeded con2prim, refine {refine}")
    # warm states: the workload after one stage, seeded by the pressure before it
    wl = synth.workload("srhd3d")
    mesh = wl.mesh
    with dh.Plan(5, 3, mesh.patches, 1, mesh.var_stride, wl.params) as plan:
        prim0 = torch.from_numpy(synth.srhd_initial(mesh, wl.seed)).cuda()
        q0 = torch.empty_like(prim0)
        dh.dh_prim2con(plan, prim0, q0)
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        dh.max_wave_speed(plan, q0, prim0, lam)
        dh.dh_cfl_dt(plan, lam, 0.4, dt)
        u1 = torch.empty_like(q0)
        dh.patch_update_fv(plan, q0, None, u1, None, prim0, dt, 0, 1, 1, 0)
        p_prev = prim0[4].contiguous()
        d_w = dev(torch, w)
        res = {}
        for name, mlp, refine in (("plain", None, 0), ("learned", d_w, 3)):
            prim = torch.empty_like(u1)
            its = torch.zeros(mesh.var_stride, dtype=torch.int32, device="cuda")
            st = torch.zeros(mesh.var_stride, dtype=torch.uint8, device="cuda")
            dh.con2prim(plan, u1, prim, p_prev, mlp, 1e-12, 50, st, its, None, seed_refine=refine)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                dh.con2prim(plan, u1, prim, p_prev, mlp, 1e-12, 50, st, its, None, seed_refine=refine)
            e1.record()
            torch.cuda.synchronize()
            m = voxel_mask(mesh)
            assert np.all(host(st)[m] == 0)
            res[name] = (_warp_cost(host(its)[m]), e0.elapsed_time(e1) / 3, host(prim)[:, m][:, ::97])
    print(f"warm workload stage: FP64 iterations per warp plain {res['plain'][0]:.2f}, learned {res['learned'][0]:.2f}; "
          f"device time {res['plain'][1]:.3f} ms vs {res['learned'][1]:.3f} ms")
    assert res["learned"][0] < res["plain"][0]
    assert res["learned"][1] < res["plain"][1]
    # both seeds reach the same primitives (tolerance of con2prim)
    assert_parity(res["learned"][2], res["plain"][2], np.ones(res["plain"][2].shape[1], dtype=bool), tol=1e-10,
                  what="learned vs plain seed")


@pytest.mark.parametrize("refine", [1, 3])
@pytest.mark.parametrize("seed", ["cold", "warm", "mlp"])
def test_con2prim_refined_seed_matches_oracle(orc, refine, seed):
    """The FP32 refinement of the first seed (the same float operations on both sides): status
    arrays equal the oracle's, primitives within 1e-10 of the oracle's and of the generating
    states, mean FP64 iterations within 5% and below those without the refinement."""
    torch = require_cuda()
    w = iid_prims(50000, 61)
    n = w.shape[1]
    cons = orc.prim2con(synth.PDE_SRHD3D, w, n)
    rng = np.random.default_rng(62)
    p_prev = w[4] * np.exp(rng.uniform(-1e-3, 1e-3, n)) if seed == "warm" else None
    mlp = constant_seed_mlp(-1.0) if seed == "mlp" else None
    ref, st_ref, it_ref, f_ref = orc.con2prim(cons, n, p_prev=p_prev, mlp=mlp, refine=refine)
    got, st, it, f = _flat_c2p(torch, cons, p_prev, mlp, refine)
    _, _, it0, _ = _flat_c2p(torch, cons, p_prev, mlp, 0)
    assert np.array_equal(st, st_ref) and f == f_ref == 0
    worst = assert_parity(got, ref, np.ones(n, dtype=bool), tol=1e-10, what=f"refined {seed} seed")
    assert_parity(got, w, np.ones(n, dtype=bool), tol=1e-10, what="round trip")
    assert abs(it.mean() - it_ref.mean()) < 0.05 * it_ref.mean()
    assert it.mean() < it0.mean()
    print(f"{seed} seed + {refine} FP32 steps: FP64 iterations {it0.mean():.2f} -> {it.mean():.2f}, "
          f"max relative error {worst:.2e}")


@pytest.mark.gpu
def test_integer_pipe_conversions_match_hardware():
    """The seed paths convert between FP64 and FP32 with bit operations (the hardware conversions
    run on the FP64 pipe); the results must be the hardware's bit for bit: random bit patterns
    over every exponent, exact ties between adjacent floats (round half to even) and their
    neighbours one double ulp away, the edges of the float range, and every float class."""
    torch = require_cuda()
    rng = np.random.default_rng(71)
    n = 1 << 20
    parts = [rng.integers(0, 2 ** 64, n, dtype=np.uint64, endpoint=False).view(np.float64)]
    # doubles within the float exponent range
    e = rng.integers(1023 - 130, 1023 + 130, n, dtype=np.uint64)
    m = rng.integers(0, 2 ** 52, n, dtype=np.uint64)
    s = rng.integers(0, 2, n, dtype=np.uint64)
    parts.append(((s << np.uint64(63)) | (e << np.uint64(52)) | m).view(np.float64))
    # ties between adjacent floats and one double ulp either side
    f = rng.standard_normal(n).astype(np.float32) * np.float32(2.0) ** rng.integers(-120, 120, n).astype(np.float32)
    f = f[np.isfinite(f) & (f != 0)]
    tie = (f.astype(np.float64) + np.nextafter(f, np.float32(np.inf)).astype(np.float64)) / 2.0
    parts += [tie, np.nextafter(tie, np.inf), np.nextafter(tie, -np.inf)]
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 3.4028234663852886e38, 3.4028235677973366e38,
                        3.402823669209385e38, 1.1754943508222875e-38, 1.1754942e-38, 1.4e-45, 7e-46, 1e-300,
                        1e300, 1.0, -1.0, 0.1, 2.0 ** -126, 2.0 ** -127, 2.0 ** 127, 2.0 ** 128])
    parts.append(special)
    x = np.ascontiguousarray(np.concatenate(parts))
    g = rng.integers(0, 2 ** 32, len(x), dtype=np.uint64).astype(np.uint32).view(np.float32)
    g[: 8] = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.4e-45, 1.1754942e-38, 3.4028235e38], dtype=np.float32)
    dx = torch.from_numpy(x).cuda()
    dg = torch.from_numpy(np.ascontiguousarray(g)).cuda()
    fi, fh = (torch.empty(len(x), dtype=torch.float32, device="cuda") for _ in range(2))
    di, dh_ = (torch.empty(len(x), dtype=torch.float64, device="cuda") for _ in range(2))
    dh.dh_check_convert(dx, fi, fh, dg, di, dh_)
    torch.cuda.synchronize()
    fi, fh, di, dh_ = (t.cpu().numpy() for t in (fi, fh, di, dh_))
    nan_f = np.isnan(fi) & np.isnan(fh)
    assert np.all((fi.view(np.uint32) == fh.view(np.uint32)) | nan_f)
    with np.errstate(over="ignore", invalid="ignore"):
        x32 = x.astype(np.float32)
    assert np.all((fh.view(np.uint32) == x32.view(np.uint32)) | nan_f)  # IEEE RN
    nan_d = np.isnan(di) & np.isnan(dh_)
    assert np.all((di.view(np.uint64) == dh_.view(np.uint64)) | nan_d)


@pytest.mark.gpu
@pytest.mark.parametrize("seed,wmax", [(81, 10.0), (82, 10.0), (83, 1.5), (84, 3.0)])
def test_srhd_max_wave_speed_matches_oracle(orc, seed, wmax):
    """max_wave_speed for SRHD evaluates only the direction of the largest |v_d| (the speed grows
    with |v_d|); the maximum over the mesh must equal the oracle's three-direction maximum to one
    unit in the last place, on i.i.d. states of several Lorentz factor ranges."""
    torch = require_cuda()
    mesh = single_level((4, 4, 4), 16, 1.0 / 64)
    n = mesh.var_stride
    w = iid_prims(n, seed, wmax=wmax)
    params = synth.workload("srhd3d").params
    q = orc.prim2con(synth.PDE_SRHD3D, w, n)
    ref = orc.max_wave_speed(synth.PDE_SRHD3D, 3, mesh.patches, n, q, mat=w, params=params)
    with dh.Plan(synth.PDE_SRHD3D, 3, mesh.patches, 1, n, params) as plan:
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dh.max_wave_speed(plan, dev(torch, q), dev(torch, w), lam)
        got = float(host(lam)[0])
    assert abs(got - ref) <= 2.3e-16 * ref, (got, ref)
