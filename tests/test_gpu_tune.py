"""Every compiled kernel variant gives the oracle's result, and the autotuner
picks one of them and caches its choice."""
import numpy as np
import pytest

from gpu_util import assert_parity, dev, host, require_cuda
from helpers import voxel_mask
from paper_2608_19273_gb300 import dh, synth

pytestmark = pytest.mark.gpu


# every valid FV variant: bits 0-1 kernel form, bit 2 persistent grid, bits 3-4 tile shape (the
# persistent grid and 32x8 columns come with the register cap, bit 1)
FV_VARIANTS = [v for v in range(24) if (v >> 3) <= 2 and (v & 2 or not (v & 4 or (v >> 3) == 1))]
# one 8x8 column per 64-thread CTA (tile set 3), every kernel form, no persistent grid
FV_VARIANTS += [24, 25, 26, 27]
# TMA staging of the column planes (bit 5; 3D Euler): register cap, one CTA per tile, tile shape 0 or 1
FV_TMA_VARIANTS = [34, 35, 42, 43]


@pytest.mark.parametrize("fv_var", FV_VARIANTS + FV_TMA_VARIANTS)
@pytest.mark.parametrize("fv_zs", [0, 1])
def test_fv_variants_match_oracle(orc, fv_var, fv_zs):
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=4)
    qs = orc.prim2con(3, synth.euler_prims(mesh, 91), mesh.var_stride)
    q0 = orc.prim2con(3, synth.euler_prims(mesh, 92), mesh.var_stride)
    ref = np.zeros_like(qs)
    lam_ref = orc.stage(0, 3, 3, mesh.patches, 1, mesh.var_stride, qs, q0=q0, out=ref, dt=1e-3, a=0.75, b=0.25,
                        g=0.25, want_lam=True)
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        dh.dh_plan_set_variant(plan, fv_var, fv_zs, 0)
        out = torch.zeros(qs.shape, dtype=torch.float64, device="cuda")
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        d_dt = torch.tensor([1e-3], dtype=torch.float64, device="cuda")
        dh.patch_update_fv(plan, dev(torch, qs), dev(torch, q0), out, None, None, d_dt, 0.75, 0.25, 0.25, 0, lam)
        got = host(out)
        assert abs(float(host(lam)[0]) - lam_ref) <= 1e-14 * lam_ref
    assert_parity(got, ref, voxel_mask(mesh), what=f"variant {fv_var}/{fv_zs}")


@pytest.mark.parametrize("fd_var", [0, 2, 4, 6, 12, 20])
@pytest.mark.parametrize("pde", [synth.PDE_WAVE3D, synth.PDE_GW59])
def test_fd_variants_match_oracle(orc, fd_var, pde):
    torch = require_cuda()
    if pde == synth.PDE_GW59 and fd_var in (12, 20):
        with dh.Plan(pde, 3, synth.workload("gw59", scale=8).mesh.patches, 3,
                     synth.workload("gw59", scale=8).mesh.var_stride, synth.workload("gw59", scale=8).params) as plan:
            with pytest.raises(dh.DhError):
                dh.dh_plan_set_variant(plan, 2, 0, fd_var)
        return
    name = "wave3d" if pde == synth.PDE_WAVE3D else "gw59"
    w = synth.workload(name, scale=8)
    mesh = w.mesh
    if pde == synth.PDE_WAVE3D:
        q, mat = synth.wave_initial(mesh, w.seed)
    else:
        q, mat = synth.gw59_initial(mesh, w.seed, amp=1e-3, noise=0.05), None
    ref = np.zeros_like(q)
    orc.stage(1, pde, 3, mesh.patches, 3, mesh.var_stride, q, out=ref, mat=mat, dt=2e-3, sigma=0.1, params=w.params)
    with dh.Plan(pde, 3, mesh.patches, 3, mesh.var_stride, w.params) as plan:
        dh.dh_plan_set_variant(plan, 2, 0, fd_var)
        out = torch.zeros(q.shape, dtype=torch.float64, device="cuda")
        d_dt = torch.tensor([2e-3], dtype=torch.float64, device="cuda")
        dh.patch_update_fd_ko(plan, dev(torch, q), None, out, None, dev(torch, mat) if mat is not None else None, d_dt,
                              0, 1, 1, 0, 0.1)
        got = host(out)
    assert_parity(got, ref, voxel_mask(mesh), what=f"fd variant {fd_var}")


def test_autotune_picks_and_caches(orc, tmp_path):
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=4)
    qs = dev(torch, orc.prim2con(3, synth.euler_prims(mesh, 93), mesh.var_stride))
    out = torch.zeros_like(qs)
    d_dt = torch.tensor([1e-3], dtype=torch.float64, device="cuda")
    cache = str(tmp_path / "tune.jsonl")
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        v, z, f, cached, times = dh.dh_autotune(plan, 0, qs, out, None, d_dt, reps=2, cache_path=cache)
        assert not cached and v in FV_VARIANTS + FV_TMA_VARIANTS and z in (0, 1)
        timed = [t for t in times if t > 0]
        # candidate order: tile shape, grid, z-march, kernel form (bits 0-1); the mix has 32^3
        # and 16^3 patches, so all three tile shapes are candidates (32), then one 8x8 column
        # per 64-thread CTA (8), then the TMA-staged variants (8)
        order = [(vv | (pers << 2) | (tile << 3), zz) for tile in range(3) for pers in range(2) for zz in range(2)
                 for vv in range(4) if not ((pers or tile == 1) and not vv & 2)]
        order += [(24 | vv, zz) for zz in range(2) for vv in range(4)]
        order += [(32 | vv | (tile << 3), zz) for tile in range(2) for zz in range(2) for vv in (2, 3)]
        assert len(order) == 48 and len(timed) == len(order)
        assert min(timed) == timed[order.index((v, z))]
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        v2, z2, f2, cached2, _ = dh.dh_autotune(plan, 0, qs, out, None, d_dt, reps=2, cache_path=cache)
        assert cached2 and (v2, z2, f2) == (v, z, f)


def test_fd_tma_on_single_self_periodic_patch(orc):
    """TMA staging when every face neighbour is the patch itself (all slabs wrap around)."""
    torch = require_cuda()
    mesh = synth.make_mesh([synth.Level((1, 1, 1), 16, 1.0 / 16, 0)], dim=3)
    q, mat = synth.wave_initial(mesh, 3)
    ref = np.zeros_like(q)
    orc.stage(1, synth.PDE_WAVE3D, 3, mesh.patches, 3, mesh.var_stride, q, out=ref, mat=mat, dt=1e-3, sigma=0.1,
              params=[0.1])
    with dh.Plan(synth.PDE_WAVE3D, 3, mesh.patches, 3, mesh.var_stride, [0.1]) as plan:
        dh.dh_plan_set_variant(plan, 2, 0, 6)
        out = torch.zeros(q.shape, dtype=torch.float64, device="cuda")
        d_dt = torch.tensor([1e-3], dtype=torch.float64, device="cuda")
        dh.patch_update_fd_ko(plan, dev(torch, q), None, out, None, dev(torch, mat), d_dt, 0, 1, 1, 0, 0.1)
        got = host(out)
        assert dh.dh_plan_errors(plan) == 0
    assert_parity(got, ref, voxel_mask(mesh), what="tma self-periodic")


def test_fd_tma_bounded_wait_reports_timeout(orc):
    """With the test hook that arms the TMA barriers but issues no copy, every wait runs out:
    the kernel skips its tiles, raises the error flag and the context stays usable."""
    torch = require_cuda()
    mesh = synth.make_mesh([synth.Level((1, 1, 1), 16, 1.0 / 16, 0)], dim=3)
    q, mat = synth.wave_initial(mesh, 4)
    with dh.Plan(synth.PDE_WAVE3D, 3, mesh.patches, 3, mesh.var_stride, [0.1]) as plan:
        dh.dh_plan_set_variant(plan, 2, 0, 6)
        dh.dh_plan_set_debug(plan, 1)
        out = torch.full(q.shape, float("nan"), dtype=torch.float64, device="cuda")
        d_dt = torch.tensor([1e-3], dtype=torch.float64, device="cuda")
        dh.patch_update_fd_ko(plan, dev(torch, q), None, out, None, dev(torch, mat), d_dt, 0, 1, 1, 0, 0.1)
        torch.cuda.synchronize()
        assert dh.dh_plan_errors(plan) & 1
        assert torch.isnan(out).all()          # every tile was skipped
        dh.dh_plan_set_debug(plan, 0)
        dh.patch_update_fd_ko(plan, dev(torch, q), None, out, None, dev(torch, mat), d_dt, 0, 1, 1, 0, 0.1)
        torch.cuda.synchronize()
        assert dh.dh_plan_errors(plan) == 0
        assert torch.isfinite(out[:, :16 ** 3]).all()


def test_variant_rules_rejected(orc):
    """The persistent grid and the 32x8 columns exist only with the register cap (bit 1)."""
    require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=8)
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        for bad in (4, 5, 8, 9, 28, 31, 32, 33, 38, 50, 58, 64):
            with pytest.raises(dh.DhError):
                dh.dh_plan_set_variant(plan, bad, 0, 0)
    # the TMA-staged variant is 3D Euler only
    w = synth.workload("srhd3d", scale=8)
    with dh.Plan(5, 3, w.mesh.patches, 1, w.mesh.var_stride) as plan:
        with pytest.raises(dh.DhError):
            dh.dh_plan_set_variant(plan, 34, 0, 0)


@pytest.mark.parametrize("fv_var", [2 | 4, 2 | 8, 3 | 4 | 8, 2 | 16, 3 | 4 | 16, 24, 3 | 24])
@pytest.mark.parametrize("pde", [synth.PDE_EULER3D, synth.PDE_SRHD3D, synth.PDE_EULER2D])
def test_new_fv_variants_in_captured_graph_steps(orc, fv_var, pde):
    """Persistent grids and the new tile shapes over whole time steps: three SSP-RK3 steps in a
    captured graph (Euler: derived quantities handed between stages; SRHD: con2prim before
    every stage) replayed twice, so that the tile queue is reset and reused, against the
    oracle's steps."""
    torch = require_cuda()
    if pde == synth.PDE_EULER2D:
        mesh = synth.make_mesh([synth.Level((4, 4, 1), 32, 1.0 / 128, 0), synth.Level((4, 4, 1), 16, 1.0 / 64, 1)],
                               dim=2)
        q = orc.prim2con(2, synth.euler_prims(mesh, 95), mesh.var_stride)
        mat, params, dim = None, None, 2
    elif pde == synth.PDE_EULER3D:
        mesh = synth.euler3d_amr_mesh(scale=4)
        q = orc.prim2con(3, synth.euler_prims(mesh, 96), mesh.var_stride)
        mat, params, dim = None, None, 3
    else:
        mesh = synth.make_mesh([synth.Level((2, 2, 2), 32, 1.0 / 64, 0), synth.Level((2, 2, 2), 16, 1.0 / 32, 1)],
                               dim=3)
        mat = synth.srhd_initial(mesh, 97, wmax=3.0)
        q = orc.prim2con(5, mat, mesh.var_stride)
        params, dim = None, 3
    with dh.Plan(pde, dim, mesh.patches, 1, mesh.var_stride, params) as plan:
        dh.dh_plan_set_variant(plan, fv_var, fv_var & 1, 0)
        Q = dev(torch, q)
        M = dev(torch, mat) if mat is not None else None
        U1, U2, R = torch.empty_like(Q), torch.empty_like(Q), torch.empty_like(Q)
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        if pde == synth.PDE_SRHD3D:
            P2 = torch.empty_like(Q)
            dh.con2prim(plan, Q, P2, M[4])
            M.copy_(P2)
        dh.max_wave_speed(plan, Q, M, lam)
        s = torch.cuda.Stream()
        torch.cuda.synchronize()
        dh.dh_graph_capture(plan, 0, 3, 3, Q, U1, U2, R, M, dt, lam, 0.4, 0.1, False, s)
        dh.dh_graph_launch(plan, s)
        dh.dh_graph_launch(plan, s)
        s.synchronize()
        got = host(Q)
    ref = q.copy()
    if pde == synth.PDE_SRHD3D:
        vs = mesh.var_stride
        pr = mat.copy()
        for _ in range(6):
            pr[:], st, _, _ = orc.con2prim(ref, vs, p_prev=np.ascontiguousarray(pr[4]))
            lam_o = orc.max_wave_speed(5, 3, mesh.patches, vs, ref, mat=pr)
            dto = orc.cfl_dt(0.4, float(mesh.patches["dx"].min()), 3, lam_o)
            u1, u2 = np.zeros_like(ref), np.zeros_like(ref)
            for qs, q0, o, a, b, g in ((ref, None, u1, 0, 1, 1), (u1, ref, u2, 0.75, 0.25, 0.25),
                                       (u2, ref, ref, 1 / 3, 2 / 3, 2 / 3)):
                if qs is not ref:
                    pr[:], st, _, _ = orc.con2prim(qs, vs, p_prev=np.ascontiguousarray(pr[4]))
                orc.stage(0, 5, 3, mesh.patches, 1, vs, qs, q0=q0, out=o, mat=pr, dt=dto, a=a, b=b, g=g)
    else:
        orc.rk_steps(0, pde, dim, mesh.patches, 1, mesh.var_stride, ref, rk=3, steps=6, cfl=0.4)
    assert_parity(got, ref, voxel_mask(mesh), what=f"variant {fv_var} pde {pde}, 6 graph steps")


@pytest.mark.parametrize("fv_var", FV_TMA_VARIANTS)
def test_tma_fv_variant_in_captured_graph_steps(orc, fv_var):
    """The TMA-staged stage over whole time steps (derived quantities handed between stages),
    three steps in a captured graph replayed twice, against the oracle's six steps."""
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=4)
    q = orc.prim2con(3, synth.euler_prims(mesh, 98), mesh.var_stride)
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        dh.dh_plan_set_variant(plan, fv_var, fv_var & 1, 0)
        Q = dev(torch, q)
        U1, U2, R = torch.empty_like(Q), torch.empty_like(Q), torch.empty_like(Q)
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        dh.max_wave_speed(plan, Q, None, lam)
        s = torch.cuda.Stream()
        torch.cuda.synchronize()
        dh.dh_graph_capture(plan, 0, 3, 3, Q, U1, U2, R, None, dt, lam, 0.4, 0.1, False, s)
        dh.dh_graph_launch(plan, s)
        dh.dh_graph_launch(plan, s)
        s.synchronize()
        got = host(Q)
        assert dh.dh_plan_errors(plan) == 0
    ref = q.copy()
    orc.rk_steps(0, 3, 3, mesh.patches, 1, mesh.var_stride, ref, rk=3, steps=6, cfl=0.4)
    assert_parity(got, ref, voxel_mask(mesh), what=f"TMA variant {fv_var}, 6 graph steps")


def test_tma_fv_bounded_wait_reports_timeout(orc):
    """With the test hook that arms the barriers but issues no copy, the TMA-staged FV stage's
    first wait of every CTA runs out (later waits of that CTA stop at once): the error flag is
    raised, the launch completes and the context stays usable; without the hook the same plan
    gives the oracle's result."""
    torch = require_cuda()
    mesh = synth.make_mesh([synth.Level((1, 1, 1), 16, 1.0 / 16, 0)], dim=3)
    q = orc.prim2con(3, synth.euler_prims(mesh, 99), mesh.var_stride)
    ref = np.zeros_like(q)
    orc.stage(0, 3, 3, mesh.patches, 1, mesh.var_stride, q, out=ref, dt=1e-3)
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        dh.dh_plan_set_variant(plan, 34, 0, 0)
        dh.dh_plan_set_debug(plan, 1)
        d_q = dev(torch, q)
        out = torch.zeros_like(d_q)
        d_dt = torch.tensor([1e-3], dtype=torch.float64, device="cuda")
        dh.patch_update_fv(plan, d_q, None, out, None, None, d_dt, 0, 1, 1, 0)
        torch.cuda.synchronize()
        assert dh.dh_plan_errors(plan) & 1
        dh.dh_plan_set_debug(plan, 0)
        dh.patch_update_fv(plan, d_q, None, out, None, None, d_dt, 0, 1, 1, 0)
        torch.cuda.synchronize()
        assert dh.dh_plan_errors(plan) == 0
        got = host(out)
    assert_parity(got, ref, voxel_mask(mesh), what="TMA variant after the timeout test")


def test_autotune_steps_picks_a_variant_of_the_step_path(orc, tmp_path):
    """Tuning over whole SSP-RK3 steps (stage-sum form, derived quantities handed between stages):
    every candidate is timed, the choice is one of them, it is cached under its own key, and the
    plan then advances the caller's state like the oracle."""
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=4)
    q = orc.prim2con(3, synth.euler_prims(mesh, 94), mesh.var_stride)
    cache = str(tmp_path / "tune_steps.jsonl")
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as plan:
        Q = dev(torch, q)
        Qt = Q.clone()
        U1, U2, R = torch.empty_like(Q), torch.empty_like(Q), torch.empty_like(Q)
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        dh.max_wave_speed(plan, Q, None, lam)
        lam_t = lam.clone()
        v, z, f, cached, times = dh.dh_autotune_steps(plan, 0, 3, 1, Qt, U1, U2, R, None, dt, lam_t, 0.4, 0.1, reps=1,
                                                      cache_path=cache)
        assert not cached and v in FV_VARIANTS + FV_TMA_VARIANTS
        assert len([x for x in times if x > 0]) == 48
        # the stage tuner's cache entry (other key) is not taken for the step tuner, and vice versa
        v2, z2, _, cached2, _ = dh.dh_autotune_steps(plan, 0, 3, 1, Qt, U1, U2, R, None, dt, lam_t, 0.4, 0.1,
                                                     reps=1, cache_path=cache)
        assert cached2 and (v2, z2) == (v, z)
        _, _, _, cached3, _ = dh.dh_autotune(plan, 0, Q, U1, None, dt, reps=1, cache_path=cache)
        assert not cached3
        dh.dh_plan_set_variant(plan, v, z, 0)
        for _ in range(2):
            dh.dh_rk_step(plan, 0, 3, Q, U1, U2, R, None, dt, lam, 0.4, 0.1)
        got = host(Q)
    ref = q.copy()
    orc.rk_steps(0, 3, 3, mesh.patches, 1, mesh.var_stride, ref, rk=3, steps=2, cfl=0.4)
    assert_parity(got, ref, voxel_mask(mesh), what="after step tuning")
