"""Concurrency rule of the C ABI: different plans share nothing, so two plans advanced on two
streams at once give bitwise the results of each advanced alone on one stream (every stage
accumulates its wave speed into its own plan's reduction slots; device-side dt)."""
import numpy as np
import pytest

from gpu_util import dev, host, require_cuda
from paper_2608_19273_gb300 import dh, synth

pytestmark = pytest.mark.gpu


def _advance(torch, plan, q, steps, stream):
    """Every operation (buffer set-up included) on `stream`."""
    with torch.cuda.stream(stream):
        Q = q.clone()
        U1, U2, R = torch.empty_like(Q), torch.empty_like(Q), torch.empty_like(Q)
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        dh.max_wave_speed(plan, Q, None, lam, stream)
        for _ in range(steps):
            dh.dh_rk_step(plan, 0, 3, Q, U1, U2, R, None, dt, lam, 0.4, 0.1, stream)
    return Q, lam, dt


def test_two_plans_on_two_streams_bitwise(orc):
    torch = require_cuda()
    mesh = synth.euler3d_amr_mesh(scale=4)
    qa = dev(torch, orc.prim2con(3, synth.euler_prims(mesh, 91), mesh.var_stride))
    qb = dev(torch, orc.prim2con(3, synth.euler_prims(mesh, 92), mesh.var_stride))
    s0 = torch.cuda.Stream()
    s1 = torch.cuda.Stream()
    with dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as pa, dh.Plan(3, 3, mesh.patches, 1, mesh.var_stride) as pb:
        torch.cuda.synchronize()
        alone = [_advance(torch, pa, qa, 4, s0), _advance(torch, pb, qb, 4, s0)]
        s0.synchronize()
        ra = [host(t) for t in alone[0]]
        rb = [host(t) for t in alone[1]]
        # both at once: plan a on s0, plan b on s1 (no ordering between the streams)
        ca = _advance(torch, pa, qa, 4, s0)
        cb = _advance(torch, pb, qb, 4, s1)
        s0.synchronize()
        s1.synchronize()
        for got, ref in zip(ca, ra):
            assert np.array_equal(host(got), ref)
        for got, ref in zip(cb, rb):
            assert np.array_equal(host(got), ref)
