"""The multi-rank bench logic (replicas, max over ranks, whole-job rate) with a
world-size-2 gloo process group on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank           # the slower rank decides
    m = bench.max_over_ranks(ms, tdist)
    rate = bench.whole_job_rate(world, 1000, 10, m)
    tdist.barrier()
    out[rank] = (m, rate)
    tdist.destroy_process_group()


def test_two_rank_max_and_rate():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1]
    m, rate = out[0]
    assert m == 150.0
    assert rate == pytest.approx(2 * 1000 * 10 / 0.150)


def test_single_rank_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(1, 10, 10, 1000.0) == pytest.approx(100.0)
