"""The multi-rank (replicas) bench path on CPU: two gloo ranks, each with its
own step time, must agree on the slowest rank's time and on the whole-job
throughput (every rank's work over that time)."""

import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 175.5][rank]
        dist.barrier()
        ms = bench.job_time_ms(local_ms, world)
        q.put((rank, ms, bench.job_value(world, 2.0e12, ms)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in res:
        assert ms == 175.5
        assert value == pytest.approx(2 * 2.0e12 / 0.1755 / 1e12)


def test_single_rank_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_ms(42.0, 1) == 42.0
    assert bench.job_value(1, 1.0e12, 1000.0) == pytest.approx(1.0)
