"""The multi-GPU path of bench.py is replicas only: every rank builds and
queries on its own GPU, and the only exchanges are a barrier and the maximum
of the ranks' times. This checks that host logic with two gloo ranks on CPU
(no GPU): the job time is the slowest rank's, the throughput counts every
rank's units, and every rank sees the same result."""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = 10.0 * (rank + 1) + 0.25          # rank 1 is the slow replica
        t = bench.max_over_ranks(ms, world)
        value = bench.job_throughput(1000, world, t / 1000.0)
        q.put((rank, t, value))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replica_timing_takes_the_slowest_rank(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    slowest = 10.0 * world + 0.25
    for rank, t, value in res:
        assert t == slowest
        assert value == pytest.approx(world * 1000 / (slowest / 1000.0))


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_throughput(10, 1, 2.0) == 5.0
