"""The multi-GPU path of bench.py is replicas: each rank runs the whole frame, the job's time is
the slowest rank's and its throughput the sum over ranks.  Host logic on two gloo ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys

    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    assert bench.dist_env() == (rank, world, rank)
    t = bench.max_over_ranks(0.5 + rank, torch.device("cpu"))     # rank 1 is the slow one
    v = bench.job_throughput(world, 1920 * 1080 * 8, 100, t)
    dist.barrier()
    q.put((rank, t, v))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [1.5, 1.5]
    assert got[0][2] == got[1][2] == pytest.approx(2 * 1920 * 1080 * 8 * 100 / 1.5)


def test_single_process_needs_no_group():
    import sys

    import torch
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, torch.device("cpu")) == 3.0
    assert bench.job_throughput(1, 10, 4, 2.0) == 20.0
