"""The replica path of bench.py with more than one rank, on CPU (gloo,
world size 2): every rank reports its own step time, the job takes the
slowest, and the whole-job throughput counts every rank's points."""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    assert bench.dist_setup()[:2] == (world, rank)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist)  # rank 1 is the slowest
    out.put((rank, ms, bench.job_points_per_s(world, 1_000_000, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_points():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in res:
        assert ms == 15.0
        assert abs(value - 2 * 2.0 * 1_000_000 / 0.015 / 1e6) < 1e-6
