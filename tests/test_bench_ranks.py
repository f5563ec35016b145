"""The multi-rank logic of bench.py on CPU: two gloo ranks, each with its
own shard (seed), the job's time is the slowest rank's, and the job's rate
counts every rank's units."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [10.0 + rank, 5.0 - rank, 1.0 * (rank + 1)]
        got = bench.max_over_ranks(torch, mine, world, "cpu")
        dist.barrier()
        q.put((rank, bench.rank_seed(rank), got))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_slowest_time_and_distinct_shards():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=100) for _ in range(world)]
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    out.sort()
    assert out[0][2] == out[1][2] == [11.0, 5.0, 2.0]
    assert out[0][1] != out[1][1]


def test_job_rate_counts_every_rank():
    # 2 ranks x 1e6 units x 5 steps in 1000 ms = 10 M units/s for the job
    assert bench.job_rate(1_000_000, 5, 1000.0, 2) == pytest.approx(10.0)
    assert bench.max_over_ranks(torch, [1.5, 2.5], 1, "cpu") == [1.5, 2.5]
