"""The multi-rank logic of bench.py on CPU: two gloo ranks, each with its
own shard (seed), the job's time is the slowest rank's, and the job's rate
counts every rank's units; a rank that leaves between steps makes the
survivor's next collective fail with an error within the process group's
timeout instead of hanging."""
import os
import socket
import sys
import time

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


def _rank_leaves(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    bench.init_ranks("gloo", timeout_s=5)
    bench.max_over_ranks(torch, [1.0], world, "cpu")  # one step together
    if rank == 1:
        q.put((rank, "left"))
        q.close()
        q.join_thread()
        os._exit(0)  # gone between steps, without a goodbye
    t0 = time.monotonic()
    try:
        bench.max_over_ranks(torch, [2.0], world, "cpu")
        q.put((rank, "no error"))
    except Exception as e:  # the collective gives up on the missing rank
        q.put((rank, "error after %.1f s: %s" % (time.monotonic() - t0, type(e).__name__)))
    q.close()
    q.join_thread()
    os._exit(0)


@pytest.mark.timeout(120)
def test_a_rank_that_leaves_fails_the_next_collective():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_leaves, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=100) for _ in range(world))
    for p in procs:
        p.join(timeout=30)
    assert out[1] == "left"
    assert out[0].startswith("error after"), out[0]
    assert float(out[0].split()[2]) < 60


def test_job_rate_counts_every_rank():
    # 2 ranks x 1e6 units x 5 steps in 1000 ms = 10 M units/s for the job
    assert bench.job_rate(1_000_000, 5, 1000.0, 2) == pytest.approx(10.0)
    assert bench.max_over_ranks(torch, [1.5, 2.5], 1, "cpu") == [1.5, 2.5]
