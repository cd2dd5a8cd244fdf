"""Multi-process logic of the benchmark on CPU (gloo, world size 2).

The filter shards by plane / image with no exchange, so the only multi-rank logic is
the timing: every rank times its own replica, the slowest rank's time is taken (max
all-reduce), and the whole-job value counts the units of all ranks.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        ms = 10.0 + 5.0 * rank  # rank 1 is slower
        slowest = bench.reduce_max(ms, dist)
        value = bench.whole_job_rate(1000.0, ws, slowest * 1e-3)
        q.put((r, ws, local, slowest, value))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, (r, ws, local, slowest, value) in enumerate(res):
        assert (r, ws, local) == (rank, 2, rank)
        assert slowest == pytest.approx(15.0)
        assert value == pytest.approx(2 * 1000.0 / 0.015)


def test_single_process_defaults():
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert bench.dist_env() == (1, 0, 0)
    assert bench.reduce_max(3.5, None) == 3.5
