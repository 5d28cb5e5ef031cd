"""The benchmark's multi-GPU host logic on CPU ranks (gloo, world size 2): every rank runs an
independent replica, the timing is the slowest rank's and the throughput counts every rank's work."""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds = [2.0, 3.0][rank]  # rank 1 is the slowest
    slowest = bench.reduce_max(seconds, "cpu")
    out[rank] = (slowest, bench.whole_job_rate(world, 100.0, slowest))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1] == (3.0, pytest.approx(2 * 100.0 / 3.0))


def test_single_process_without_group():
    import bench
    assert bench.reduce_max(1.5, "cpu") == 1.5
    assert bench.whole_job_rate(1, 10.0, 2.0) == 5.0
