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


@pytest.mark.parametrize("W,H,S", [(1920, 1080, 10), (37, 23, 5), (1, 1, 1), (7, 9, 64), (13, 4, 3)])
def test_segmentation_roofline_counts_every_existing_candidate(W, H, S):
    """The segmentation roofline divides by the exact number of (pixel, candidate cell) pairs of one
    assignment pass: the cells (i + a, j + b), a, b in {-1, 0, 1}, that exist. Brute force on a grid."""
    import numpy as np

    import bench
    gw, gh = -(-W // S), -(-H // S)
    ci = np.arange(W) // S
    cj = np.arange(H) // S
    nx = sum(1 for a in (-1, 0, 1) for i in ci if 0 <= i + a < gw)
    ny = sum(1 for b in (-1, 0, 1) for j in cj if 0 <= j + b < gh)
    assert bench.seg_candidates(W, H, S) == nx * ny
