"""Multi-rank host logic of bench.py on CPU: world size 2 over gloo.

Each rank reports its own time and match count; the whole-job figures are the
slowest rank's time and the sum of the matches (the one exchange the
arc-range partition needs).
"""
from __future__ import annotations

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = [12.5, 20.0][rank]
    matches = [1000, 234][rank]
    t, m = bench.reduce_over_ranks(ms, matches, dist, "cpu")
    out.put((rank, t, m))
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(2))
    assert got == [(0, 20.0, 1234), (1, 20.0, 1234)]


def test_reduce_single_rank_is_identity():
    import bench

    assert bench.reduce_over_ranks(3.5, 7) == (3.5, 7)
