"""Multi-rank layout: disjoint shot ranges and the max / sum reductions, on
CPU with two gloo ranks (the GPU path has no data-path collective)."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp

import synth
from paper_2402_04834_gb300.sharding import reduce_max, reduce_sum, shot_range


def test_shot_ranges_tile_the_job():
    world, per = 4, 25
    seen = []
    for r in range(world):
        a, b = shot_range(r, world, per, first_shot=100)
        seen.extend(range(a, b))
    assert seen == list(range(100, 200))
    with pytest.raises(ValueError):
        shot_range(4, 4, 10)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        a, b = shot_range(rank, world, 8)
        # Each rank samples its own shots; concatenated they are the job's shots.
        _, _, S = synth.sample_syndromes(7, a, b - a, 5, 0.1)
        t = reduce_max(1.0 + rank, dist)
        n = reduce_sum(float(S.shape[0]), dist)
        q.put((rank, a, b, S.sum(), t, n))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_counts():
    world = 2
    port = _free_port()
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    _, _, S = synth.sample_syndromes(7, 0, 16, 5, 0.1)
    assert res[0][1:3] == (0, 8) and res[1][1:3] == (8, 16)
    assert res[0][3] + res[1][3] == S.sum()
    assert all(r[4] == 2.0 for r in res)          # slowest rank wins
    assert all(r[5] == 16.0 for r in res)
