"""Rotation sharding and the cross-rank max-loc merge, on CPU gloo ranks."""
import math
import os
import socket

import numpy as np
import pytest

from paper_2110_10156_gb300 import shard


def test_shard_range_covers_all_rotations_once():
    for R in (1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            seen = []
            for rank in range(world):
                a, b = shard.shard_range(R, world, rank)
                seen.extend(range(a, b))
            assert seen == list(range(R))


def test_merge_tie_rule_and_invalid():
    e = [(0.5, 10, (1, 2, 3)), (0.7, 40, (0, 0, 1)), (0.7, 12, (4, 5, 6)), (-math.inf, -1, (0, 0, 0))]
    assert shard.merge_best(e) == (0.7, 12, (4, 5, 6))
    assert shard.merge_best([(-math.inf, -1, (0, 0, 0))]) == (-math.inf, -1, (0, 0, 0))
    s, r, sh = shard.local_best([-np.inf, 0.2, 0.2], [[0, 0, 0], [1, 1, 1], [2, 2, 2]], offset=100)
    assert (s, r, sh) == (0.2, 101, (1, 1, 1))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, scores, shifts, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        a, b = shard.shard_range(len(scores), world, rank)
        best = shard.all_merge_best(shard.local_best(scores[a:b], shifts[a:b], a))
        q.put((rank, best))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_all_merge_best_on_gloo_ranks_matches_single_process(world):
    import torch.multiprocessing as mp
    rng = np.random.default_rng(world)
    R = 23
    scores = rng.random(R)
    scores[[3, 17]] = scores.max() + 0.5          # a tie across ranks: index 3 wins
    scores[5] = -np.inf
    shifts = rng.integers(-5, 6, size=(R, 3))
    expect = shard.local_best(scores, shifts, 0)
    assert expect[1] == 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, scores, shifts, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert results[r] == expect
