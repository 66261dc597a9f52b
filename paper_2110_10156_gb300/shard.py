"""Rotation sharding across processes (one GPU each) and the max-loc merge.

Rotations are independent (Section 3.2: each candidate rotation gets its own
all-shift map), so a job shards its candidate rotations across ranks with no
exchange on the data path.  Only the final maximum over rotations (Fig. 1)
crosses ranks: each rank contributes its best (score, rotation, shift), a few
bytes, and every rank gets the global best with the library's tie rule (larger
score, then smaller global rotation index).
"""
from __future__ import annotations

import math

import numpy as np


def shard_range(R: int, world: int, rank: int):
    """Contiguous [start, stop) of R rotations for `rank` of `world`."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    base, extra = divmod(R, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def local_best(scores, shifts, offset: int):
    """Best (score, global rotation index, shift) of one rank's results;
    (-inf, -1, (0, 0, 0)) if none is valid."""
    scores = np.asarray(scores, dtype=np.float64)
    shifts = np.asarray(shifts).reshape(-1, 3)
    fin = np.isfinite(scores)
    if not fin.any():
        return -math.inf, -1, (0, 0, 0)
    cand = np.where(fin, scores, -np.inf)
    r = int(np.argmax(cand))               # first maximum: smallest local index
    return float(scores[r]), offset + r, tuple(int(v) for v in shifts[r])


def merge_best(entries):
    """Merge (score, global index, shift) entries with the tie rule."""
    best = (-math.inf, -1, (0, 0, 0))
    for s, r, sh in entries:
        if r < 0:
            continue
        if best[1] < 0 or s > best[0] or (s == best[0] and r < best[1]):
            best = (s, r, tuple(sh))
    return best


def all_merge_best(entry, group=None):
    """Every rank contributes its local best; every rank returns the global one.
    Uses one all_gather of a 5-element float64 tensor on the group's backend."""
    import torch
    import torch.distributed as dist
    s, r, sh = entry
    dev = torch.device("cuda", torch.cuda.current_device()) \
        if dist.get_backend(group) == "nccl" else torch.device("cpu")
    t = torch.tensor([s, float(r), *[float(v) for v in sh]], dtype=torch.float64, device=dev)
    world = dist.get_world_size(group)
    out = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(out, t, group=group)
    rows = [o.cpu().tolist() for o in out]
    return merge_best([(row[0], int(row[1]), tuple(int(v) for v in row[2:])) for row in rows])
