"""Sharding of batched registration across processes, one per GPU.

Registration pairs are independent of one another, so a batch shards by
pair with no exchange during the registration: every rank registers its own
subset of the pairs through its own batch context on its own GPU, and the
poses are gathered once at the end.  This module holds only that host-side
bookkeeping -- which rank takes which pairs, and the gather of the results --
and does no registration arithmetic.
"""
from __future__ import annotations

import numpy as np


def partition_pairs(work, world_size: int) -> list[list[int]]:
    """Pairs for each rank: the pair with the most work first, each to the
    rank with the least work so far (ties to the lower rank), so the slowest
    rank's share stays close to the mean.  `work` holds one non-negative
    estimate per pair (for example its source + target points).  Each rank's
    list is in ascending pair order; together they hold every pair once.
    Deterministic: every rank computes the same partition."""
    w = np.asarray(work, dtype=np.float64)
    if w.ndim != 1 or (w < 0).any():
        raise ValueError("work: one non-negative value per pair")
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(w.shape[0]), key=lambda k: (-w[k], k))
    load = [0.0] * world_size
    parts: list[list[int]] = [[] for _ in range(world_size)]
    for k in order:
        r = min(range(world_size), key=lambda i: (load[i], i))
        parts[r].append(k)
        load[r] += float(w[k])
    return [sorted(p) for p in parts]


def gather_results(local_pairs, local_poses, local_iters, n_pairs: int, world_size: int):
    """All ranks' (pair index, pose, iterations) into full arrays, on every
    rank: poses (n_pairs, 4, 4) float64 and iterations (n_pairs,) int32.
    Raises if a pair is missing or reported twice."""
    local_pairs = [int(k) for k in local_pairs]
    local_poses = np.asarray(local_poses, dtype=np.float64).reshape(len(local_pairs), 4, 4)
    local_iters = np.asarray(local_iters, dtype=np.int32).reshape(len(local_pairs))
    if world_size > 1:
        import torch.distributed as dist
        parts = [None] * world_size
        dist.all_gather_object(parts, (local_pairs, local_poses, local_iters))
    else:
        parts = [(local_pairs, local_poses, local_iters)]
    poses = np.full((n_pairs, 4, 4), np.nan)
    iters = np.full(n_pairs, -1, np.int32)
    seen = np.zeros(n_pairs, np.int32)
    for idx, P, it in parts:
        for j, k in enumerate(idx):
            poses[k] = P[j]
            iters[k] = it[j]
            seen[k] += 1
    if not (seen == 1).all():
        raise RuntimeError(f"gathered results: {int((seen == 0).sum())} pairs missing, "
                           f"{int((seen > 1).sum())} reported twice")
    return poses, iters
