"""Splitting a decryption batch over GPUs (one process per GPU).

Ciphertexts are independent, so a batch shards with no exchange: each rank
decrypts its own slice and only the host gathers m if it wants it.  These
helpers are host logic only; the kernels see a plain per-rank batch.
"""
from __future__ import annotations

import numpy as np


def shard_range(count: int, world: int, rank: int):
    """[start, end) of rank's contiguous slice; slice sizes differ by <= 1."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(int(count), world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def shard_mixed(levels, world: int, rank: int) -> np.ndarray:
    """Item indices of rank for a mixed-level list: every level is split
    evenly, so each rank gets the same work (the levels cost differently)."""
    levels = np.asarray(levels)
    out = []
    for lvl in np.unique(levels):
        idx = np.nonzero(levels == lvl)[0]
        s, e = shard_range(idx.size, world, rank)
        out.append(idx[s:e])
    return np.sort(np.concatenate(out)) if out else np.zeros(0, np.int64)
