"""Sharding of a ranking job across GPUs (one process per GPU).

Every kernel's variants are scored and selected independently, so the job
splits by whole kernels with no exchange on the data path: rank r takes a
contiguous range of kernel segments whose rows are balanced by count, ranks
its shard, and the per-kernel answers are concatenated in rank order.
"""
from __future__ import annotations

import numpy as np


def shard_segments(offsets: np.ndarray, rank: int, world: int):
    """Kernel range [k_lo, k_hi) of `rank`, its row range [r_lo, r_hi) and
    the local offsets (starting at 0).  Boundaries are the kernels closest to
    equal row shares; every kernel belongs to exactly one rank."""
    offsets = np.asarray(offsets, dtype=np.int64)
    K = len(offsets) - 1
    total = int(offsets[-1])
    targets = [total * i // world for i in range(world + 1)]
    bounds = [0] + [int(np.searchsorted(offsets, t, side="left")) for t in targets[1:-1]] + [K]
    bounds = [min(max(b, 0), K) for b in bounds]
    for i in range(1, len(bounds)):               # monotone
        bounds[i] = max(bounds[i], bounds[i - 1])
    k_lo, k_hi = bounds[rank], bounds[rank + 1]
    r_lo, r_hi = int(offsets[k_lo]), int(offsets[k_hi])
    return k_lo, k_hi, r_lo, r_hi, offsets[k_lo:k_hi + 1] - r_lo
