"""Seeded test inputs shared by the GPU parity tests (inputs only, no arithmetic
of the method)."""
import numpy as np

from paper_2301_03636_gb300 import workloads as W


def edge_descriptors() -> np.ndarray:
    """Rows at and beyond every validation bound, plus depth-4 nests."""
    rows = []

    def d(depth, trips, flops, byts, h2d, d2h, teams, threads, pf, dc, pc, sched, dm):
        t = list(trips) + [1] * (4 - len(trips))
        rows.append([depth] + t + [flops, byts, h2d, d2h, teams, threads, pf, dc, pc, sched, dm])

    big = 1 << 24
    d(1, [1], 1, 1, 0, 0, 1, 1, 0, 0, 1, 0, 0)                             # all minima
    d(4, [32, 32, 32, 16], 1320, 2400, 1 << 30, 1 << 29, 80, 128, 1, 1, 3, 0, 1)   # a Wilson-Dslash-like nest
    d(4, [16, 8, 4, 2], 7, 9, 123, 456, 3, 33, 3, 2, 1, 2, 0)
    d(4, [2, 2, 2, 2], 1, 1, 1, 1, 1, 1, 2, 2, 2, 1, 1)
    d(2, [big, big], 1 << 14, 1 << 14, 1 << 48, 1 << 48, big, big, 0, 0, 2, 1, 1)   # products at 2^62
    d(3, [big, 1 << 20, 16], 1, 1, 0, 0, 1, 1, 0, 0, 3, 0, 0)                     # T = 2^48 exactly
    d(1, [(1 << 24) - 1], (1 << 32), (1 << 32) - 1, (1 << 48) - 1, 3, 1023, 1025, 0, 0, 1, 2, 0)
    # invalid rows, one per status bit
    d(0, [], 1, 1, 0, 0, 1, 1, 0, 0, 1, 0, 0)
    d(5, [2, 2, 2, 2], 1, 1, 0, 0, 1, 1, 0, 0, 1, 0, 0)
    d(2, [0, 4], 1, 1, 0, 0, 1, 1, 0, 0, 1, 0, 0)
    d(2, [big + 1, 4], 1, 1, 0, 0, 1, 1, 0, 0, 1, 0, 0)
    rows.append([1, 4, 3, 1, 1, 1, 1, 0, 0, 1, 1, 0, 0, 1, 0, 0])              # trip beyond depth != 1
    d(1, [4], 0, 1, 0, 0, 1, 1, 0, 0, 1, 0, 0)
    d(1, [4], 1, (1 << 32) + 1, 0, 0, 1, 1, 0, 0, 1, 0, 0)
    d(1, [4], 1, 1, -1, 0, 1, 1, 0, 0, 1, 0, 0)
    d(1, [4], 1, 1, 0, (1 << 48) + 1, 1, 1, 0, 0, 1, 0, 0)
    d(1, [4], 1, 1, 0, 0, 0, 1, 0, 0, 1, 0, 0)
    d(1, [4], 1, 1, 0, 0, 1, big + 1, 0, 0, 1, 0, 0)
    d(2, [4, 4], 1, 1, 0, 0, 1, 1, 2, 0, 1, 0, 0)
    d(2, [4, 4], 1, 1, 0, 0, 1, 1, 1, 0, 1, 0, 0)
    d(2, [4, 4], 1, 1, 0, 0, 1, 1, 0, 1, 1, 0, 0)
    d(2, [4, 4], 1, 1, 0, 0, 1, 1, 1, 1, 2, 0, 0)
    d(2, [4, 4], 1, 1, 0, 0, 1, 1, 0, 0, 1, 3, 0)
    d(2, [4, 4], 1, 1, 0, 0, 1, 1, 0, 0, 1, 0, 2)
    d(4, [big, big, 4, 1], 1, 1, 0, 0, 1, 1, 0, 0, 1, 0, 0)                      # T = 2^50
    d(2, [big, big], 1 << 16, 1, 0, 0, 1, 1, 0, 0, 1, 0, 0)                      # FL = 2^64
    d(2, [big, big], 1, (1 << 14) + 1, 0, 0, 1, 1, 0, 0, 1, 0, 0)               # BY > 2^62
    d(-3, [4], 1, 1, 0, 0, 1, 1, 0, 0, 1, 0, 0)
    rows.append([np.iinfo(np.int64).max] * 16)
    rows.append([np.iinfo(np.int64).min] * 16)
    return np.array(rows, dtype=np.int64)


def mixed_descriptors(n: int, seed: int) -> np.ndarray:
    """Random valid rows of depth 1..4 with the edge rows spliced in."""
    d = W.make_descriptors(n, seed, max_depth=4)
    e = edge_descriptors()
    pos = np.random.Generator(np.random.PCG64(seed)).choice(n, size=len(e), replace=False)
    d[pos] = e
    return d
