"""Pins of the oracle's descriptor validation and feature extraction.

Hand-worked descriptors (all counts powers of two, so every logarithm is an
exact integer), the variant counts of Table 1 (6 / 18 / 42 / 84 for 1..4
loops, also observed in Table 4), and invariants.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2301_03636_gb300 import workloads as W

Q = 65536


def desc(depth, trips, flops, byts, h2d, d2h, teams, threads, pf_pos, dc, pc, sched, dm):
    t = list(trips) + [1] * (4 - len(trips))
    return np.array([depth] + t + [flops, byts, h2d, d2h, teams, threads, pf_pos, dc, pc, sched, dm],
                    dtype=np.int64)


# depth 1, trip 16, flops 1, bytes 4, h2d = d2h = 1024, 1 team x 32 threads,
# 'teams distribute parallel for' on loop 0 (collapse 1), static, data mode 0.
D1 = desc(1, [16], 1, 4, 1024, 1024, 1, 32, 0, 0, 1, 0, 0)
# T = 16, FL = 16, BY = 64, MB = 2048, P = 32, D = Q = 16
D1_BASE = [1 * Q, 4 * Q, 0, 0, 0, 4 * Q, 0, 2 * Q, 4 * Q, 6 * Q, 10 * Q, 10 * Q, 11 * Q, 0, 5 * Q, 5 * Q,
           4 * Q, 4 * Q, 0, 4 * Q, 0, -2 * Q, -5 * Q, Q, 0, 0, 0, 0, 0, Q, Q, 4 * Q]
D1_LEVELS = [[4 * Q, Q, Q, 0, 4 * Q, 4 * Q, 6 * Q, 4 * Q]] + [[0] * 8] * 3

# depth 3, trips (8, 4, 2), flops 2, bytes 8, h2d 4096, d2h 0, 64 teams x 128
# threads, 'teams distribute collapse(1)' on loop 0 and 'parallel for
# collapse(2)' on loop 1, guided, data mode 1.
D3 = desc(3, [8, 4, 2], 2, 8, 4096, 0, 64, 128, 1, 1, 2, 2, 1)
# T = 64, FL = 128, BY = 512, MB = 4096, P = 8192, D = 8, Q = 4*2 = 8
D3_BASE = [3 * Q, 3 * Q, 2 * Q, 1 * Q, 0, 6 * Q, 1 * Q, 3 * Q, 7 * Q, 9 * Q, 12 * Q, 0, 12 * Q, 6 * Q, 7 * Q,
           13 * Q, 3 * Q, 3 * Q, 0, 0, 0, -2 * Q, -3 * Q, 0, 0, Q, Q, Q, Q, 2 * Q, 0, 6 * Q]
D3_LEVELS = [
    [3 * Q, Q, 0, 0, 3 * Q, 6 * Q, 6 * Q, 4 * Q],
    [2 * Q, 0, Q, Q, 5 * Q, 3 * Q, 5 * Q, 3 * Q],
    [1 * Q, 0, Q, Q, 6 * Q, 1 * Q, 4 * Q, 2 * Q],
    [0] * 8,
]


# depth 2, trips (32, 16), flops 4, bytes 16, h2d 2^20, d2h 0, 256 teams x 64
# threads, 'teams distribute parallel for collapse(2)' on loop 0 (combined:
# both loops distributed and parallel), dynamic, data mode 0.
D2 = desc(2, [32, 16], 4, 16, 1 << 20, 0, 256, 64, 0, 0, 2, 1, 0)
# T = 2^9, FL = 2^11, BY = 2^13, MB = 2^20, P = 2^14, D = Q = 32*16 = 2^9
D2_BASE = [2 * Q, 5 * Q, 4 * Q, 0, 0, 9 * Q, 2 * Q, 4 * Q, 11 * Q, 13 * Q, 20 * Q, 0, 20 * Q, 8 * Q, 6 * Q,
           14 * Q, 9 * Q, 9 * Q, 0, 1 * Q, 3 * Q, -2 * Q, -7 * Q, 0, Q, 0, 0, 0, 0, 2 * Q, Q, 9 * Q]
D2_LEVELS = [
    [5 * Q, Q, Q, Q, 5 * Q, 9 * Q, 9 * Q, 7 * Q],
    [4 * Q, Q, Q, Q, 9 * Q, 4 * Q, 8 * Q, 6 * Q],
    [0] * 8,
    [0] * 8,
]

# depth 4 (the Dslash nest shape), trips (32, 32, 32, 16), flops 1024, bytes
# 2048, h2d = d2h = 2^24, 1024 teams x 128 threads, 'teams distribute
# collapse(2)' on loops 0-1 and 'parallel for collapse(2)' on loops 2-3,
# static, data mode 1.
D4 = desc(4, [32, 32, 32, 16], 1024, 2048, 1 << 24, 1 << 24, 1024, 128, 2, 2, 2, 0, 1)
# T = 2^19, FL = 2^29, BY = 2^30, MB = 2^25, P = 2^17, D = 2^10, Q = 2^9
D4_BASE = [4 * Q, 5 * Q, 5 * Q, 5 * Q, 4 * Q, 19 * Q, 10 * Q, 11 * Q, 29 * Q, 30 * Q, 24 * Q, 24 * Q, 25 * Q,
           10 * Q, 7 * Q, 17 * Q, 10 * Q, 9 * Q, 2 * Q, 0, 2 * Q, -1 * Q, 5 * Q, Q, 0, 0, Q, 2 * Q, 2 * Q,
           2 * Q, 0, 17 * Q]
D4_LEVELS = [
    [5 * Q, Q, 0, Q, 5 * Q, 19 * Q, 16 * Q, 15 * Q],
    [5 * Q, Q, 0, Q, 10 * Q, 14 * Q, 16 * Q, 15 * Q],
    [5 * Q, 0, Q, Q, 15 * Q, 9 * Q, 16 * Q, 15 * Q],
    [4 * Q, 0, Q, Q, 19 * Q, 4 * Q, 15 * Q, 14 * Q],
]


@pytest.mark.parametrize("d,base,levels,collapsed", [(D1, D1_BASE, D1_LEVELS, 1), (D2, D2_BASE, D2_LEVELS, 2),
                                                     (D3, D3_BASE, D3_LEVELS, 3), (D4, D4_BASE, D4_LEVELS, 4)])
def test_hand_worked(d, base, levels, collapsed):
    f32, st = oracle.extract_features(d, 32)
    assert st.tolist() == [0]
    assert f32[0].tolist() == base
    f33, _ = oracle.extract_features(d, 33)   # the base features and dist_collapse + pf_collapse
    assert f33[0].tolist() == base + [collapsed * Q]
    f64, _ = oracle.extract_features(d, 64)
    assert f64[0, :32].tolist() == base
    assert f64[0, 32:].tolist() == sum(levels, [])


def test_pairwise_differences_hand_worked():
    f, _ = oracle.extract_features(D3, 128)
    f = f[0]
    b = D3_BASE
    # pair u: a = 1 + u mod 21, step s = 1 + u // 21, partner = 1 + (a - 1 + s) mod 22
    assert f[64 + 0] == b[1] - b[2] == Q
    assert f[64 + 20] == b[21] - b[22] == Q
    assert f[64 + 21] == b[1] - b[3] == 2 * Q
    assert f[64 + 63] == b[1] - b[5] == -3 * Q
    assert f[:64].tolist() == oracle.extract_features(D3, 64)[0][0].tolist()


def _count_valid(depth):
    n = 0
    for pf_pos, dc, pc, sched, dm in itertools.product(range(-1, 6), range(-1, 6), range(-1, 6),
                                                       range(-1, 4), range(-1, 3)):
        d = desc(depth, [4] * depth, 1, 1, 0, 0, 1, 1, pf_pos, dc, pc, sched, dm)
        n += int(oracle.validate(d)[0] == 0)
    return n


def test_table1_variant_counts():
    # Table 1: 1, 2, 3, 4 nested loops give 6, 18, 42, 84 variants.
    assert [_count_valid(k) for k in (1, 2, 3, 4)] == [6, 18, 42, 84]
    assert [6 * len(W.valid_variant_params(k)) for k in (1, 2, 3, 4)] == [6, 18, 42, 84]


@pytest.mark.parametrize("field,value,bit", [
    (0, 0, 1), (0, 5, 1),
    (1, 0, 2), (1, (1 << 24) + 1, 2), (4, 2, 2),
    (5, 0, 4), (6, (1 << 32) + 1, 4),
    (7, -1, 8), (8, (1 << 48) + 1, 8),
    (9, 0, 16), (10, (1 << 24) + 1, 16),
    (11, 3, 32), (12, 2, 32), (12, 0, 32), (13, 3, 32), (13, 0, 32), (14, 3, 32), (15, 2, 32),
])
def test_validation_bits(field, value, bit):
    d = D3.copy()
    d[field] = value
    feat, st = oracle.extract_features(d, 64)
    assert st[0] & bit
    if field == 0:
        assert st[0] == 1
    assert not feat.any()


@pytest.mark.parametrize("field,lo,hi,bit", [
    (1, 1, 1 << 24, 2), (2, 1, 1 << 24, 2), (3, 1, 1 << 24, 2),   # trip counts of the three loops
    (5, 1, 1 << 32, 4), (6, 1, 1 << 32, 4),                       # flops, bytes per iteration
    (7, 0, 1 << 48, 8), (8, 0, 1 << 48, 8),                       # mapped bytes each way
    (9, 1, 1 << 24, 16), (10, 1, 1 << 24, 16),                    # teams, threads
])
def test_validation_ranges_both_sides(field, lo, hi, bit):
    """Both ends of every range: the bound itself is valid, one past it is not."""
    for value, bad in ((lo - 1, True), (lo, False), (hi, False), (hi + 1, True)):
        d = D3.copy()
        d[field] = value
        st = int(oracle.validate(d)[0])
        assert bool(st & bit) == bad, (field, value, st)


def test_overflow_range_bit():
    d = desc(4, [1 << 24, 1 << 24, 1 << 2, 1], 1, 1, 0, 0, 1, 1, 0, 0, 1, 0, 0)  # T = 2^50
    assert oracle.validate(d)[0] == 64
    d = desc(2, [1 << 24, 1 << 24], 1 << 16, 1, 0, 0, 1, 1, 0, 0, 1, 0, 0)  # FL = 2^64
    assert oracle.validate(d)[0] == 64
    d = desc(2, [1 << 24, 1 << 24], 1 << 14, 1 << 14, 0, 0, 1, 1, 0, 0, 1, 0, 0)  # 2^62: allowed
    assert oracle.validate(d)[0] == 0


def test_generated_rows_valid_and_derived_logs():
    d = W.make_descriptors(5000, 77)
    f, st = oracle.extract_features(d, 64)
    assert not st.any()
    trips = d[:, 1:5].astype(object)
    T = [int(np.prod(r)) for r in trips]
    L = oracle.log2_q16(np.array(T, dtype=np.uint64))
    assert np.array_equal(f[:, 5], L)
    FL = np.array([t * int(x) for t, x in zip(T, d[:, 5])], dtype=np.uint64)
    assert np.array_equal(f[:, 8], oracle.log2_q16(FL))
    MB = (d[:, 7] + d[:, 8]).astype(np.uint64)
    assert np.array_equal(f[:, 12], oracle.log2_q16(MB))
    # schedule one-hot sums to one; flags are 0 or 1 (x 2^16)
    assert np.all(f[:, 23:26].sum(axis=1) == Q)
    assert set(np.unique(f[:, [26, 30] + [33 + 8 * i + j for i in range(4) for j in range(3)]])) <= {0, Q}


def test_row_permutation_permutes_features():
    d = W.make_descriptors(300, 3)
    perm = np.random.Generator(np.random.PCG64(1)).permutation(300)
    f, _ = oracle.extract_features(d, 128)
    fp, _ = oracle.extract_features(d[perm], 128)
    assert np.array_equal(f[perm], fp)
