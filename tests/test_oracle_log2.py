"""Pins of the oracle's Q16.16 binary logarithm against the mathematics.

L(x) is the digit-by-digit base-2 logarithm by repeated squaring, truncated
to 16 fraction bits.  Truncation at every squaring only lowers the result, so
0 <= 65536*log2(x) - L(x) < 2 must hold for every x >= 1, L(2^k) = k*65536
exactly, and L must be non-decreasing.
"""
import math
import random

import numpy as np

import oracle


def test_zero_and_one():
    assert oracle.log2_q16([0, 1]).tolist() == [0, 0]


def test_powers_of_two_exact():
    xs = np.array([1 << k for k in range(64)], dtype=np.uint64)
    assert oracle.log2_q16(xs).tolist() == [k * 65536 for k in range(64)]


def test_exhaustive_below_2_20():
    x = np.arange(1, 1 << 20, dtype=np.uint64)
    L = oracle.log2_q16(x).astype(np.float64)
    gap = 65536.0 * np.log2(x.astype(np.float64)) - L
    assert gap.min() >= -1e-6
    assert gap.max() < 2.0
    assert np.all(np.diff(L) >= 0)


def test_random_large_values():
    rng = np.random.Generator(np.random.PCG64(11))
    x = rng.integers(1, (1 << 63) - 1, size=1_000_000, dtype=np.uint64)
    x = np.concatenate([x, (x >> rng.integers(0, 62, size=x.size).astype(np.uint64)) | np.uint64(1)])
    L = oracle.log2_q16(x).astype(np.float64)
    gap = 65536.0 * np.log2(x.astype(np.float64)) - L
    assert gap.min() >= -1e-6 and gap.max() < 2.0
    xs = np.sort(x)
    assert np.all(np.diff(oracle.log2_q16(xs).astype(np.int64)) >= 0)


def test_exact_integer_bound_on_samples():
    # 2^L <= x^65536 < 2^(L+2), i.e. L/65536 <= log2 x < (L+2)/65536, checked
    # with exact integer arithmetic: x^65536 >> L >= 1 and x^65536 >> (L+2) == 0.
    rnd = random.Random(5)
    xs = [3, 5, 7, 1000, 65535, 65537, (1 << 40) + 1] + [rnd.randrange(2, 1 << 62) for _ in range(24)]
    L = oracle.log2_q16(np.array(xs, dtype=np.uint64)).tolist()
    for x, l in zip(xs, L):
        p = x ** 65536
        assert (p >> l) >= 1, x
        assert (p >> (l + 2)) == 0, x


def test_against_float_log_small_known_values():
    # log2(3) * 65536 = 103872.3..., log2(10) * 65536 = 217706.0...
    assert oracle.log2_q16([3]).tolist()[0] in (103871, 103872)
    assert oracle.log2_q16([10]).tolist()[0] in (217705, 217706)
    assert math.floor(65536 * math.log2(3)) == 103872


def test_log_of_min_is_min_of_logs():
    """The digit-by-digit logarithm is non-decreasing, so L(min(a, b)) =
    min(L(a), L(b)) exactly (the GPU feature kernels derive L(min(T, P)) that
    way instead of computing it again)."""
    rng = np.random.default_rng(17)
    a = rng.integers(1, 2**62, 50000, dtype=np.uint64) >> rng.integers(0, 62, 50000).astype(np.uint64)
    b = rng.integers(1, 2**62, 50000, dtype=np.uint64) >> rng.integers(0, 62, 50000).astype(np.uint64)
    a = np.maximum(a, np.uint64(1))
    b = np.maximum(b, np.uint64(1))
    la, lb = oracle.log2_q16(a), oracle.log2_q16(b)
    assert np.array_equal(oracle.log2_q16(np.minimum(a, b)), np.minimum(la, lb))
    # neighbours, where a truncation could in principle reorder the values
    x = rng.integers(2**20, 2**62, 20000, dtype=np.uint64)
    assert (oracle.log2_q16(x + np.uint64(1)) >= oracle.log2_q16(x)).all()


def test_squaring_that_lands_on_two_gives_the_exact_floor():
    """0xB504F334 = 3,037,000,500 is the one 32-bit mantissa whose square,
    truncated to Q1.31, is exactly 2.0 (its square lies in
    [2^63, 2^63 + 2^31)); 2 counts as >= 2, so the first digit is 1 and the
    rest are 0.  Since log2 of it lies just above 31.5, the digit-by-digit
    result is then the exact floor of 65536 log2 x: 2^L <= x^65536 < 2^(L+1).
    The same holds for the mantissa at every binary shift."""
    m = 0xB504F334
    assert (1 << 63) <= m * m < (1 << 63) + (1 << 31)
    xs = [m << s for s in range(33)]
    L = oracle.log2_q16(np.array(xs, dtype=np.uint64)).tolist()
    assert L == [(31 + s) * 65536 + 32768 for s in range(33)]
    for x, l in ((xs[0], L[0]), (xs[32], L[32])):
        p = x ** 65536
        assert (1 << l) <= p < (1 << (l + 1))
