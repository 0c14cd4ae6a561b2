"""Writes large_sweep_best.npy: the FP64 oracle's best variant of every kernel
of the large sweep (2^20 variants of 65,536 kernels, F = 128, MLP
128-1024-1024-1024-1; Fig. 2: the best variant per kernel), so that the GPU
tests can check all 65,536 selections at full size, not only a sample.

Only oracle/ computes here; the inputs are the seeded synthetic generators
(paper_2301_03636_gb300.workloads, no method arithmetic).  The standardiser is
fitted by the oracle on calibration_descriptors(16384), as the tests and the
benchmark do.  Local indices are < 64, stored as int8 (-1: no finite score).

    python tests/golden/make_large_sweep_golden.py      # a few minutes on 8 cores
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2301_03636_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "large_sweep_best.npy")


def main():
    wl = W.LARGE_SWEEP
    off = wl.offsets()
    d = wl.descriptors()
    fc, sc = oracle.extract_features(W.calibration_descriptors(16384), wl.n_features)
    mu, sigma = oracle.fit_standardizer(fc, sc)
    best = oracle.rank(d, off, wl.widths, wl.weights(), mu, sigma)[0]
    assert best.max() < 64 and best.min() >= -1
    np.save(OUT, best.astype(np.int8))
    print(f"{OUT}: {len(best)} kernels")


if __name__ == "__main__":
    main()
