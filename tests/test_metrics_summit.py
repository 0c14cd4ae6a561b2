"""The metric helpers against the paper's own Summit data (Fig.
plot_variants_summit): the caption prints the maximum prediction error as
3.04 s for kernels above 45 s and 0.76 s for kernels below 2 s."""
import os

import numpy as np

from paper_2301_03636_gb300 import metrics

HERE = os.path.dirname(os.path.abspath(__file__))


def _load():
    a = np.loadtxt(os.path.join(HERE, "golden", "summit_dslash_84.txt"))
    assert a.shape == (84, 3) and a[:, 0].tolist() == list(range(1, 85))
    return a[:, 1], a[:, 2]


def test_max_errors_match_caption():
    actual, pred = _load()
    assert round(metrics.max_abs_error(pred, actual, actual > 45.0), 2) == 3.04
    assert round(metrics.max_abs_error(pred, actual, actual < 2.0), 2) == 0.76


def test_rmse_nrmse():
    actual, pred = _load()
    r = metrics.rmse(pred, actual)
    assert abs(r - np.sqrt(np.mean((pred - actual) ** 2))) < 1e-12
    assert abs(r - 0.812) < 5e-4
    n = metrics.nrmse(pred, actual)
    assert abs(n - r / (actual.max() - actual.min())) < 1e-12   # Eq. nrmse: RMSE over the range of the actual values
    assert abs(n - 0.0169) < 5e-5   # 0.812 s over the 48.07 s range of the 84 measured runtimes
    assert n < metrics.SUCCESS_NRMSE  # the paper's success criterion


def test_top_k_overlap():
    actual, pred = _load()
    assert metrics.top_k_overlap(pred, actual, 84) == 84
    assert 0 <= metrics.top_k_overlap(pred, actual, 10) <= 10
    assert metrics.top_k_overlap([3, 2, 1], [1, 2, 3], 1) == 0
