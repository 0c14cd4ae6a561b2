"""Accuracy metrics of the cost model (Sec. 5, Experiment 3 and 4).

RMSE (Eq. rmse) is the root of the mean squared difference between predicted
and measured runtimes over the N rows; NRMSE (Eq. nrmse) divides it by the
range of the measured values.  A model with NRMSE below 0.1 counts as
successful.  Host-side numpy helpers used by the benchmark and the training
driver.
"""
from __future__ import annotations

import numpy as np

SUCCESS_NRMSE = 0.1


def rmse(pred, actual) -> float:
    pred = np.asarray(pred, dtype=np.float64)
    actual = np.asarray(actual, dtype=np.float64)
    return float(np.sqrt(np.mean((pred - actual) ** 2)))


def nrmse(pred, actual) -> float:
    actual = np.asarray(actual, dtype=np.float64)
    span = float(actual.max() - actual.min())
    return rmse(pred, actual) / span if span > 0 else float("inf")


def max_abs_error(pred, actual, mask=None) -> float:
    d = np.abs(np.asarray(pred, dtype=np.float64) - np.asarray(actual, dtype=np.float64))
    if mask is not None:
        d = d[np.asarray(mask)]
    return float(d.max()) if d.size else 0.0


def top_k_overlap(pred, actual, k: int) -> int:
    """How many of the k variants with the smallest predicted runtime are among
    the k with the smallest measured runtime (the top-N output of Fig. 2)."""
    p = set(np.argsort(np.asarray(pred), kind="stable")[:k].tolist())
    a = set(np.argsort(np.asarray(actual), kind="stable")[:k].tolist())
    return len(p & a)
