"""Selections at the batched-scoring workload's full size (4,096 kernels with
4..64 variants each, ~140k rows, F=64, MLP 64-256-256-256-1) identical to the
FP64 oracle for every kernel, with the tensor-core scorer plus the tiered
near-tie re-score, and for the FP32 plain scorer."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03636_gb300 import advisor
from paper_2301_03636_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batched():
    wl = W.BATCHED_4096
    off = wl.offsets()
    d = wl.descriptors()
    cal = W.calibration_descriptors(65536)
    fc, sc = oracle.extract_features(cal, wl.n_features)
    mu, sigma = oracle.fit_standardizer(fc, sc)
    p = wl.weights()
    best_ref, score_ref, y_ref, _, _ = oracle.rank(d, off, wl.widths, p, mu, sigma)
    m = advisor.Model(wl.widths, max_rows=len(d), max_kernels=wl.n_kernels)
    m.set_params(p, mu, sigma)
    fcal, scal = advisor.advisor_extract_features(torch.from_numpy(cal).cuda(), wl.n_features)
    return dict(wl=wl, off=off, d=d, m=m, best_ref=best_ref, y_ref=y_ref, fcal=fcal, scal=scal)


@pytest.mark.parametrize("precision", ["bf16", "fp16", "fp32"])
def test_full_size_selection_identical(gpu_lib, batched, precision):
    m = batched["m"]
    eps = m.calibrate_eps(batched["fcal"], batched["scal"], precision)
    eps32 = m.calibrate_eps(batched["fcal"], batched["scal"], "fp32") if precision != "fp32" else eps
    d = torch.from_numpy(batched["d"]).cuda()
    o = torch.from_numpy(batched["off"]).cuda()
    scores = torch.empty(len(batched["d"]), dtype=torch.float32, device="cuda")
    best, bscore = m.rank(d, o, precision, eps=eps, eps32=eps32, scores=scores)
    b = best.cpu().numpy()
    ref = batched["best_ref"]
    y = scores.cpu().numpy().astype(np.float64)
    err = np.abs(y - batched["y_ref"])
    print(f"{precision}: eps={eps:.3e} eps32={eps32:.3e} max|dy|={err.max():.3e} mismatches={int((b != ref).sum())}")
    assert err.max() <= eps / 2 * 1.5   # the calibrated bound holds on the measured set (with slack)
    assert np.array_equal(b, ref)
    assert m.device_status() == 0
