"""Failure detection on the GPU without a fault: a bounded device wait that
can never complete (a barrier nothing arrives at) gives up after its limit,
the host reads ADVISOR_ERR_TIMEOUT from the model's status word, and the same
model then ranks correctly (the context stays usable)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03636_gb300 import advisor
from paper_2301_03636_gb300 import workloads as W

pytestmark = pytest.mark.gpu

WIDTHS = (32, 128, 128, 1)
ADVISOR_ERR_INVALID_ARGUMENT = 1
ADVISOR_ERR_TIMEOUT = 5


def test_bounded_wait_runs_out_and_reports_timeout(gpu_lib):
    off = W.make_segments(64, 2, 16, seed=21)
    n = int(off[-1])
    d = W.make_descriptors(n, 21)
    cal = W.calibration_descriptors(4096)
    fc, sc = oracle.extract_features(cal, 32)
    mu, sigma = oracle.fit_standardizer(fc, sc)
    p = W.make_weights(WIDTHS, 21)
    ref = oracle.rank(d, off, WIDTHS, p, mu, sigma)[0]
    m = advisor.Model(WIDTHS, max_rows=max(n, 4096), max_kernels=64)
    m.set_params(p, mu, sigma)
    fcal, scal = advisor.advisor_extract_features(torch.from_numpy(cal).cuda(), 32)
    eps, eps32 = m.calibrate_eps(fcal, scal, "bf16"), m.calibrate_eps(fcal, scal, "fp32")
    assert m.device_status() == 0

    m.check_wait_timeout(1_000_000)   # 1 ms
    assert m.device_status() == ADVISOR_ERR_TIMEOUT
    assert m.device_status() == 0      # read and cleared

    best, _ = m.rank(torch.from_numpy(d).cuda(), torch.from_numpy(off).cuda(), "bf16", eps=eps, eps32=eps32)
    assert np.array_equal(best.cpu().numpy(), ref)
    assert m.device_status() == 0

    for bad in (10, 2_000_000_000):   # outside 1 us .. 1 s
        with pytest.raises(advisor.AdvisorError) as e:
            m.check_wait_timeout(bad)
        assert e.value.code == ADVISOR_ERR_INVALID_ARGUMENT
