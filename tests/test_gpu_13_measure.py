"""Measurement helpers behind the benchmark's rooflines: the measured FP32
FMA rate of the CUDA cores is plausible for the part (152 SMs x 128 FP32
lanes at 1-2.1 GHz: 39-82 TFLOP/s), and the argmin that the benchmark times
at 2^26 rows is the plain segmented argmin (lowest index on ties)."""
import numpy as np
import pytest
import torch

from paper_2301_03636_gb300 import advisor
from paper_2301_03636_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_fp32_fma_peak_plausible(gpu_lib):
    t = advisor.advisor_measure_fp32_fma_peak()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    print(f"FP32 FMA peak {t:.1f} TFLOP/s on {sms} SMs")
    assert 2 * 128 * sms * 0.8e9 / 1e12 < t < 2 * 128 * sms * 2.2e9 / 1e12


def test_select_without_rescore_is_segmented_argmin(gpu_lib):
    rows, K = 1 << 20, (1 << 20) // 34
    off = W.make_segments(K, 4, 64, seed=78, total=rows)
    g = torch.Generator().manual_seed(3)
    s = torch.randint(0, 1000, (rows,), generator=g).float()   # many exact ties
    m = advisor.Model((32, 16, 1), max_rows=rows, max_kernels=K)
    m.set_params(W.make_weights((32, 16, 1), 1), np.zeros(32), np.ones(32))
    best, score = m.select(s.cuda(), torch.from_numpy(off).cuda())
    sn = s.numpy()
    ref = np.array([int(np.argmin(sn[off[k]:off[k + 1]])) for k in range(K)])   # first minimum
    assert np.array_equal(best.cpu().numpy(), ref)
    assert np.array_equal(score.cpu().numpy(), np.array([sn[off[k] + ref[k]] for k in range(K)]))
