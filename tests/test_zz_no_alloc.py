"""advisor_score_variants_noalloc: tensor-core scoring for callers that cannot
allocate device memory (the 16-bit activations live in the library's fixed
device scratch instead of a caller workspace).  Called through the C ABI and
compared with advisor_score_variants on two calls in a row with different
inputs, plus the size limit.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2301_03636_gb300 import advisor
from paper_2301_03636_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# the tolerances the tensor-core scorer tests use (max |score - reference|)
TOL = {"bf16": 8e-2, "fp16": 1e-2}
PREC = {"bf16": advisor.BF16, "fp16": advisor.FP16}


def _noalloc(L, m, feat, status, precision, out):
    return L.advisor_score_variants_noalloc(m.handle, ctypes.c_void_p(feat.data_ptr()),
                                           ctypes.c_void_p(status.data_ptr()), feat.shape[0], PREC[precision],
                                           ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_noalloc_matches_workspace_path_twice(gpu_lib, precision):
    L = gpu_lib
    widths = (64, 256, 256, 256, 1)
    cal = W.calibration_descriptors(16384)
    fc, sc = oracle.extract_features(cal, 64)
    mu, sigma = oracle.fit_standardizer(fc, sc)
    m = advisor.Model(widths, max_rows=16384, max_kernels=1)
    m.set_params(W.make_weights(widths, 3, "he", 0.1), mu, sigma)
    # two calls in a row with different inputs, the larger first: the second, ragged call
    # (5003 rows, not a multiple of the 128-row tile) must read nothing the first one left
    # in the shared scratch; the output is poisoned with NaN before each call
    for call, (n, seed) in enumerate([(16384, 42), (5003, 41)]):
        d = torch.from_numpy(W.make_descriptors(n, seed)).cuda()
        f, st = advisor.advisor_extract_features(d, 64)
        ref = m.score(f, st, precision)
        out = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        assert _noalloc(L, m, f, st, precision, out) == advisor.OK
        torch.cuda.synchronize()
        diff = float((out - ref).abs().max().item())
        print(f"{precision} call {call}: n={n} max|noalloc - workspace| = {diff}")
        assert diff <= TOL[precision]
        assert torch.equal(out, ref)   # same kernels, same order: identical bits


def test_noalloc_rejects_sizes_beyond_scratch(gpu_lib):
    L = gpu_lib
    widths = (32, 128, 128, 1)
    m = advisor.Model(widths, max_rows=64, max_kernels=1)
    m.set_params(W.make_weights(widths, 1), np.zeros(32), np.ones(32))
    f = torch.zeros((16385, 32), dtype=torch.int32, device="cuda")
    st = torch.zeros(16385, dtype=torch.uint8, device="cuda")
    out = torch.zeros(16385, dtype=torch.float32, device="cuda")
    assert _noalloc(L, m, f, st, "bf16", out) == 3          # ADVISOR_ERR_OUT_OF_MEMORY, nothing enqueued
    with pytest.raises(advisor.AdvisorError):
        m.score_noalloc(f, st, "bf16")
    assert L.advisor_score_variants_noalloc(m.handle, ctypes.c_void_p(f.data_ptr()), None, 10, advisor.FP32,
                                            ctypes.c_void_p(out.data_ptr()), None) == 6   # unsupported precision
