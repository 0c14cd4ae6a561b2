"""a3-a7 on the GPU against the FP64 oracle: the FP32 plain scorer within its
rounding tolerance, the FP64 scorer bit-identical, and the per-kernel
selection (argmin, lowest index on ties) identical, including the near-tie
re-score, empty / single-row / all-invalid kernels and malformed offsets."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03636_gb300 import advisor
from paper_2301_03636_gb300 import workloads as W
from tests._cases import mixed_descriptors

pytestmark = pytest.mark.gpu

# FP32 with FP32 accumulation over <= 1,024 terms per layer: |y - y64| stays
# below ~1e-5 relative; the bound below leaves over a decade of margin.
FP32_ATOL, FP32_RTOL = 2e-4, 2e-4


def setup_model(widths, n_rows, n_kernels, seed, bias_scale=0.2, max_depth=3):
    cal = W.calibration_descriptors(16384)
    fc, sc = oracle.extract_features(cal, widths[0])
    mu, sigma = oracle.fit_standardizer(fc, sc)
    params = W.make_weights(widths, seed, "he", bias_scale)
    m = advisor.Model(widths, max_rows=max(n_rows, 1), max_kernels=max(n_kernels, 1))
    m.set_params(params, mu, sigma)
    return m, params, mu, sigma


@pytest.mark.parametrize("widths,n", [((32, 128, 128, 1), 512), ((64, 256, 256, 256, 1), 3001),
                                      ((128, 96, 200, 1), 777), ((32, 33, 66, 132, 66, 33, 1), 1000),
                                      # wider than 256 (up to the library's 1,024): the 16-row
                                      # scorer with a full or a partial 1,024-column block
                                      ((128, 1024, 1024, 1024, 1), 1000), ((64, 600, 300, 1), 777),
                                      ((32, 1000, 64, 1), 333)])
def test_fp32_and_fp64_scores(gpu_lib, widths, n):
    m, p, mu, sg = setup_model(widths, n, 1, 11)
    d = mixed_descriptors(n, 77 + n)
    f_ref, st_ref = oracle.extract_features(d, widths[0])
    y_ref = oracle.mlp_forward(f_ref, widths, p, mu, sg, st_ref)
    f, st = advisor.advisor_extract_features(torch.from_numpy(d).cuda(), widths[0])
    y32 = m.score(f, st, "fp32").cpu().numpy().astype(np.float64)
    y64 = m.score_fp64(f, st).cpu().numpy()
    ok = st_ref == 0
    assert np.all(np.isinf(y32[~ok])) and np.all(np.isinf(y64[~ok]))
    assert np.allclose(y32[ok], y_ref[ok], atol=FP32_ATOL, rtol=FP32_RTOL)
    assert np.array_equal(y64, y_ref)  # same summation order, IEEE rounding: identical bits


def _segments(n_kernels, lo, hi, seed):
    return W.make_segments(n_kernels, lo, hi, seed)


def test_select_plain_argmin_matches_oracle(gpu_lib):
    rng = np.random.Generator(np.random.PCG64(2))
    counts = rng.integers(0, 30, size=300)
    counts[[0, 5, 17]] = 0
    counts[[1, 9]] = 1
    off = W.counts_to_offsets(counts)
    n = int(off[-1])
    m, p, mu, sg = setup_model((32, 128, 128, 1), n, 300, 3)
    y = rng.integers(-3, 4, size=n).astype(np.float32)  # many exact ties
    y[rng.choice(n, 40, replace=False)] = np.inf
    y[rng.choice(n, 10, replace=False)] = np.nan
    y[off[20]:off[21]] = np.inf                          # a kernel with no finite score
    y[y == 0] = -0.0 if rng.random() < 0.5 else 0.0
    best_ref, score_ref = oracle.select_best(y.astype(np.float64), off)
    best, score = m.select(torch.from_numpy(y).cuda(), torch.from_numpy(off).cuda())
    assert np.array_equal(best.cpu().numpy(), best_ref)
    s = score.cpu().numpy()
    fin = best_ref >= 0
    assert np.array_equal(s[fin], score_ref[fin]) and np.all(np.isinf(s[~fin]))


@pytest.mark.parametrize("precision", ["fp32"])
def test_plain_method_full_path(gpu_lib, precision):
    """64 kernels x 8 variants, F=32, MLP 32-128-128-1 (He init), FP32 plain
    scorer with the near-tie re-score: selections identical to the oracle."""
    wl = W.PLAIN_FP32_512
    off = wl.offsets()
    d = wl.descriptors()
    m, p, mu, sg = setup_model(wl.widths, len(d), wl.n_kernels, wl.seed, bias_scale=0.0)
    best_ref, score_ref, y_ref, _, _ = oracle.rank(d, off, wl.widths, p, mu, sg)
    dt, ot = torch.from_numpy(d).cuda(), torch.from_numpy(off).cuda()
    scores = torch.empty(len(d), dtype=torch.float32, device="cuda")
    best, score = m.rank(dt, ot, precision, eps=1e-4, eps32=1e-4, scores=scores)
    assert np.array_equal(best.cpu().numpy(), best_ref)
    assert np.allclose(scores.cpu().numpy(), y_ref, atol=FP32_ATOL, rtol=FP32_RTOL)
    # without re-score the FP32 argmin may differ only where the FP64 values nearly tie
    b0, _ = m.rank(dt, ot, precision)
    diff = np.nonzero(b0.cpu().numpy() != best_ref)[0]
    for k in diff:
        seg = y_ref[off[k]:off[k + 1]]
        assert abs(seg[b0.cpu().numpy()[k]] - seg[best_ref[k]]) < 1e-4


def test_exact_ties_resolved_by_fp64_to_lowest_index(gpu_lib):
    widths = (64, 256, 256, 256, 1)
    base = W.make_descriptors(200, 9)
    rng = np.random.Generator(np.random.PCG64(4))
    # each kernel: a few random rows plus two or three copies of one row
    rows, counts = [], []
    for k in range(60):
        c = int(rng.integers(2, 9))
        seg = base[rng.choice(200, size=c, replace=False)].copy()
        dup = int(rng.integers(0, c))
        for j in rng.choice(c, size=int(rng.integers(1, 3)), replace=False):
            seg[j] = seg[dup]
        rows.append(seg)
        counts.append(c)
    d = np.concatenate(rows)
    off = W.counts_to_offsets(np.array(counts))
    m, p, mu, sg = setup_model(widths, len(d), 60, 5)
    best_ref, _, _, _, _ = oracle.rank(d, off, widths, p, mu, sg)
    best, _ = m.rank(torch.from_numpy(d).cuda(), torch.from_numpy(off).cuda(), "fp32", eps=1e-3, eps32=1e-4)
    assert np.array_equal(best.cpu().numpy(), best_ref)


def test_invalid_and_empty_kernels(gpu_lib):
    widths = (32, 128, 128, 1)
    d = mixed_descriptors(400, 8)
    counts = np.array([0, 1, 30, 0, 100, 269])
    off = W.counts_to_offsets(counts)
    d[1:31] = np.iinfo(np.int64).min  # kernel 2: only invalid rows
    m, p, mu, sg = setup_model(widths, len(d), len(counts), 7)
    best_ref, _, _, _, st = oracle.rank(d, off, widths, p, mu, sg)
    best, score = m.rank(torch.from_numpy(d).cuda(), torch.from_numpy(off).cuda(), "fp32", eps=1e-3, eps32=1e-4)
    b = best.cpu().numpy()
    assert np.array_equal(b, best_ref)
    assert b[0] == -1 and b[2] == -1 and b[3] == -1 and b[1] == 0
    assert np.isinf(score.cpu().numpy()[[0, 2, 3]]).all()


def test_malformed_offsets_report_status(gpu_lib):
    m, _, _, _ = setup_model((32, 128, 128, 1), 100, 4, 1)
    y = torch.zeros(100, dtype=torch.float32, device="cuda")
    off = torch.tensor([0, 50, 40, 100, 130], dtype=torch.int64, device="cuda")
    best, _ = m.select(y, off)
    assert m.device_status() == 7
    b = best.cpu().numpy()
    assert b[1] == -1 and b[3] == -1 and b[0] == 0
    assert m.device_status() == 0  # cleared by the read
