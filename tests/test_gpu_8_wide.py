"""Wide MLPs on the tensor cores, one launch per hidden layer (the large
sweep's 128-1024-1024-1024-1 network, Sec. 5 Exp. 3 shape family): scores
against the FP64 oracle within the bound the model's own calibration gives,
and selections after the tiered near-tie re-score identical to the oracle's
(Fig. 2: the best variant per kernel)."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2301_03636_gb300 import advisor
from paper_2301_03636_gb300 import workloads as W

pytestmark = pytest.mark.gpu

WIDE = (128, 1024, 1024, 1024, 1)
GOLDEN_LARGE_SWEEP = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "large_sweep_best.npy")


@pytest.fixture(scope="module")
def wide():
    off = W.make_segments(192, 2, 64, seed=5)
    n = int(off[-1])
    d = W.make_descriptors(n, 5)
    cal = W.calibration_descriptors(16384)
    fc, sc = oracle.extract_features(cal, 128)
    mu, sigma = oracle.fit_standardizer(fc, sc)
    p = W.make_weights(WIDE, 5)
    best_ref, _, y_ref, _, _ = oracle.rank(d, off, WIDE, p, mu, sigma)
    m = advisor.Model(WIDE, max_rows=max(n, 16384), max_kernels=192)
    m.set_params(p, mu, sigma)
    fcal, scal = advisor.advisor_extract_features(torch.from_numpy(cal).cuda(), 128)
    m.calibrate_fp8(fcal)   # static E4M3 activation scales from the calibration sample
    return dict(off=off, d=d, n=n, m=m, best_ref=best_ref, y_ref=y_ref, fcal=fcal, scal=scal)


@pytest.mark.parametrize("precision", ["bf16", "fp16", "fp8"])
def test_wide_scores_within_calibrated_bound(gpu_lib, wide, precision):
    m = wide["m"]
    d = torch.from_numpy(wide["d"]).cuda()
    f, st = advisor.advisor_extract_features(d, 128)
    y = m.score(f, st, precision).double().cpu().numpy()
    y64 = m.score_fp64(f, st).cpu().numpy()
    assert np.array_equal(y64, wide["y_ref"])            # the FP64 scorer is the oracle's value
    eps = m.calibrate_eps(wide["fcal"], wide["scal"], precision)
    err = np.abs(y - wide["y_ref"])
    print(f"{precision}: n={wide['n']} max|dy|={err.max():.4e} p99={np.quantile(err, 0.99):.4e} "
          f"eps={eps:.4e} score range {wide['y_ref'].min():.3f}..{wide['y_ref'].max():.3f}")
    assert np.isfinite(y).all()
    assert err.max() <= eps / 2 * 1.5   # eps = 2 x the max on the calibration sample


@pytest.mark.parametrize("precision", ["bf16", "fp16", "fp8"])
def test_wide_rank_selection_identical(gpu_lib, wide, precision):
    m = wide["m"]
    eps = m.calibrate_eps(wide["fcal"], wide["scal"], precision)
    eps32 = m.calibrate_eps(wide["fcal"], wide["scal"], "fp32")
    d = torch.from_numpy(wide["d"]).cuda()
    o = torch.from_numpy(wide["off"]).cuda()
    best, _ = m.rank(d, o, precision, eps=eps, eps32=eps32)
    b = best.cpu().numpy()
    c32, c64 = m.rescore_counts()
    print(f"{precision}: mismatches {(b != wide['best_ref']).sum()} of {len(b)}; re-scored {c32} FP32, {c64} FP64")
    assert np.array_equal(b, wide["best_ref"])
    assert m.device_status() == 0


def test_wide_ragged_tail_and_single_row(gpu_lib, wide):
    """Row counts that are not multiples of the 128-row tile, down to one row."""
    m = wide["m"]
    eps = m.calibrate_eps(wide["fcal"], wide["scal"], "fp16")
    for n in (1, 127, 129, 1000):
        d = torch.from_numpy(wide["d"][:n]).cuda()
        f, st = advisor.advisor_extract_features(d, 128)
        y = m.score(f, st, "fp16").double().cpu().numpy()
        err = np.abs(y - wide["y_ref"][:n])
        assert err.max() <= eps / 2 * 1.5, (n, err.max())


def test_large_sweep_full_size_sampled_kernels(gpu_lib):
    """The large sweep at full size (2^20 variants of 65,536 kernels, counts
    2..64): one rank call on the GPU over every kernel, in the launch
    configuration the benchmark uses (BF16 layers + FP32 / FP64 near-tie
    re-score).  All 65,536 selections must equal the oracle's stored ones
    (tests/golden/large_sweep_best.npy, written by the oracle), and the
    oracle re-ranks a seeded sample of 256 kernels here as well."""
    wl = W.LARGE_SWEEP
    off = wl.offsets()
    n, K = int(off[-1]), wl.n_kernels
    assert n == 1 << 20
    d = wl.descriptors()
    cal = W.calibration_descriptors(16384)
    fc, sc = oracle.extract_features(cal, 128)
    mu, sigma = oracle.fit_standardizer(fc, sc)
    p = wl.weights()
    m = advisor.Model(wl.widths, max_rows=n, max_kernels=K)
    m.set_params(p, mu, sigma)
    fcal, scal = advisor.advisor_extract_features(torch.from_numpy(cal).cuda(), 128)
    eps = m.calibrate_eps(fcal, scal, "bf16")
    eps32 = m.calibrate_eps(fcal, scal, "fp32")
    best, _ = m.rank(torch.from_numpy(d).cuda(), torch.from_numpy(off).cuda(), "bf16", eps=eps, eps32=eps32)
    b = best.cpu().numpy()
    c32, c64 = m.rescore_counts()
    print(f"near-tie rows: {c32} FP32 ({c32 / n:.4f} of all), {c64} FP64")
    golden = np.load(GOLDEN_LARGE_SWEEP).astype(np.int32)
    assert np.array_equal(b, golden)
    ks = np.sort(np.random.default_rng(11).choice(K, 256, replace=False))
    rows = [d[off[k]:off[k + 1]] for k in ks]
    sub_off = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    ref = oracle.rank(np.concatenate(rows), sub_off, wl.widths, p, mu, sigma)[0]
    assert np.array_equal(b[ks], ref)
    assert m.device_status() == 0


def test_fp8_needs_a_wide_model_and_a_calibration(gpu_lib, wide):
    """E4M3 scoring: rejected for models that fit the fused 16-bit scorer,
    before the activation scales are calibrated, and again after new
    parameters are set."""
    narrow = advisor.Model((64, 256, 256, 256, 1), max_rows=256, max_kernels=1)
    narrow.set_params(W.make_weights((64, 256, 256, 256, 1), 1), np.zeros(64), np.ones(64))
    f = torch.zeros((256, 64), dtype=torch.int32, device="cuda")
    with pytest.raises(advisor.AdvisorError) as e:
        narrow.calibrate_fp8(f)
    assert e.value.code == 6   # ADVISOR_ERR_UNSUPPORTED
    with pytest.raises(advisor.AdvisorError) as e:
        narrow.score(f, None, "fp8")
    assert e.value.code == 6
    m = advisor.Model(WIDE, max_rows=16384, max_kernels=1)
    p = W.make_weights(WIDE, 6)
    m.set_params(p, np.zeros(128), np.ones(128))
    f8 = wide["fcal"][:300]
    with pytest.raises(advisor.AdvisorError) as e:
        m.score(f8, None, "fp8")
    assert e.value.code == 1   # ADVISOR_ERR_INVALID_ARGUMENT: not calibrated
    m.calibrate_fp8(wide["fcal"])
    y = m.score(f8, None, "fp8")
    assert torch.isfinite(y).all()
    m.set_params(p, np.zeros(128), np.ones(128))   # new parameters clear the scales
    with pytest.raises(advisor.AdvisorError):
        m.score(f8, None, "fp8")
