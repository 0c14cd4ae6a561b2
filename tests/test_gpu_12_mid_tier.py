"""FP16 tensor-core middle tier of the near-tie re-score (advisor_rank_ex,
advisor_rank_topn_ex): the tier-1 candidates are re-extracted into a compact
FP16 image and scored on the tensor cores before the FP32 tier.  Selections
(Fig. 2: the best variant, or the top N, per kernel) must stay identical to
the FP64 oracle's; the FP16 tier sees exactly the tier-1 candidates and
passes on no more rows than it received."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2301_03636_gb300 import advisor
from paper_2301_03636_gb300 import workloads as W

pytestmark = pytest.mark.gpu

WIDE = (128, 1024, 1024, 1024, 1)
NARROW = (64, 256, 256, 256, 1)


def _setup(widths, n_kernels, seed, lo=2, hi=64, invalid_every=0):
    F = widths[0]
    off = W.make_segments(n_kernels, lo, hi, seed=seed)
    d = W.make_descriptors(int(off[-1]), seed)
    if invalid_every:
        d[::invalid_every, 5] = 0   # work 0: invalid rows, never selected
    cal = W.calibration_descriptors(16384)
    fc, sc = oracle.extract_features(cal, F)
    mu, sigma = oracle.fit_standardizer(fc, sc)
    p = W.make_weights(widths, seed)
    f, st = oracle.extract_features(d, F)
    y_ref = oracle.mlp_forward(f, widths, p, mu, sigma, status=st)
    m = advisor.Model(widths, max_rows=max(len(d), 16384), max_kernels=n_kernels)
    m.set_params(p, mu, sigma)
    fcal, scal = advisor.advisor_extract_features(torch.from_numpy(cal).cuda(), F)
    eps = {q: m.calibrate_eps(fcal, scal, q) for q in ("bf16", "fp16", "fp32")}
    if widths[1] > 256:
        m.calibrate_fp8(fcal)
        eps["fp8"] = m.calibrate_eps(fcal, scal, "fp8")
    return dict(off=off, d=d, m=m, y_ref=y_ref, eps=eps,
                dt=torch.from_numpy(d).cuda(), ot=torch.from_numpy(off).cuda())


@pytest.fixture(scope="module")
def wide():
    return _setup(WIDE, 192, 5, invalid_every=61)


@pytest.fixture(scope="module")
def narrow():
    return _setup(NARROW, 512, 12, lo=1, invalid_every=53)


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_wide_mid_tier_argmin_identical(gpu_lib, wide, precision):
    m, e = wide["m"], wide["eps"]
    ref, _ = oracle.select_best(wide["y_ref"], wide["off"])
    b0, _ = m.rank(wide["dt"], wide["ot"], precision, eps=e[precision], eps32=e["fp32"])
    c32_plain, c64_plain = m.rescore_counts()
    b, s = m.rank(wide["dt"], wide["ot"], precision, eps=e[precision], eps32=e["fp32"], eps16=e["fp16"])
    c16, c32, c64 = m.rescore_counts_ex()
    print(f"{precision}: plain FP32 {c32_plain} FP64 {c64_plain}; mid FP16 {c16} -> FP32 {c32} -> FP64 {c64}")
    assert np.array_equal(b.cpu().numpy(), ref)
    assert np.array_equal(b0.cpu().numpy(), ref)
    assert c16 == c32_plain            # the FP16 tier takes exactly the tier-1 candidates
    assert c32 <= c16
    assert m.rescore_counts() == (c32, c64)
    assert m.device_status() == 0


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
@pytest.mark.parametrize("N", [1, 5, 17])
def test_wide_mid_tier_topn_identical(gpu_lib, wide, precision, N):
    m, e = wide["m"], wide["eps"]
    ref_best, ref_score = oracle.select_topn(wide["y_ref"], wide["off"], N)
    best, score = m.rank_topn(wide["dt"], wide["ot"], N, precision, eps=e[precision], eps32=e["fp32"],
                              eps16=e["fp16"])
    c16, c32, _ = m.rescore_counts_ex()
    assert np.array_equal(best.cpu().numpy(), ref_best)
    ok = ref_best >= 0
    sc = score.cpu().numpy()
    assert np.isinf(sc[~ok]).all()
    assert np.abs(sc[ok] - ref_score[ok]).max() <= e["fp32"]
    assert c32 <= c16
    assert m.device_status() == 0


@pytest.mark.parametrize("layer_path", [0, 1])
def test_narrow_mid_tier_fused_and_layered(gpu_lib, narrow, layer_path):
    """The batched model shape: the middle tier on the fused scorer (device
    row count in the persistent kernel) and on the layer-by-layer path."""
    m, e = narrow["m"], narrow["eps"]
    cfg = m.launch_config
    cfg.layer_path = layer_path
    m.launch_config = cfg
    try:
        ref, _ = oracle.select_best(narrow["y_ref"], narrow["off"])
        b, _ = m.rank(narrow["dt"], narrow["ot"], "bf16", eps=e["bf16"], eps32=e["fp32"], eps16=e["fp16"])
        assert np.array_equal(b.cpu().numpy(), ref)
        ref_t, _ = oracle.select_topn(narrow["y_ref"], narrow["off"], 10)
        t, _ = m.rank_topn(narrow["dt"], narrow["ot"], 10, "bf16", eps=e["bf16"], eps32=e["fp32"], eps16=e["fp16"])
        assert np.array_equal(t.cpu().numpy(), ref_t)
        assert m.device_status() == 0
    finally:
        cfg.layer_path = 0
        m.launch_config = cfg


def test_mid_tier_wide_windows_many_tiles(gpu_lib, narrow):
    """A first-tier bound far above the real error sends whole kernels to the
    FP16 tier (many 128-row tiles of gathered rows, a ragged last tile); the
    FP16 tier must still cut them down and the selection stay exact."""
    m, e = narrow["m"], narrow["eps"]
    ref, _ = oracle.select_best(narrow["y_ref"], narrow["off"])
    b, _ = m.rank(narrow["dt"], narrow["ot"], "bf16", eps=50 * e["bf16"], eps32=e["fp32"], eps16=e["fp16"])
    c16, c32, _ = m.rescore_counts_ex()
    print(f"FP16 tier {c16} rows -> FP32 {c32}")
    assert np.array_equal(b.cpu().numpy(), ref)
    assert c16 > 1000
    assert c32 < c16


def test_mid_tier_without_candidates(gpu_lib, narrow):
    """eps = 0: almost no kernel has two rows in its window; the gathered
    launches see a zero (or tiny) device count and the result is the plain
    argmin's."""
    m, e = narrow["m"], narrow["eps"]
    b0, _ = m.rank(narrow["dt"], narrow["ot"], "bf16")
    b, _ = m.rank(narrow["dt"], narrow["ot"], "bf16", eps=0.0, eps32=e["fp32"], eps16=e["fp16"])
    c16, c32, _ = m.rescore_counts_ex()
    assert c32 <= c16
    if c16 == 0:
        assert torch.equal(b, b0)
    assert m.device_status() == 0


def test_mid_tier_argument_rules(gpu_lib, narrow):
    m, e = narrow["m"], narrow["eps"]
    with pytest.raises(advisor.AdvisorError) as x:
        m.rank(narrow["dt"], narrow["ot"], "fp32", eps=e["fp32"], eps32=e["fp32"], eps16=e["fp16"])
    assert x.value.code == 6   # ADVISOR_ERR_UNSUPPORTED: the first tier is already FP32
    with pytest.raises(advisor.AdvisorError) as x:
        m.rank(narrow["dt"], narrow["ot"], "bf16", eps=-1.0, eps32=e["fp32"], eps16=e["fp16"])
    assert x.value.code == 1   # ADVISOR_ERR_INVALID_ARGUMENT: no re-score, no middle tier
    b, _ = m.rank(narrow["dt"], narrow["ot"], "bf16", eps=e["bf16"], eps32=e["fp32"], eps16=-1.0)
    assert m.rescore_counts_ex()[0] == 0   # eps16 < 0: the plain tiers


def test_large_sweep_fp8_mid_tier_full_size_sampled(gpu_lib):
    """The large sweep at full size (2^20 variants of 65,536 kernels) in the
    benchmark's tiered configuration (E4M3 layers, FP16 middle tier, FP32,
    FP64): all 65,536 selections against the oracle's stored ones, and the
    oracle re-ranks a seeded sample of 256 kernels."""
    wl = W.LARGE_SWEEP
    off = wl.offsets()
    n, K = int(off[-1]), wl.n_kernels
    d = wl.descriptors()
    cal = W.calibration_descriptors(16384)
    fc, sc = oracle.extract_features(cal, 128)
    mu, sigma = oracle.fit_standardizer(fc, sc)
    p = wl.weights()
    m = advisor.Model(wl.widths, max_rows=n, max_kernels=K)
    m.set_params(p, mu, sigma)
    fcal, scal = advisor.advisor_extract_features(torch.from_numpy(cal).cuda(), 128)
    m.calibrate_fp8(fcal)
    eps8, eps16, eps32 = (m.calibrate_eps(fcal, scal, q) for q in ("fp8", "fp16", "fp32"))
    best, _ = m.rank(torch.from_numpy(d).cuda(), torch.from_numpy(off).cuda(), "fp8", eps=eps8, eps32=eps32,
                     eps16=eps16)
    b = best.cpu().numpy()
    c16, c32, c64 = m.rescore_counts_ex()
    print(f"near-tie rows: FP16 {c16} ({c16 / n:.3f}), FP32 {c32} ({c32 / n:.4f}), FP64 {c64}")
    assert c32 < c16
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "large_sweep_best.npy")
    assert np.array_equal(b, np.load(golden).astype(np.int32))   # every kernel, against the oracle's answers
    ks = np.sort(np.random.default_rng(12).choice(K, 256, replace=False))
    rows = [d[off[k]:off[k + 1]] for k in ks]
    sub_off = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    ref = oracle.rank(np.concatenate(rows), sub_off, wl.widths, p, mu, sigma)[0]
    assert np.array_equal(b[ks], ref)
    assert m.device_status() == 0
