"""Measurement helpers behind the benchmark's rooflines: the measured FP32
FMA rate of the CUDA cores is plausible for the part (152 SMs x 128 FP32
lanes at 1-2.1 GHz: 39-82 TFLOP/s), and the argmin that the benchmark times
at 2^26 rows is the plain segmented argmin (lowest index on ties).  Many
kernels (>= 32,768) take the lane-per-kernel form of the first selection
tier; its selections, with and without the near-tie re-score, must equal
the oracle's (Fig. 2: the best variant per kernel)."""
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
    rows, K = 1 << 21, (1 << 21) // 34
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


def test_many_kernels_lane_form_identical_to_oracle(gpu_lib):
    """40,000 kernels of 0..40 variants, every 97th kernel 150 variants (the
    whole-warp fallback for long kernels), invalid rows: rank with the
    re-score (and with the FP16 tier) against the FP64 oracle."""
    import oracle
    widths = (32, 128, 128, 1)
    K = 40000
    rng = np.random.default_rng(41)
    counts = rng.integers(0, 41, size=K)
    counts[::97] = 150
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    n = int(off[-1])
    d = W.make_descriptors(n, 41)
    d[::89, 5] = 0   # invalid rows (work 0)
    cal = W.calibration_descriptors(16384)
    fc, sc = oracle.extract_features(cal, 32)
    mu, sigma = oracle.fit_standardizer(fc, sc)
    p = W.make_weights(widths, 41)
    ref, _, y_ref, _, _ = oracle.rank(d, off, widths, p, mu, sigma)
    m = advisor.Model(widths, max_rows=n, max_kernels=K)
    m.set_params(p, mu, sigma)
    fcal, scal = advisor.advisor_extract_features(torch.from_numpy(cal).cuda(), 32)
    eps = {q: m.calibrate_eps(fcal, scal, q) for q in ("bf16", "fp16", "fp32")}
    dt, ot = torch.from_numpy(d).cuda(), torch.from_numpy(off).cuda()
    b, _ = m.rank(dt, ot, "bf16", eps=eps["bf16"], eps32=eps["fp32"])
    assert np.array_equal(b.cpu().numpy(), ref)
    b16, _ = m.rank(dt, ot, "bf16", eps=eps["bf16"], eps32=eps["fp32"], eps16=eps["fp16"])
    assert np.array_equal(b16.cpu().numpy(), ref)
    # without re-score: the argmin of the BF16 scores themselves (first minimum, never +inf)
    scores = torch.empty(n, dtype=torch.float32, device="cuda")
    b0, s0 = m.rank(dt, ot, "bf16", scores=scores)
    y = scores.cpu().numpy()
    exp = np.full(K, -1)
    for k in range(K):
        seg = y[off[k]:off[k + 1]]
        if len(seg) and np.isfinite(seg).any():
            exp[k] = int(np.argmin(np.where(np.isfinite(seg), seg, np.inf)))
    assert np.array_equal(b0.cpu().numpy(), exp)
    assert (exp[counts == 0] == -1).all()
    assert m.device_status() == 0


def test_descriptors_in_pinned_host_memory(gpu_lib):
    """advisor_rank and a plan reading the descriptors straight from
    page-locked host memory give the same selections as from device memory."""
    widths = (64, 256, 256, 256, 1)
    off = W.make_segments(300, 4, 64, seed=31)
    n = int(off[-1])
    d = W.make_descriptors(n, 31)
    m = advisor.Model(widths, max_rows=n, max_kernels=300)
    m.set_params(W.make_weights(widths, 31), np.zeros(64), np.full(64, 8.0))
    dd, ot = torch.from_numpy(d).cuda(), torch.from_numpy(off).cuda()
    dh = torch.from_numpy(d).pin_memory()
    for eps in (-1.0, 0.05):
        b_dev, s_dev = m.rank(dd, ot, "bf16", eps=eps, eps32=1e-4)
        b_host, s_host = m.rank(dh, ot, "bf16", eps=eps, eps32=1e-4)
        assert torch.equal(b_dev, b_host) and torch.equal(s_dev, s_host)
    plan = m.plan_rank(dh, ot, "bf16", 0.05, 1e-4)
    b_plan, s_plan = plan.launch()
    torch.cuda.synchronize()
    assert torch.equal(b_plan, b_dev) and torch.equal(s_plan, s_dev)


@pytest.mark.parametrize("which", ["desc", "offsets", "best", "best_score"])
def test_pageable_host_pointers_rejected(gpu_lib, which):
    """A descriptor, offset or answer pointer the device cannot access is
    refused before any launch."""
    widths = (32, 16, 1)
    m = advisor.Model(widths, max_rows=64, max_kernels=1)
    m.set_params(W.make_weights(widths, 1), np.zeros(32), np.ones(32))
    args = {"desc": torch.from_numpy(W.make_descriptors(64, 1)).cuda(),
            "offsets": torch.tensor([0, 64], dtype=torch.int64, device="cuda"),
            "best": torch.empty(1, dtype=torch.int32, device="cuda"),
            "best_score": torch.empty(1, dtype=torch.float64, device="cuda")}
    args[which] = args[which].cpu()                           # ordinary (pageable) host memory
    with pytest.raises(advisor.AdvisorError) as e:
        m.rank(args["desc"], args["offsets"], "bf16", best=args["best"], best_score=args["best_score"])
    assert e.value.code == 1


def test_pinned_host_offsets_and_answers(gpu_lib):
    """Descriptors and offsets read from, and answers written to, page-locked
    host memory (the serving pipelines' form): the same answers as with
    device buffers."""
    widths = (32, 128, 128, 1)
    off = W.make_segments(100, 4, 64, seed=8)
    n = int(off[-1])
    d = W.make_descriptors(n, 8)
    m = advisor.Model(widths, max_rows=n, max_kernels=100)
    m.set_params(W.make_weights(widths, 8), np.zeros(32), np.full(32, 8.0))
    b_dev, s_dev = m.rank(torch.from_numpy(d).cuda(), torch.from_numpy(off).cuda(), "bf16", 0.05, 1e-4)
    hb = torch.empty(100, dtype=torch.int32).pin_memory()
    hs = torch.empty(100, dtype=torch.float64).pin_memory()
    m.rank(torch.from_numpy(d).pin_memory(), torch.from_numpy(off).pin_memory(), "bf16", 0.05, 1e-4,
           best=hb, best_score=hs)
    torch.cuda.synchronize()
    assert torch.equal(hb, b_dev.cpu()) and torch.equal(hs, s_dev.cpu())


@pytest.mark.parametrize("n_stages", [1, 3, 8])
def test_staged_copy_rank_equals_rank(gpu_lib, n_stages):
    """advisor_rank_staged (pinned host descriptors copied in chunks that
    overlap the scoring) and its plan select exactly what advisor_rank
    selects on the same descriptors in device memory."""
    widths = (64, 256, 256, 256, 1)
    off = W.make_segments(500, 4, 64, seed=33)
    n = int(off[-1])
    d = W.make_descriptors(n, 33)
    m = advisor.Model(widths, max_rows=n, max_kernels=500)
    m.set_params(W.make_weights(widths, 33), np.zeros(64), np.full(64, 8.0))
    dd, ot = torch.from_numpy(d).cuda(), torch.from_numpy(off).cuda()
    dh = torch.from_numpy(d).pin_memory()
    for prec, eps in (("bf16", 0.05), ("fp32", 1e-3), ("bf16", -1.0)):
        s_ref = torch.empty(n, device="cuda")
        s_stg = torch.empty(n, device="cuda")
        b_ref, bs_ref = m.rank(dd, ot, prec, eps=eps, eps32=1e-4, scores=s_ref)
        stage = torch.zeros_like(dd)
        b, bs = m.rank_staged(dh, stage, ot, prec, eps=eps, eps32=1e-4, n_stages=n_stages, scores=s_stg)
        torch.cuda.synchronize()
        assert torch.equal(stage, dd)
        assert torch.equal(s_stg, s_ref) and torch.equal(b, b_ref) and torch.equal(bs, bs_ref)
    stage = torch.zeros_like(dd)
    plan = m.plan_rank_staged(dh, stage, ot, "bf16", 0.05, 1e-4, n_stages=n_stages)
    b_plan, _ = plan.launch()
    torch.cuda.synchronize()
    b_ref, _ = m.rank(dd, ot, "bf16", eps=0.05, eps32=1e-4)
    assert torch.equal(b_plan, b_ref)


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_staged_copy_rank_wide_model(gpu_lib, precision):
    """The staged copy-in on a model scored layer by layer (hidden width 1024),
    including E4M3 layers: the same selections as advisor_rank."""
    widths = (128, 1024, 1024, 1024, 1)
    off = W.make_segments(96, 2, 64, seed=35)
    n = int(off[-1])
    d = W.make_descriptors(n, 35)
    m = advisor.Model(widths, max_rows=max(n, 16384), max_kernels=96)
    cal = torch.from_numpy(W.calibration_descriptors(16384)).cuda()
    fcal, scal = advisor.advisor_extract_features(cal, 128)
    mu, sg = advisor.advisor_fit_standardizer(fcal, scal)
    m.set_params(W.make_weights(widths, 35), mu, sg)
    m.calibrate_fp8(fcal)
    eps, eps32 = m.calibrate_eps(fcal, scal, precision), m.calibrate_eps(fcal, scal, "fp32")
    dd, ot = torch.from_numpy(d).cuda(), torch.from_numpy(off).cuda()
    b_ref, s_ref = m.rank(dd, ot, precision, eps=eps, eps32=eps32)
    stage = torch.zeros_like(dd)
    b, s = m.rank_staged(torch.from_numpy(d).pin_memory(), stage, ot, precision, eps=eps, eps32=eps32, n_stages=5)
    torch.cuda.synchronize()
    assert torch.equal(b, b_ref) and torch.equal(s, s_ref)
    assert m.device_status() == 0
