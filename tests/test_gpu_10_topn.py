"""Top-N selection per kernel (Fig. 2: "sort codes based on cost and select
top N") on the GPU against the FP64 oracle: identical indices, in order,
with the tiered re-score; N = 1 equals the argmin path; short kernels are
padded; invalid rows are never selected; without re-score the list is the
plain sort of the precision's own scores."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03636_gb300 import advisor
from paper_2301_03636_gb300 import workloads as W

pytestmark = pytest.mark.gpu

WIDTHS = (64, 256, 256, 256, 1)


@pytest.fixture(scope="module")
def env():
    off = W.make_segments(512, 1, 64, seed=12)
    d = W.make_descriptors(int(off[-1]), 12)
    d[::53, 5] = 0          # invalid rows (work 0): never selected
    cal = W.calibration_descriptors(16384)
    fc, sc = oracle.extract_features(cal, 64)
    mu, sigma = oracle.fit_standardizer(fc, sc)
    p = W.make_weights(WIDTHS, 12)
    m = advisor.Model(WIDTHS, max_rows=max(len(d), 16384), max_kernels=512)
    m.set_params(p, mu, sigma)
    fcal, scal = advisor.advisor_extract_features(torch.from_numpy(cal).cuda(), 64)
    eps = {q: m.calibrate_eps(fcal, scal, q) for q in ("bf16", "fp16", "fp32")}
    f, st = oracle.extract_features(d, 64)
    y_ref = oracle.mlp_forward(f, WIDTHS, p, mu, sigma, status=st)
    return dict(off=off, d=d, m=m, p=p, mu=mu, sigma=sigma, eps=eps, y_ref=y_ref)


@pytest.mark.parametrize("precision", ["bf16", "fp16", "fp32"])
@pytest.mark.parametrize("N", [1, 5, 10, 84])
def test_topn_identical_to_oracle(gpu_lib, env, precision, N):
    m = env["m"]
    d, o = torch.from_numpy(env["d"]).cuda(), torch.from_numpy(env["off"]).cuda()
    best, score = m.rank_topn(d, o, N, precision, eps=env["eps"][precision], eps32=env["eps"]["fp32"])
    ref_best, ref_score = oracle.select_topn(env["y_ref"], env["off"], N)
    b, sc = best.cpu().numpy(), score.cpu().numpy()
    assert np.array_equal(b, ref_best)
    ok = ref_best >= 0
    assert np.isinf(sc[~ok]).all()
    assert np.abs(sc[ok] - ref_score[ok]).max() <= env["eps"]["fp32"]   # the deciding values are FP32 or FP64
    assert m.device_status() == 0


def test_top1_equals_argmin(gpu_lib, env):
    m = env["m"]
    d, o = torch.from_numpy(env["d"]).cuda(), torch.from_numpy(env["off"]).cuda()
    eps, eps32 = env["eps"]["bf16"], env["eps"]["fp32"]
    b1, s1 = m.rank_topn(d, o, 1, "bf16", eps=eps, eps32=eps32)
    b, s = m.rank(d, o, "bf16", eps=eps, eps32=eps32)
    assert torch.equal(b1[:, 0], b)


def test_topn_without_rescore_is_the_sort_of_the_scores(gpu_lib, env):
    m = env["m"]
    d, o = torch.from_numpy(env["d"]).cuda(), torch.from_numpy(env["off"]).cuda()
    scores = torch.empty(len(env["d"]), dtype=torch.float32, device="cuda")
    best, score = m.rank_topn(d, o, 7, "bf16", eps=-1.0, scores=scores)
    y = scores.cpu().numpy().astype(np.float64)
    ref_best, ref_score = oracle.select_topn(y, env["off"], 7)   # the definition applied to the GPU's own scores
    assert np.array_equal(best.cpu().numpy(), ref_best)
    assert np.array_equal(score.cpu().numpy(), ref_score)


def test_dslash_top10(gpu_lib, env):
    kernels = W.make_dslash_kernels(64, 29)
    v, off = advisor.advisor_enumerate_variants(torch.from_numpy(kernels).cuda())
    m = env["m"]
    best, _ = m.rank_topn(v.contiguous(), off, 10, "bf16", eps=env["eps"]["bf16"], eps32=env["eps"]["fp32"])
    ref_v, ref_off = oracle.enumerate_variants(kernels)
    ref_best, _, _ = oracle.rank_topn(ref_v, ref_off, WIDTHS, env["p"], env["mu"], env["sigma"], 10)
    assert np.array_equal(best.cpu().numpy(), ref_best)
