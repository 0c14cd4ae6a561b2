"""Batching under a CUDA graph: advisor_rank captured once into a plan and
replayed, the autotuner over launch shapes, and the launch shapes themselves.

Every launch configuration must give bit-identical outputs (scores, indices,
decided values); a replay must read the current contents of its input
buffers; selections stay identical to the FP64 oracle (Fig. 2: every
variant scored, the best one per kernel selected)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03636_gb300 import advisor
from paper_2301_03636_gb300 import workloads as W

pytestmark = pytest.mark.gpu

WIDTHS = (64, 256, 256, 256, 1)
N_KERNELS = 1024


@pytest.fixture(scope="module")
def setup():
    off = W.make_segments(N_KERNELS, 4, 64, seed=7)
    n = int(off[-1])
    d_a = W.make_descriptors(n, 7)
    d_b = W.make_descriptors(n, 8)
    cal = W.calibration_descriptors(16384)
    fc, sc = oracle.extract_features(cal, 64)
    mu, sigma = oracle.fit_standardizer(fc, sc)
    p = W.make_weights(WIDTHS, 2)
    ref_a = oracle.rank(d_a, off, WIDTHS, p, mu, sigma)[0]
    ref_b = oracle.rank(d_b, off, WIDTHS, p, mu, sigma)[0]
    m = advisor.Model(WIDTHS, max_rows=n, max_kernels=N_KERNELS)
    m.set_params(p, mu, sigma)
    fcal, scal = advisor.advisor_extract_features(torch.from_numpy(cal).cuda(), 64)
    eps = {pr: m.calibrate_eps(fcal, scal, pr) for pr in ("bf16", "fp16", "fp32")}
    return dict(off=off, n=n, d_a=d_a, d_b=d_b, ref_a=ref_a, ref_b=ref_b, m=m, eps=eps)


def _direct(m, d, o, precision, eps, eps32):
    scores = torch.empty(d.shape[0], dtype=torch.float32, device="cuda")
    status = torch.empty(d.shape[0], dtype=torch.uint8, device="cuda")
    best, bs = m.rank(d, o, precision, eps=eps, eps32=eps32, scores=scores, status=status)
    torch.cuda.synchronize()
    return best.clone(), bs.clone(), scores, status


CONFIGS = [
    dict(extract_block=128, tc_ctas=0, list_blocks_per_sm=1, list_chunk_kb=32, select_block=256, layer_path=0),  # default
    dict(extract_block=64, tc_ctas=0, list_blocks_per_sm=1, list_chunk_kb=32, select_block=256),
    dict(extract_block=256, tc_ctas=37, list_blocks_per_sm=2, list_chunk_kb=16, select_block=128),
    dict(extract_block=128, tc_ctas=1, list_blocks_per_sm=1, list_chunk_kb=16, select_block=128),
    dict(extract_block=256, tc_ctas=100000, list_blocks_per_sm=2, list_chunk_kb=32, select_block=256),
]


def _cfg(**kw):
    c = advisor.LaunchConfig()
    for k, v in kw.items():
        setattr(c, k, v)
    return c


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_every_launch_config_gives_identical_bits(gpu_lib, setup, precision):
    m = setup["m"]
    d = torch.from_numpy(setup["d_a"]).cuda()
    o = torch.from_numpy(setup["off"]).cuda()
    eps, eps32 = setup["eps"][precision], setup["eps"]["fp32"]
    base = None
    try:
        for kw in CONFIGS:
            m.launch_config = _cfg(**kw)
            got = _direct(m, d, o, precision, eps, eps32)
            if base is None:
                base = got
                assert np.array_equal(got[0].cpu().numpy(), setup["ref_a"])
                continue
            for a, b in zip(got, base):
                assert torch.equal(a, b), kw
    finally:
        m.launch_config = _cfg(**CONFIGS[0])
    assert m.device_status() == 0


def test_invalid_launch_config_rejected(gpu_lib, setup):
    m = setup["m"]
    before = m.launch_config.as_dict()
    for bad in (dict(extract_block=96), dict(list_blocks_per_sm=3), dict(list_chunk_kb=64), dict(select_block=64),
                dict(tc_ctas=-1), dict(layer_path=2)):
        kw = dict(CONFIGS[0])
        kw.update(bad)
        with pytest.raises(advisor.AdvisorError):
            m.launch_config = _cfg(**kw)
        assert m.launch_config.as_dict() == before


def test_plan_replays_match_direct_and_read_refilled_inputs(gpu_lib, setup):
    m = setup["m"]
    eps, eps32 = setup["eps"]["bf16"], setup["eps"]["fp32"]
    d = torch.from_numpy(setup["d_a"]).cuda()
    o = torch.from_numpy(setup["off"]).cuda()
    direct_a = _direct(m, d, o, "bf16", eps, eps32)
    counts_a = m.rescore_counts()
    assert counts_a[0] > 0   # near ties exist on this workload
    plan = m.plan_rank(d, o, "bf16", eps, eps32, autotune=False)
    info = plan.info()
    assert info["kernels_per_replay"] == 6   # extract, scorer, tier 1, FP32, tier 2, FP64 (+ final selection)
    assert info["replay_us"] == 0.0
    n0 = advisor.launch_count()
    for _ in range(3):
        plan.launch()
    torch.cuda.synchronize()
    assert advisor.launch_count() - n0 == 3 * info["kernels_per_replay"]
    for a, b in zip((plan.best, plan.best_score, plan.scores, plan.status), direct_a):
        assert torch.equal(a, b)
    assert m.rescore_counts() == counts_a   # a replay leaves the tier counts the direct call leaves
    # refill the bound descriptor buffer in place: the next replay ranks the new rows
    d.copy_(torch.from_numpy(setup["d_b"]).cuda())
    plan.launch()
    torch.cuda.synchronize()
    assert np.array_equal(plan.best.cpu().numpy(), setup["ref_b"])
    direct_b = _direct(m, d, o, "bf16", eps, eps32)
    for a, b in zip((plan.best, plan.best_score, plan.scores, plan.status), direct_b):
        assert torch.equal(a, b)
    plan.close()
    assert m.device_status() == 0


def test_autotuned_plan(gpu_lib, setup):
    m = setup["m"]
    eps, eps32 = setup["eps"]["bf16"], setup["eps"]["fp32"]
    d = torch.from_numpy(setup["d_a"]).cuda()
    o = torch.from_numpy(setup["off"]).cuda()
    before = m.launch_config.as_dict()
    direct = _direct(m, d, o, "bf16", eps, eps32)
    plan = m.plan_rank(d, o, "bf16", eps, eps32, autotune=True)
    info = plan.info()
    print("autotuned:", info)
    assert m.launch_config.as_dict() == before          # the model's own shapes are untouched
    assert info["replay_us"] > 0.0
    c = info["config"]
    assert c["extract_block"] in (64, 128, 256) and c["select_block"] in (128, 256) and c["layer_path"] in (0, 1)
    assert (c["list_blocks_per_sm"], c["list_chunk_kb"]) in ((1, 32), (2, 16), (1, 16))
    plan.launch()
    torch.cuda.synchronize()
    assert np.array_equal(plan.best.cpu().numpy(), setup["ref_a"])
    assert torch.equal(plan.status, direct[3])
    if c["layer_path"] == 0:   # the same kernels as the direct call: identical bits
        for a, b in zip((plan.best, plan.best_score, plan.scores), direct):
            assert torch.equal(a, b)
    else:                      # another accumulation order: within the calibrated bound
        assert float((plan.scores - direct[2]).abs().max()) <= eps
    plan.close()


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_layer_path_on_a_fused_model(gpu_lib, setup, precision):
    """The layer-by-layer scorer run on a model the fused kernel also covers:
    selections identical to the oracle, scores within the calibrated bound of
    the fused kernel's."""
    m = setup["m"]
    eps, eps32 = setup["eps"][precision], setup["eps"]["fp32"]
    d = torch.from_numpy(setup["d_a"]).cuda()
    o = torch.from_numpy(setup["off"]).cuda()
    fused = _direct(m, d, o, precision, eps, eps32)
    try:
        m.launch_config = _cfg(**dict(CONFIGS[0], layer_path=1))
        layered = _direct(m, d, o, precision, eps, eps32)
    finally:
        m.launch_config = _cfg(**CONFIGS[0])
    assert np.array_equal(layered[0].cpu().numpy(), setup["ref_a"])
    assert float((layered[2] - fused[2]).abs().max()) <= eps
    assert m.device_status() == 0


def test_plan_rejects_what_rank_rejects(gpu_lib, setup):
    m = setup["m"]
    d = torch.from_numpy(setup["d_a"]).cuda()
    too_many = torch.zeros(N_KERNELS + 2, dtype=torch.int64, device="cuda")   # more kernels than the workspace holds
    with pytest.raises(advisor.AdvisorError) as e:
        m.plan_rank(d, too_many, "bf16", 0.1, 0.01)
    assert e.value.code == 3   # ADVISOR_ERR_OUT_OF_MEMORY
    with pytest.raises(advisor.AdvisorError):
        m.plan_rank(d, torch.from_numpy(setup["off"]).cuda(), "bf16", 0.1, -1.0)   # eps32 < 0 with re-score on


def _direct_ex(m, d, o, precision, eps, eps16, eps32):
    scores = torch.empty(d.shape[0], dtype=torch.float32, device="cuda")
    status = torch.empty(d.shape[0], dtype=torch.uint8, device="cuda")
    best, bs = m.rank(d, o, precision, eps=eps, eps32=eps32, scores=scores, status=status, eps16=eps16)
    torch.cuda.synchronize()
    return best.clone(), bs.clone(), scores, status


@pytest.mark.parametrize("staged", [False, True])
def test_plan_with_fp16_tier_matches_rank_ex(gpu_lib, setup, staged):
    """The FP16 tensor-core tier captured into a plan (advisor_plan_rank_ex /
    advisor_plan_rank_staged_ex): every replay equals the direct
    advisor_rank_ex call bit for bit, leaves the same per-tier counts, ranks
    refilled inputs, and selects what the FP64 oracle selects."""
    m = setup["m"]
    eps, eps16, eps32 = setup["eps"]["bf16"], setup["eps"]["fp16"], setup["eps"]["fp32"]
    d = torch.from_numpy(setup["d_a"]).cuda()
    o = torch.from_numpy(setup["off"]).cuda()
    direct = _direct_ex(m, d, o, "bf16", eps, eps16, eps32)
    counts = m.rescore_counts_ex()
    assert counts[0] > 0 and counts[1] < counts[0]   # the FP16 tier took candidates and passed on fewer
    if staged:
        h = torch.from_numpy(setup["d_a"]).pin_memory()
        dd = torch.empty_like(d)
        plan = m.plan_rank_staged(h, dd, o, "bf16", eps, eps32, n_stages=3, eps16=eps16)
    else:
        plan = m.plan_rank(d, o, "bf16", eps, eps32, eps16=eps16)
    assert plan.info()["kernels_per_replay"] > 7   # the FP16 tier adds its own kernels
    for _ in range(2):
        plan.launch()
    torch.cuda.synchronize()
    for a, b in zip((plan.best, plan.best_score, plan.scores, plan.status), direct):
        assert torch.equal(a, b)
    assert m.rescore_counts_ex() == counts
    assert np.array_equal(plan.best.cpu().numpy(), setup["ref_a"])
    # refill the bound inputs in place: the next replay ranks the new rows
    if staged:
        h.copy_(torch.from_numpy(setup["d_b"]))
    else:
        d.copy_(torch.from_numpy(setup["d_b"]).cuda())
    plan.launch()
    torch.cuda.synchronize()
    assert np.array_equal(plan.best.cpu().numpy(), setup["ref_b"])
    plan.close()
    if not staged:
        d.copy_(torch.from_numpy(setup["d_a"]).cuda())
    assert m.device_status() == 0


def test_rescore_counts_follow_the_replayed_plan(gpu_lib, setup):
    """Two plans of one model, with and without the FP16 tier: the per-tier
    counts after a replay are the replayed plan's, whichever was captured
    last."""
    m = setup["m"]
    eps, eps16, eps32 = setup["eps"]["bf16"], setup["eps"]["fp16"], setup["eps"]["fp32"]
    d = torch.from_numpy(setup["d_a"]).cuda()
    o = torch.from_numpy(setup["off"]).cuda()
    m.rank(d, o, "bf16", eps, eps32)
    plain_counts = m.rescore_counts_ex()
    assert plain_counts[0] == 0 and plain_counts[1] > 0
    _direct_ex(m, d, o, "bf16", eps, eps16, eps32)
    tier_counts = m.rescore_counts_ex()
    plain = m.plan_rank(d, o, "bf16", eps, eps32)
    tiered = m.plan_rank(d, o, "bf16", eps, eps32, eps16=eps16)   # captured last
    plain.launch()
    torch.cuda.synchronize()
    assert m.rescore_counts_ex() == plain_counts
    tiered.launch()
    torch.cuda.synchronize()
    assert m.rescore_counts_ex() == tier_counts
    plain.launch()
    torch.cuda.synchronize()
    assert m.rescore_counts_ex() == plain_counts
    plain.close()
    tiered.close()

