"""The paper's own cost-model recipe (Sec. 5 Exp. 3): 33 input features, the
33-66-132-66-33-1 network (odd widths, zero-padded on the tensor cores),
Glorot weights with zero biases, RMSprop (lr 0.01 x 0.1 every 30 epochs,
weight decay 1e-4) on the RMSE loss with batch 16 for 150 epochs, an 80/20
split and the NRMSE criterion.  Against the oracle: the 33 features
bit-exact, scores within the calibrated bounds and selections identical, one
RMSprop + RMSE step; then the whole recipe on synthetic data."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03636_gb300 import advisor, metrics, training
from paper_2301_03636_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PAPER = (33, 66, 132, 66, 33, 1)


def test_33_features_bit_exact(gpu_lib):
    d = W.make_descriptors(5000, 61, max_depth=4)
    d[::37, 3] = 0   # some invalid rows
    f, st = advisor.advisor_extract_features(torch.from_numpy(d).cuda(), 33)
    fr, sr = oracle.extract_features(d, 33)
    assert np.array_equal(st.cpu().numpy(), sr)
    assert np.array_equal(f.cpu().numpy(), fr)


@pytest.fixture(scope="module")
def paper_model():
    off = W.make_segments(256, 2, 48, seed=62)
    d = W.make_descriptors(int(off[-1]), 62)
    cal = W.calibration_descriptors(16384)
    fc, sc = oracle.extract_features(cal, 33)
    mu, sigma = oracle.fit_standardizer(fc, sc)
    p = W.make_weights(PAPER, 62, "glorot")
    m = advisor.Model(PAPER, max_rows=max(len(d), 16384), max_kernels=256)
    m.set_params(p, mu, sigma)
    fcal, scal = advisor.advisor_extract_features(torch.from_numpy(cal).cuda(), 33)
    f, st = oracle.extract_features(d, 33)
    y_ref = oracle.mlp_forward(f, PAPER, p, mu, sigma, status=st)
    return dict(off=off, d=d, m=m, p=p, mu=mu, sigma=sigma, fcal=fcal, scal=scal, y_ref=y_ref)


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
def test_paper_network_scores_and_selection(gpu_lib, paper_model, precision):
    m = paper_model["m"]
    d = torch.from_numpy(paper_model["d"]).cuda()
    o = torch.from_numpy(paper_model["off"]).cuda()
    eps = m.calibrate_eps(paper_model["fcal"], paper_model["scal"], precision)
    eps32 = m.calibrate_eps(paper_model["fcal"], paper_model["scal"], "fp32")
    scores = torch.empty(len(paper_model["d"]), dtype=torch.float32, device="cuda")
    best, _ = m.rank(d, o, precision, eps=eps, eps32=eps32, scores=scores)
    err = np.abs(scores.cpu().numpy().astype(np.float64) - paper_model["y_ref"])
    print(f"{precision}: max|dy| {err.max():.3e} eps {eps:.3e}")
    assert err.max() <= eps / 2 * 1.5
    ref_best, _ = oracle.select_best(paper_model["y_ref"], paper_model["off"])
    assert np.array_equal(best.cpu().numpy(), ref_best)
    top, _ = m.rank_topn(d, o, 5, precision, eps=eps, eps32=eps32)
    assert np.array_equal(top.cpu().numpy(), oracle.select_topn(paper_model["y_ref"], paper_model["off"], 5)[0])


def test_rmsprop_rmse_step_matches_oracle(gpu_lib):
    d = W.make_descriptors(2048, 63)
    f, st = oracle.extract_features(d, 33)
    mu, sigma = oracle.fit_standardizer(f, st)
    p = W.make_weights(PAPER, 63, "glorot", 0.05)
    t = W.make_labels(d, 63)
    m = advisor.Model(PAPER, max_rows=2048, max_kernels=1)
    m.set_params(p, mu, sigma)
    loss_ref, g_ref = oracle.rmse_grad(f, t, PAPER, p, mu, sigma)
    new_ref, _ = oracle.rmsprop_step(p.astype(np.float64), g_ref, np.zeros(len(p)), 0.01, 0.99, 1e-8, 1e-4)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    m.train_step_ex(torch.from_numpy(f).cuda(), torch.from_numpy(t).cuda(), "fp32", "rmsprop", "rmse", lr=0.01,
                    weight_decay=1e-4, loss=loss)
    assert abs(float(loss.item()) - loss_ref) <= 1e-5 * loss_ref
    new = m.get_params().cpu().numpy().astype(np.float64)
    diff = np.abs(new - new_ref)
    # step 1 moves each weight by about lr g' / (0.1 |g'|): identical except where g' is near zero
    assert np.mean(diff <= 1e-4 * 0.01 + 1e-7) > 0.995
    assert diff.max() <= 0.2


def test_paper_recipe_meets_nrmse_criterion(gpu_lib):
    d = W.make_descriptors(5000, 64, max_depth=4)
    t = W.make_labels(d, 64)
    n_tr = 4000   # the 80 / 20 split
    f_all, s_all = advisor.advisor_extract_features(torch.from_numpy(d).cuda(), 33)
    f_tr, f_va = f_all[:n_tr].contiguous(), f_all[n_tr:].contiguous()
    mu, sigma = advisor.advisor_fit_standardizer(f_tr, s_all[:n_tr].contiguous())   # the training split's statistics
    m = advisor.Model(PAPER, max_rows=n_tr, max_kernels=1)
    m.set_params(W.make_weights(PAPER, 64, "glorot"), mu, sigma)
    losses = []
    training.train_paper_recipe(m, f_tr, torch.from_numpy(t[:n_tr]).cuda(), epoch_losses=losses)
    ev = training.evaluate(m, f_va, torch.from_numpy(t[n_tr:]).cuda())
    print(f"RMSE per epoch: {losses[0]:.4f} -> {losses[29]:.4f} -> {losses[-1]:.4f}; "
          f"validation RMSE {ev['rmse']:.4f} NRMSE {ev['nrmse']:.4f}")
    assert losses[-1] < 0.5 * losses[0]
    assert ev["nrmse"] < metrics.SUCCESS_NRMSE
