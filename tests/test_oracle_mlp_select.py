"""Pins of the oracle's standardisation, FP64 MLP, selection, gradient and
Adam step: closed forms, brute force, an independent matrix formulation and
finite differences."""
import numpy as np
import pytest

import oracle
from paper_2301_03636_gb300 import workloads as W


def _rand_feat(n, F, seed):
    d = W.make_descriptors(n, seed)
    f, st = oracle.extract_features(d, F)
    return f, st


def _layers(params, widths):
    out, off = [], 0
    for i in range(len(widths) - 1):
        fi, fo = widths[i], widths[i + 1]
        Wm = params[off:off + fo * fi].reshape(fo, fi).astype(np.float64)
        b = params[off + fo * fi: off + fo * fi + fo].astype(np.float64)
        out.append((Wm, b))
        off += fo * fi + fo
    return out


def _matrix_forward(f, widths, params, mu, sigma):
    h = (f.astype(np.float64) / 65536.0 - mu) / sigma
    layers = _layers(params, widths)
    for i, (Wm, b) in enumerate(layers):
        h = h @ Wm.T + b
        if i + 1 < len(layers):
            h = np.maximum(h, 0.0)
    return h[:, 0]


def test_standardizer_against_moments():
    f, st = _rand_feat(4000, 64, 8)
    st[::7] = 1  # mark some rows invalid: they must be excluded
    mu, sigma = oracle.fit_standardizer(f, st)
    x = f[st == 0].astype(np.float64) / 65536.0
    assert np.allclose(mu, x.mean(axis=0), rtol=1e-12, atol=1e-12)
    sd = x.std(axis=0)
    assert np.allclose(sigma, np.where(sd > 0, sd, 1.0), rtol=1e-10, atol=1e-12)
    assert np.all(sigma[sd == 0] == 1.0)  # e.g. level-3 features of depth <= 3 rows


def test_standardizer_closed_form():
    """Feature j of valid row i is a_j when i is even and b_j when i is odd
    (equal counts): the mean is (a_j + b_j) / 2 and the population standard
    deviation |a_j - b_j| / 2, exactly; a constant feature gets sigma 1; rows
    marked invalid (here carrying huge values) are left out."""
    F, n = 8, 1000
    a = np.array([0, 1, 2, 3, -4, 5, 7, 7], dtype=np.int64) * 65536
    b = np.array([2, 1, 6, 3, 4, -5, 7, 9], dtype=np.int64) * 65536
    f = np.where((np.arange(n) % 2 == 0)[:, None], a, b).astype(np.int32)
    st = np.zeros(n, dtype=np.uint8)
    bad = np.full((3, F), 1 << 30, dtype=np.int32)
    f = np.concatenate([f, bad])
    st = np.concatenate([st, np.ones(3, dtype=np.uint8)])
    mu, sigma = oracle.fit_standardizer(f, st)
    assert mu.tolist() == [1.0, 1.0, 4.0, 3.0, 0.0, 0.0, 7.0, 8.0]
    assert sigma.tolist() == [1.0, 1.0, 2.0, 1.0, 4.0, 5.0, 1.0, 1.0]   # constants (j = 1, 3, 6) -> 1


def test_zero_weights_constant_output_and_all_ties():
    widths = (32, 16, 16, 1)
    p = np.zeros(W.param_count(widths), dtype=np.float32)
    p[-1] = 0.75  # output bias
    f, st = _rand_feat(100, 32, 1)
    y = oracle.mlp_forward(f, widths, p, np.zeros(32), np.ones(32), st)
    assert np.all(y == 0.75)
    off = np.array([0, 10, 30, 31, 100], dtype=np.int64)
    best, score = oracle.select_best(y, off)
    assert best.tolist() == [0, 0, 0, 0] and np.all(score == 0.75)


@pytest.mark.parametrize("j", [1, 5, 9, 14, 17])
def test_identity_embedding(j):
    # W1 = [I; 0] passes the (non-negative) raw features through the ReLU, the
    # hidden layer is the identity and the output picks feature j.
    F, H = 32, 32
    widths = (F, H, H, 1)
    W1 = np.eye(H, F)
    W2 = np.eye(H)
    w3 = np.zeros((1, H)); w3[0, j] = 1.0
    p = np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), w3.ravel(), [0.0]]).astype(np.float32)
    f, st = _rand_feat(256, F, 2)
    y = oracle.mlp_forward(f, widths, p, np.zeros(F), np.ones(F), st)
    assert np.array_equal(y, f[:, j] / 65536.0)
    off = np.arange(0, 257, 8, dtype=np.int64)
    best, _ = oracle.select_best(y, off)
    for k in range(32):
        seg = f[off[k]:off[k + 1], j]
        assert best[k] == int(np.argmin(seg))  # numpy argmin: first occurrence


def test_nonnegative_network_is_affine():
    # Non-negative standardised inputs and weights keep every ReLU inactive,
    # so the network equals the product of its affine maps.
    rng = np.random.Generator(np.random.PCG64(3))
    widths = (32, 24, 16, 1)
    f, st = _rand_feat(200, 32, 4)
    mu = np.full(32, -1.0)  # z = x + 1 > 0
    sigma = np.ones(32)
    p = np.abs(rng.normal(size=W.param_count(widths))).astype(np.float32)
    y = oracle.mlp_forward(f, widths, p, mu, sigma, st)
    A = np.eye(32)
    c = np.zeros(32)
    for Wm, b in _layers(p, widths):
        A, c = Wm @ A, Wm @ c + b
    z = f.astype(np.float64) / 65536.0 + 1.0
    assert np.allclose(y, (z @ A.T + c)[:, 0], rtol=1e-12)


def test_scalar_network():
    # widths 1-1-1: y = w2 * relu(w1 * z + b1) + b2
    f = np.array([[0], [65536], [-131072], [3 * 65536]], dtype=np.int32)
    p = np.array([2.0, -1.0, 0.5, 0.25], dtype=np.float32)  # w1, b1, w2, b2
    y = oracle.mlp_forward(f, (1, 1, 1), p, np.zeros(1), np.ones(1))
    z = np.array([0.0, 1.0, -2.0, 3.0])
    assert y.tolist() == (0.5 * np.maximum(2.0 * z - 1.0, 0.0) + 0.25).tolist()


def test_random_network_matches_matrix_form():
    widths = (64, 96, 64, 48, 1)
    f, st = _rand_feat(500, 64, 6)
    mu, sigma = oracle.fit_standardizer(f, st)
    p = W.make_weights(widths, 9, "he", bias_scale=0.3)
    y = oracle.mlp_forward(f, widths, p, mu, sigma, st)
    assert np.allclose(y, _matrix_forward(f, widths, p, mu, sigma), rtol=1e-11, atol=1e-11)


def test_invalid_rows_score_inf_and_never_selected():
    f, st = _rand_feat(20, 32, 7)
    st[[0, 1, 5]] = 2
    p = W.make_weights((32, 8, 1), 1)
    y = oracle.mlp_forward(f, (32, 8, 1), p, np.zeros(32), np.ones(32), st)
    assert np.all(np.isinf(y[[0, 1, 5]])) and np.all(np.isfinite(np.delete(y, [0, 1, 5])))
    best, score = oracle.select_best(y, np.array([0, 2, 20], dtype=np.int64))
    assert best[0] == -1 and score[0] == np.inf and best[1] >= 0 and best[1] != 3


def test_select_edge_cases():
    y = np.array([3.0, 1.0, 1.0, 2.0, -0.0, 0.0, 0.0, np.nan, 5.0, np.inf, np.inf, 7.0], dtype=np.float64)
    off = np.array([0, 4, 4, 7, 9, 11, 12], dtype=np.int64)
    best, score = oracle.select_best(y, off)
    # [3,1,1,2] -> 1 (lowest of the tied); [] -> -1; [-0,0,0] -> 0 (-0 == +0);
    # [nan,5] -> 1; [inf,inf] -> -1; [7] -> 0
    assert best.tolist() == [1, -1, 0, 1, -1, 0]
    assert score[0] == 1.0 and score[1] == np.inf and score[3] == 5.0 and score[5] == 7.0


def test_select_brute_force_and_permutation():
    rng = np.random.Generator(np.random.PCG64(12))
    counts = rng.integers(1, 40, size=300)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    y = rng.integers(0, 6, size=off[-1]).astype(np.float64)  # many exact ties
    best, score = oracle.select_best(y, off)
    for k in range(300):
        seg = y[off[k]:off[k + 1]]
        m = seg.min()
        assert best[k] == min(i for i, v in enumerate(seg) if v == m) and score[k] == m
    # permuting the variants of a kernel keeps the selected score (the selected
    # variant is the same one up to ties)
    y2 = y.copy()
    for k in range(300):
        s = slice(off[k], off[k + 1])
        y2[s] = rng.permutation(y2[s])
    _, score2 = oracle.select_best(y2, off)
    assert np.array_equal(score, score2)


def test_duplicate_min_row_lower_index_wins():
    widths = (32, 16, 1)
    d = W.make_descriptors(10, 21)
    p = W.make_weights(widths, 2)
    f, st = oracle.extract_features(d, 32)
    mu, sigma = oracle.fit_standardizer(f, st)
    y = oracle.mlp_forward(f, widths, p, mu, sigma, st)
    i = int(np.argmin(y))
    d2 = np.insert(d, 0, d[i], axis=0)  # duplicate of the minimum first
    best, _, _, _, _ = oracle.rank(d2, np.array([0, 11], dtype=np.int64), widths, p, mu, sigma)
    assert best[0] == 0


def _fd_mismatches(loss_of, p, g, h=2.0 ** -20, tol_abs=1e-8, tol_rel=1e-6):
    """Indices where the central difference of loss_of over every parameter
    disagrees with the analytic gradient g.  Parameters sit on a 2^-12 grid
    and h = 2^-20, so p +- h is exact in FP32; between ReLU kinks the output
    is affine in each parameter, so the difference is exact up to rounding
    (and O(h^2) for the RMSE), and only a kink crossed inside +-h can
    disagree."""
    bad = []
    for i in range(len(p)):
        pp, pm = p.copy(), p.copy()
        pp[i] += np.float32(h)
        pm[i] -= np.float32(h)
        assert float(pp[i]) - float(p[i]) == h and float(p[i]) - float(pm[i]) == h
        fd = (loss_of(pp) - loss_of(pm)) / (2 * h)
        if abs(fd - g[i]) > tol_abs + tol_rel * abs(g[i]):
            bad.append(i)
    return bad


def test_gradient_against_finite_differences():
    """Every entry of the MSE gradient (weights and biases of every layer)
    against central differences of the loss."""
    widths = (32, 12, 8, 1)
    rng = np.random.Generator(np.random.PCG64(5))
    p = (np.round(rng.normal(0, 0.4, size=W.param_count(widths)) * 4096) / 4096).astype(np.float32)
    f, st = _rand_feat(64, 32, 13)
    mu, sigma = oracle.fit_standardizer(f, st)
    t = rng.normal(0, 1, size=64).astype(np.float32)
    loss, g = oracle.loss_grad(f, t, widths, p, mu, sigma)
    y = oracle.mlp_forward(f, widths, p, mu, sigma)
    assert abs(loss - 0.5 * np.mean((y - t.astype(np.float64)) ** 2)) < 1e-12
    bad = _fd_mismatches(lambda q: oracle.loss_grad(f, t, widths, q, mu, sigma)[0], p, g)
    assert len(bad) <= 2, bad   # at most a ReLU kink or two inside +-h


def test_adam_first_step_closed_form():
    # step 1: m_hat = g, v_hat = g^2, so the update is -lr * g / (|g| + eps)
    p = np.array([1.0, -2.0, 0.5, 0.0])
    g = np.array([0.1, -3.0, 0.0, 1e-3])
    out, m, v = oracle.adam_step(p, g, np.zeros(4), np.zeros(4), 1e-3, 0.9, 0.999, 1e-8, 1)
    assert np.allclose(out, p - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_rmse_gradient_against_finite_differences():
    """RMSE loss of Sec. 5 Exp. 3 (sqrt of the mean squared error), checked
    against its definition on the forward values and by central differences."""
    widths = (33, 10, 6, 1)
    rng = np.random.Generator(np.random.PCG64(9))
    p = (np.round(rng.normal(0, 0.4, size=W.param_count(widths)) * 4096) / 4096).astype(np.float32)
    d = W.make_descriptors(48, 19)
    f, st = oracle.extract_features(d, 33)
    mu, sigma = oracle.fit_standardizer(f, st)
    t = rng.normal(0, 1, size=48).astype(np.float32)
    loss, g = oracle.rmse_grad(f, t, widths, p, mu, sigma)
    y = oracle.mlp_forward(f, widths, p, mu, sigma)
    assert abs(loss - np.sqrt(np.mean((y - t.astype(np.float64)) ** 2))) < 1e-12
    bad = _fd_mismatches(lambda q: oracle.rmse_grad(f, t, widths, q, mu, sigma)[0], p, g)
    assert len(bad) <= 2, bad


def test_rmsprop_first_steps_closed_form():
    """From v = 0: v1 = (1 - a) g'^2 and the update is lr g' / (sqrt(1 - a) |g'| + eps),
    with g' = g + wd w; a second step follows the recursion by hand."""
    p = np.array([1.0, -2.0, 0.5, 0.0])
    g = np.array([0.1, -3.0, 0.0, 1e-3])
    lr, a, eps, wd = 0.01, 0.99, 1e-8, 1e-4
    out, v = oracle.rmsprop_step(p, g, np.zeros(4), lr, a, eps, wd)
    gp = g + wd * p
    assert np.allclose(v, (1 - a) * gp * gp, rtol=1e-14, atol=0)
    assert np.allclose(out, p - lr * gp / (np.sqrt(1 - a) * np.abs(gp) + eps), rtol=1e-13, atol=1e-16)
    out2, v2 = oracle.rmsprop_step(out, g, v, lr, a, eps, wd)
    gp2 = g + wd * out
    vv = a * v + (1 - a) * gp2 * gp2
    assert np.allclose(v2, vv, rtol=1e-14, atol=0)
    assert np.allclose(out2, out - lr * gp2 / (np.sqrt(vv) + eps), rtol=1e-13, atol=1e-16)


def test_features_33_are_the_base_features_and_the_collapse_count():
    """F = 33 (the paper's input width): the 32 base features and
    (dist_collapse + pf_collapse) * 2^16, hand-checked on fixed variants."""
    d = np.ones((3, 16), dtype=np.int64)
    d[:, 0] = 3
    d[:, 1:4] = [[16, 8, 4], [16, 8, 4], [16, 8, 4]]
    d[:, 5], d[:, 6], d[:, 7], d[:, 8] = 2, 8, 1024, 512
    d[:, 9], d[:, 10] = 64, 128
    d[:, 11:14] = [[0, 0, 3], [1, 1, 2], [2, 2, 1]]   # (pf_pos, dist_collapse, pf_collapse)
    d[:, 14:16] = [[0, 0], [1, 1], [2, 0]]
    f33, st = oracle.extract_features(d, 33)
    f32, _ = oracle.extract_features(d, 32)
    assert (st == 0).all()
    assert np.array_equal(f33[:, :32], f32)
    assert f33[:, 32].tolist() == [3 * 65536, 3 * 65536, 3 * 65536]
    d[1, 13] = 1
    assert oracle.extract_features(d, 33)[0][1, 32] == 2 * 65536
