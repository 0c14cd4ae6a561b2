"""ctypes wrapper of the plain FP64 CPU oracle (advisor_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline / reference leg are the only callers.  The product package never
imports this module.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "advisor_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over rows where libgomp exists)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", _SRC, "-lm"]
    tmp = _LIB + f".tmp{os.getpid()}"
    try:
        subprocess.run(base[:-1] + ["-fopenmp", "-o", tmp, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp], check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        # ADVISOR_ORACLE_LIB: another build of advisor_oracle.c (the mutation
        # test runs the pins against copies with planted mistakes)
        _lib = ctypes.CDLL(os.environ.get("ADVISOR_ORACLE_LIB") or build())
        P = ctypes.c_void_p
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        _lib.orc_log2_q16.restype = i32
        _lib.orc_log2_q16.argtypes = [ctypes.c_uint64]
        _lib.orc_log2_q16_batch.argtypes = [P, i64, P]
        _lib.orc_validate.restype = ctypes.c_uint8
        _lib.orc_validate.argtypes = [P]
        _lib.orc_extract_features.restype = i64
        _lib.orc_extract_features.argtypes = [P, i64, ctypes.c_int, P, P]
        _lib.orc_fit_standardizer.argtypes = [P, P, i64, ctypes.c_int, P, P]
        _lib.orc_mlp_forward.argtypes = [P, P, i64, P, ctypes.c_int, P, P, P, P]
        _lib.orc_select_best.argtypes = [P, P, i64, P, P]
        _lib.orc_mlp_loss_grad.restype = dbl
        _lib.orc_mlp_loss_grad.argtypes = [P, P, i64, P, ctypes.c_int, P, P, P, P]
        _lib.orc_adam_step.argtypes = [P, P, P, P, i64, dbl, dbl, dbl, dbl, i64, P]
        _lib.orc_num_threads.restype = ctypes.c_int
        _lib.orc_set_num_threads.argtypes = [ctypes.c_int]
        _lib.orc_select_topn.argtypes = [P, P, i64, ctypes.c_int, P, P]
        _lib.orc_rmsprop_step.argtypes = [P, P, P, i64, dbl, dbl, dbl, dbl, P]
        _lib.orc_mlp_rmse_grad.restype = dbl
        _lib.orc_mlp_rmse_grad.argtypes = [P, P, i64, P, ctypes.c_int, P, P, P, P]
        _lib.orc_variant_count.restype = i64
        _lib.orc_variant_count.argtypes = [i64]
        _lib.orc_enumerate_variants.restype = i64
        _lib.orc_enumerate_variants.argtypes = [P, i64, P, P]
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on (timing only)."""
    lib().orc_set_num_threads(int(n))


def log2_q16(x) -> np.ndarray:
    x = _c(np.atleast_1d(x), np.uint64)
    out = np.empty(len(x), dtype=np.int32)
    lib().orc_log2_q16_batch(_p(x), len(x), _p(out))
    return out


def validate(desc) -> np.ndarray:
    desc = _c(np.atleast_2d(desc), np.int64)
    return np.array([lib().orc_validate(_p(desc[i])) for i in range(len(desc))], dtype=np.uint8)


def extract_features(desc, n_features: int):
    desc = _c(np.atleast_2d(desc), np.int64)
    n = len(desc)
    feat = np.empty((n, n_features), dtype=np.int32)
    status = np.empty(n, dtype=np.uint8)
    lib().orc_extract_features(_p(desc), n, n_features, _p(feat), _p(status))
    return feat, status


def fit_standardizer(feat, status=None):
    feat = _c(feat, np.int32)
    n, F = feat.shape
    mu = np.empty(F, dtype=np.float64)
    sigma = np.empty(F, dtype=np.float64)
    st = None if status is None else _c(status, np.uint8)
    lib().orc_fit_standardizer(_p(feat), None if st is None else _p(st), n, F, _p(mu), _p(sigma))
    return mu, sigma


def mlp_forward(feat, widths, params, mu, sigma, status=None) -> np.ndarray:
    feat = _c(feat, np.int32)
    w = _c(widths, np.int32)
    params = _c(params, np.float32)
    mu, sigma = _c(mu, np.float64), _c(sigma, np.float64)
    assert feat.shape[1] == w[0]
    y = np.empty(len(feat), dtype=np.float64)
    st = None if status is None else _c(status, np.uint8)
    lib().orc_mlp_forward(_p(feat), None if st is None else _p(st), len(feat), _p(w), len(w),
                          _p(params), _p(mu), _p(sigma), _p(y))
    return y


def select_best(y, offsets):
    y = _c(y, np.float64)
    off = _c(offsets, np.int64)
    K = len(off) - 1
    best = np.empty(K, dtype=np.int32)
    score = np.empty(K, dtype=np.float64)
    lib().orc_select_best(_p(y), _p(off), K, _p(best), _p(score))
    return best, score


def select_topn(y, offsets, N: int):
    """Top N per kernel (Fig. 2): best [K][N] local indices, score [K][N]; -1 / +inf padding."""
    y = _c(y, np.float64)
    off = _c(offsets, np.int64)
    K = len(off) - 1
    best = np.empty((K, N), dtype=np.int32)
    score = np.empty((K, N), dtype=np.float64)
    lib().orc_select_topn(_p(y), _p(off), K, int(N), _p(best), _p(score))
    return best, score


def variant_count(depth: int) -> int:
    """Variants generated for a loop nest of `depth` collapsible loops (Table 1)."""
    return int(lib().orc_variant_count(int(depth)))


def enumerate_variants(kernels):
    """Every variant of every kernel (Sec. 4.1.3): (variants [n][16] int64, seg_off [K+1])."""
    k = _c(kernels, np.int64).reshape(-1, 16)
    total = sum(variant_count(d) for d in k[:, 0])
    out = np.empty((total, 16), dtype=np.int64)
    off = np.empty(len(k) + 1, dtype=np.int64)
    n = lib().orc_enumerate_variants(_p(k), len(k), _p(out), _p(off))
    assert n == total
    return out, off


def rank_topn(desc, offsets, widths, params, mu, sigma, N: int):
    """Whole path with top-N selection: (best [K][N], score [K][N], y)."""
    feat, status = extract_features(desc, widths[0])
    y = mlp_forward(feat, widths, params, mu, sigma, status)
    best, score = select_topn(y, offsets, N)
    return best, score, y


def loss_grad(feat, labels, widths, params, mu, sigma):
    feat = _c(feat, np.int32)
    labels = _c(labels, np.float32)
    w = _c(widths, np.int32)
    params = _c(params, np.float32)
    mu, sigma = _c(mu, np.float64), _c(sigma, np.float64)
    grad = np.empty(len(params), dtype=np.float64)
    loss = lib().orc_mlp_loss_grad(_p(feat), _p(labels), len(feat), _p(w), len(w), _p(params),
                                   _p(mu), _p(sigma), _p(grad))
    return float(loss), grad


def rmse_grad(feat, labels, widths, params, mu, sigma):
    """RMSE loss (Sec. 5 Exp. 3) and its FP64 gradient."""
    feat = _c(feat, np.int32)
    labels = _c(labels, np.float32)
    w = _c(widths, np.int32)
    params = _c(params, np.float32)
    mu, sigma = _c(mu, np.float64), _c(sigma, np.float64)
    grad = np.empty(len(params), dtype=np.float64)
    loss = lib().orc_mlp_rmse_grad(_p(feat), _p(labels), len(feat), _p(w), len(w), _p(params),
                                   _p(mu), _p(sigma), _p(grad))
    return float(loss), grad


def rmsprop_step(params, grad, v, lr, alpha, eps, weight_decay):
    params = _c(params, np.float64)
    grad = _c(grad, np.float64)
    v = _c(v, np.float64).copy()
    out = np.empty_like(params)
    lib().orc_rmsprop_step(_p(params), _p(grad), _p(v), len(params), lr, alpha, eps, weight_decay, _p(out))
    return out, v


def adam_step(params, grad, m, v, lr, beta1, beta2, eps, step):
    params = _c(params, np.float64)
    grad = _c(grad, np.float64)
    m = _c(m, np.float64).copy()
    v = _c(v, np.float64).copy()
    out = np.empty_like(params)
    lib().orc_adam_step(_p(params), _p(grad), _p(m), _p(v), len(params), lr, beta1, beta2, eps,
                        step, _p(out))
    return out, m, v


def rank(desc, offsets, widths, params, mu, sigma):
    """Whole path: features -> FP64 scores -> per-kernel best (local index, score)."""
    feat, status = extract_features(desc, widths[0])
    y = mlp_forward(feat, widths, params, mu, sigma, status)
    best, score = select_best(y, offsets)
    return best, score, y, feat, status
