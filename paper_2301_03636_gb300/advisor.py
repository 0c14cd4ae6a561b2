"""Python binding of libadvisor (include/advisor.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  torch provides device memory and streams.  There is no CPU
fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import torch

from . import build as _build

OK = 0
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "bad descriptor", 3: "out of memory", 4: "CUDA error",
                5: "device wait timed out", 6: "unsupported", 7: "malformed segment offsets"}
FP32, BF16, FP16, FP64, FP8 = 0, 1, 2, 3, 4
PRECISIONS = {"fp32": FP32, "bf16": BF16, "fp16": FP16, "fp64": FP64, "fp8": FP8}

_lib = None


class AdvisorError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS_NAMES.get(code, code)} ({code})")
        self.code = code


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libadvisor.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libadvisor.so is not built ({path}); run paper_2301_03636_gb300.build.build()")
    L = ctypes.CDLL(path)
    P, i64, i32, f32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_size_t
    st = ctypes.c_int
    sig = {
        "advisor_status_string": (ctypes.c_char_p, [st]),
        "advisor_launch_count": (i64, []),
        "advisor_model_create": (st, [P, i32, ctypes.POINTER(P)]),
        "advisor_model_destroy": (st, [P]),
        "advisor_model_param_bytes": (sz, [P]),
        "advisor_model_param_count": (i64, [P]),
        "advisor_workspace_bytes": (sz, [P, i64, i64]),
        "advisor_model_bind": (st, [P, P, sz, P, sz, i64, i64]),
        "advisor_model_set_params": (st, [P, P, P, P, P]),
        "advisor_model_get_params": (st, [P, P, P]),
        "advisor_fit_standardizer": (st, [P, P, i64, i32, P, P, P]),
        "advisor_extract_features": (st, [P, i64, i32, P, P, P]),
        "advisor_score_variants": (st, [P, P, P, i64, st, P, P]),
        "advisor_score_variants_fp64": (st, [P, P, P, i64, P, P]),
        "advisor_select_best": (st, [P, P, i64, P, i64, P, f32, f32, P, P, P]),
        "advisor_rank": (st, [P, P, i64, P, i64, st, f32, f32, P, P, P, P, P]),
        "advisor_rank_ex": (st, [P, P, i64, P, i64, st, f32, f32, f32, P, P, P, P, P]),
        "advisor_rank_topn_ex": (st, [P, P, i64, P, i64, i32, st, f32, f32, f32, P, P, P, P, P]),
        "advisor_get_rescore_counts_ex": (st, [P, P, P]),
        "advisor_measure_fp32_fma_peak": (st, [P, P]),
        "advisor_model_check_wait_timeout": (st, [P, i64, P]),
        "advisor_train_step": (st, [P, P, P, i64, st, P, P, P]),
        "advisor_loss_grad": (st, [P, P, P, i64, st, P, P, P]),
        "advisor_get_device_status": (st, [P, P]),
        "advisor_model_set_profile_events": (st, [P, P, P]),
        "advisor_forward_saved": (st, [P, P, i64, st, P, P]),
        "advisor_score_variants_noalloc": (st, [P, P, P, i64, st, P, P]),
        "advisor_backward": (st, [P, P, i64, P, P]),
        "advisor_model_repack": (st, [P, P]),
        "advisor_model_master_offset": (sz, [P]),
        "advisor_model_get_adam_step": (i64, [P]),
        "advisor_model_set_adam_step": (st, [P, i64]),
        "advisor_model_get_launch_config": (st, [P, P]),
        "advisor_get_rescore_counts": (st, [P, P, P]),
        "advisor_model_calibrate_fp8": (st, [P, P, i64, P]),
        "advisor_variant_count": (i64, [i64]),
        "advisor_rank_topn": (st, [P, P, i64, P, i64, i32, st, f32, f32, P, P, P, P, P]),
        "advisor_train_step_ex": (st, [P, P, P, i64, st, P, P, P]),
        "advisor_enumerate_variants": (st, [P, i64, P, i64, P, P, P]),
        "advisor_model_set_launch_config": (st, [P, P]),
        "advisor_plan_rank": (st, [P, P, i64, P, i64, st, f32, f32, P, P, P, P, i32, P, ctypes.POINTER(P)]),
        "advisor_rank_staged": (st, [P, P, P, i64, P, i64, st, f32, f32, P, P, P, P, i32, P]),
        "advisor_plan_rank_staged": (st, [P, P, P, i64, P, i64, st, f32, f32, P, P, P, P, i32, i32, P,
                                          ctypes.POINTER(P)]),
        "advisor_rank_staged_ex": (st, [P, P, P, i64, P, i64, st, f32, f32, f32, P, P, P, P, i32, P]),
        "advisor_plan_rank_ex": (st, [P, P, i64, P, i64, st, f32, f32, f32, P, P, P, P, i32, P, ctypes.POINTER(P)]),
        "advisor_plan_rank_staged_ex": (st, [P, P, P, i64, P, i64, st, f32, f32, f32, P, P, P, P, i32, i32, P,
                                             ctypes.POINTER(P)]),
        "advisor_plan_launch": (st, [P, P]),
        "advisor_plan_info": (st, [P, P, P, P]),
        "advisor_plan_destroy": (st, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class LaunchConfig(ctypes.Structure):
    """advisor_launch_config: launch shapes of the hot path (results do not depend on them)."""
    _fields_ = [("extract_block", ctypes.c_int32), ("tc_ctas", ctypes.c_int32),
                ("list_blocks_per_sm", ctypes.c_int32), ("list_chunk_kb", ctypes.c_int32),
                ("select_block", ctypes.c_int32), ("layer_path", ctypes.c_int32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class TrainOptions(ctypes.Structure):
    """advisor_train_options: optimizer 0 Adam / 1 RMSprop, loss 0 MSE / 1 RMSE."""
    _fields_ = [("optimizer", ctypes.c_int32), ("loss", ctypes.c_int32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("alpha", ctypes.c_float),
                ("eps", ctypes.c_float), ("weight_decay", ctypes.c_float)]


def header_functions() -> list[str]:
    """Names of the functions declared in include/advisor.h."""
    h = os.path.join(_build.ROOT, "include", "advisor.h")
    text = open(h).read()
    return sorted(set(re.findall(r"\b(advisor_[a-z0-9_]+)\s*\(", text)))


def launch_count() -> int:
    return int(lib().advisor_launch_count())


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(code, what):
    if code != OK:
        raise AdvisorError(code, what)


def _prec(p):
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def _dev(x, dtype, device):
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=dtype).contiguous()
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=device)


# ---- stateless entry points --------------------------------------------------------


def advisor_extract_features(desc: torch.Tensor, n_features: int, stream=None):
    """a1-a2: descriptors [n,16] int64 (CUDA) -> (features [n,F] int32, status [n] uint8)."""
    assert desc.is_cuda and desc.dtype == torch.int64 and desc.is_contiguous() and desc.shape[-1] == 16
    n = desc.shape[0]
    feat = torch.empty((n, n_features), dtype=torch.int32, device=desc.device)
    status = torch.empty(n, dtype=torch.uint8, device=desc.device)
    _check(lib().advisor_extract_features(_ptr(desc), n, n_features, _ptr(feat), _ptr(status), _stream(stream)),
           "advisor_extract_features")
    return feat, status


def advisor_measure_fp32_fma_peak(stream=None) -> float:
    """Measured FP32 FMA rate of the CUDA cores, TFLOP/s (measurement only)."""
    v = ctypes.c_double()
    _check(lib().advisor_measure_fp32_fma_peak(ctypes.byref(v), _stream(stream)), "advisor_measure_fp32_fma_peak")
    return float(v.value)


def advisor_variant_count(depth: int) -> int:
    return int(lib().advisor_variant_count(int(depth)))


def advisor_enumerate_variants(kernels: torch.Tensor, stream=None):
    """Every offload variant of each kernel's loop nest (Sec. 4.1.3): kernels
    [K][16] int64 on the device -> (variants [n][16], seg_off [K+1])."""
    K = kernels.shape[0]
    cap = 84 * K   # the largest count per kernel (Table 1)
    out = torch.empty((max(cap, 1), 16), dtype=torch.int64, device=kernels.device)
    off = torch.empty(K + 1, dtype=torch.int64, device=kernels.device)
    total = torch.empty(1, dtype=torch.int64, device=kernels.device)
    _check(lib().advisor_enumerate_variants(_ptr(kernels), K, _ptr(out), cap, _ptr(off), _ptr(total),
                                            _stream(stream)), "advisor_enumerate_variants")
    n = int(total.item())
    return out[:n], off


def workspace_bytes(widths, max_rows: int, max_kernels: int) -> int:
    """Device bytes of the workspace a model of these widths needs for batches of
    up to max_rows variants and max_kernels kernels (advisor_workspace_bytes;
    nothing is allocated)."""
    w = (ctypes.c_int32 * len(widths))(*[int(x) for x in widths])
    h = ctypes.c_void_p()
    _check(lib().advisor_model_create(ctypes.cast(w, ctypes.c_void_p), len(widths), ctypes.byref(h)),
           "advisor_model_create")
    try:
        return int(lib().advisor_workspace_bytes(h, int(max_rows), int(max_kernels)))
    finally:
        lib().advisor_model_destroy(h)


def advisor_fit_standardizer(feat: torch.Tensor, status: torch.Tensor | None = None, stream=None):
    n, F = feat.shape
    mu = torch.empty(F, dtype=torch.float64, device=feat.device)
    sigma = torch.empty(F, dtype=torch.float64, device=feat.device)
    _check(lib().advisor_fit_standardizer(_ptr(feat), _ptr(status), n, F, _ptr(mu), _ptr(sigma), _stream(stream)),
           "advisor_fit_standardizer")
    return mu, sigma


class Model:
    """An MLP cost model bound to caller-owned (torch) device memory."""

    def __init__(self, widths, max_rows: int, max_kernels: int, device="cuda", param_block=None):
        self.widths = tuple(int(w) for w in widths)
        self.device = torch.device(device)
        w = (ctypes.c_int32 * len(self.widths))(*self.widths)
        h = ctypes.c_void_p()
        _check(lib().advisor_model_create(ctypes.cast(w, ctypes.c_void_p), len(self.widths), ctypes.byref(h)),
               "advisor_model_create")
        self.handle = h
        self.max_rows = int(max_rows)
        self.max_kernels = int(max_kernels)
        pb = lib().advisor_model_param_bytes(h)
        wb = lib().advisor_workspace_bytes(h, self.max_rows, self.max_kernels)
        if param_block is not None:
            # a second handle on another model's resident parameters (own workspace)
            assert param_block.numel() >= pb and param_block.dtype == torch.uint8
            self.param_block = param_block
        else:
            self.param_block = torch.empty(pb, dtype=torch.uint8, device=self.device)
        self.workspace = torch.empty(wb, dtype=torch.uint8, device=self.device)
        _check(lib().advisor_model_bind(h, _ptr(self.param_block), pb, _ptr(self.workspace), wb, self.max_rows,
                                        self.max_kernels), "advisor_model_bind")
        self.n_params = int(lib().advisor_model_param_count(h))

    def __del__(self):
        try:
            if getattr(self, "handle", None) is not None and _lib is not None:
                _lib.advisor_model_destroy(self.handle)
                self.handle = None
        except Exception:
            pass

    @property
    def n_features(self) -> int:
        return self.widths[0]

    def set_params(self, params, mu, sigma, stream=None):
        p = _dev(params, torch.float32, self.device)
        assert p.numel() == self.n_params
        m = _dev(mu, torch.float64, self.device)
        s = _dev(sigma, torch.float64, self.device)
        _check(lib().advisor_model_set_params(self.handle, _ptr(p), _ptr(m), _ptr(s), _stream(stream)),
               "advisor_model_set_params")
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()

    def get_params(self, stream=None) -> torch.Tensor:
        out = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        _check(lib().advisor_model_get_params(self.handle, _ptr(out), _stream(stream)), "advisor_model_get_params")
        return out

    def score(self, feat, status=None, precision="fp32", out=None, stream=None) -> torch.Tensor:
        n = feat.shape[0]
        out = torch.empty(n, dtype=torch.float32, device=self.device) if out is None else out
        _check(lib().advisor_score_variants(self.handle, _ptr(feat), _ptr(status), n, _prec(precision), _ptr(out),
                                            _stream(stream)), "advisor_score_variants")
        return out

    NOALLOC_MAX_ROWS = 16384

    def score_noalloc(self, feat, status=None, precision="bf16", out=None, stream=None) -> torch.Tensor:
        """Tensor-core scores without using the model's workspace: the
        library's fixed device scratch holds the 16-bit activations (at most
        NOALLOC_MAX_ROWS rows; calls overlapping on the GPU race)."""
        n = feat.shape[0]
        if n > self.NOALLOC_MAX_ROWS:
            raise AdvisorError(3, f"advisor_score_variants_noalloc: {n} rows exceed the fixed scratch of "
                                  f"{self.NOALLOC_MAX_ROWS} rows")
        out = torch.empty(n, dtype=torch.float32, device=self.device) if out is None else out
        _check(lib().advisor_score_variants_noalloc(self.handle, _ptr(feat), _ptr(status), n, _prec(precision),
                                                    _ptr(out), _stream(stream)), "advisor_score_variants_noalloc")
        return out

    def score_fp64(self, feat, status=None, stream=None) -> torch.Tensor:
        n = feat.shape[0]
        out = torch.empty(n, dtype=torch.float64, device=self.device)
        _check(lib().advisor_score_variants_fp64(self.handle, _ptr(feat), _ptr(status), n, _ptr(out),
                                                 _stream(stream)), "advisor_score_variants_fp64")
        return out

    def select(self, scores, offsets, feat=None, eps=-1.0, eps32=0.0, stream=None):
        K = offsets.shape[0] - 1
        best = torch.empty(K, dtype=torch.int32, device=self.device)
        best_score = torch.empty(K, dtype=torch.float64, device=self.device)
        _check(lib().advisor_select_best(self.handle, _ptr(scores), scores.shape[0], _ptr(offsets), K, _ptr(feat),
                                         float(eps), float(eps32), _ptr(best), _ptr(best_score), _stream(stream)),
               "advisor_select_best")
        return best, best_score

    def rank(self, desc, offsets, precision="bf16", eps=-1.0, eps32=0.0, scores=None, status=None, best=None,
             best_score=None, stream=None, eps16=None):
        """Best variant of every kernel (advisor_rank; with eps16, advisor_rank_ex's FP16 middle tier)."""
        K = offsets.shape[0] - 1
        best = torch.empty(K, dtype=torch.int32, device=self.device) if best is None else best
        best_score = torch.empty(K, dtype=torch.float64, device=self.device) if best_score is None else best_score
        if eps16 is None:
            _check(lib().advisor_rank(self.handle, _ptr(desc), desc.shape[0], _ptr(offsets), K, _prec(precision),
                                      float(eps), float(eps32), _ptr(best), _ptr(best_score), _ptr(scores),
                                      _ptr(status), _stream(stream)), "advisor_rank")
        else:
            _check(lib().advisor_rank_ex(self.handle, _ptr(desc), desc.shape[0], _ptr(offsets), K, _prec(precision),
                                         float(eps), float(eps16), float(eps32), _ptr(best), _ptr(best_score),
                                         _ptr(scores), _ptr(status), _stream(stream)), "advisor_rank_ex")
        return best, best_score

    def rescore_counts(self, stream=None):
        """(rows re-scored in FP32, rows re-scored in FP64) by the last selection with re-score."""
        c = (ctypes.c_int64 * 2)()
        _check(lib().advisor_get_rescore_counts(self.handle, ctypes.cast(c, ctypes.c_void_p), _stream(stream)),
               "advisor_get_rescore_counts")
        return int(c[0]), int(c[1])

    def rescore_counts_ex(self, stream=None):
        """(rows re-scored in FP16, in FP32, in FP64) by the last selection with re-score."""
        c = (ctypes.c_int64 * 3)()
        _check(lib().advisor_get_rescore_counts_ex(self.handle, ctypes.cast(c, ctypes.c_void_p), _stream(stream)),
               "advisor_get_rescore_counts_ex")
        return int(c[0]), int(c[1]), int(c[2])

    @property
    def launch_config(self) -> LaunchConfig:
        c = LaunchConfig()
        _check(lib().advisor_model_get_launch_config(self.handle, ctypes.byref(c)), "get_launch_config")
        return c

    @launch_config.setter
    def launch_config(self, c: LaunchConfig):
        _check(lib().advisor_model_set_launch_config(self.handle, ctypes.byref(c)), "set_launch_config")

    def plan_rank(self, desc, offsets, precision="bf16", eps=-1.0, eps32=0.0, autotune=False, stream=None,
                  eps16=None):
        """A Plan replaying rank() on these buffers (refill desc / offsets in place between launches);
        with eps16, the FP16 middle tier is captured too (advisor_plan_rank_ex)."""
        return Plan(self, desc, offsets, precision, eps, eps32, autotune, stream, eps16=eps16)

    def rank_staged(self, h_desc, d_desc, offsets, precision="bf16", eps=-1.0, eps32=0.0, n_stages=4,
                    scores=None, status=None, stream=None, eps16=None):
        """rank() on descriptors in pinned host memory (h_desc), copied into the device buffer
        d_desc in n_stages chunks that overlap the scoring (advisor_rank_staged[_ex])."""
        K = offsets.shape[0] - 1
        best = torch.empty(K, dtype=torch.int32, device=self.device)
        best_score = torch.empty(K, dtype=torch.float64, device=self.device)
        if eps16 is None:
            _check(lib().advisor_rank_staged(self.handle, _ptr(h_desc), _ptr(d_desc), h_desc.shape[0], _ptr(offsets),
                                             K, _prec(precision), float(eps), float(eps32), _ptr(best),
                                             _ptr(best_score), _ptr(scores), _ptr(status), int(n_stages),
                                             _stream(stream)), "advisor_rank_staged")
        else:
            _check(lib().advisor_rank_staged_ex(self.handle, _ptr(h_desc), _ptr(d_desc), h_desc.shape[0],
                                                _ptr(offsets), K, _prec(precision), float(eps), float(eps16),
                                                float(eps32), _ptr(best), _ptr(best_score), _ptr(scores),
                                                _ptr(status), int(n_stages), _stream(stream)), "advisor_rank_staged_ex")
        return best, best_score

    def plan_rank_staged(self, h_desc, d_desc, offsets, precision="bf16", eps=-1.0, eps32=0.0, n_stages=4,
                         autotune=False, stream=None, eps16=None):
        """A Plan replaying rank_staged() (refill h_desc / offsets in place between launches)."""
        return Plan(self, d_desc, offsets, precision, eps, eps32, autotune, stream, h_desc=h_desc,
                    n_stages=n_stages, eps16=eps16)

    def rank_topn(self, desc, offsets, top_n, precision="bf16", eps=-1.0, eps32=0.0, scores=None, status=None,
                  stream=None, eps16=None):
        """The top_n best variants of every kernel: (best [K][top_n] int32, score [K][top_n] float64)."""
        K = offsets.shape[0] - 1
        best = torch.empty((K, top_n), dtype=torch.int32, device=self.device)
        best_score = torch.empty((K, top_n), dtype=torch.float64, device=self.device)
        if eps16 is None:
            _check(lib().advisor_rank_topn(self.handle, _ptr(desc), desc.shape[0], _ptr(offsets), K, int(top_n),
                                           _prec(precision), float(eps), float(eps32), _ptr(best), _ptr(best_score),
                                           _ptr(scores), _ptr(status), _stream(stream)), "advisor_rank_topn")
        else:
            _check(lib().advisor_rank_topn_ex(self.handle, _ptr(desc), desc.shape[0], _ptr(offsets), K, int(top_n),
                                              _prec(precision), float(eps), float(eps16), float(eps32), _ptr(best),
                                              _ptr(best_score), _ptr(scores), _ptr(status), _stream(stream)),
                   "advisor_rank_topn_ex")
        return best, best_score

    def train_step(self, feat, labels, precision="fp32", lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                   weight_decay=0.0, loss=None, stream=None):
        h = (ctypes.c_float * 5)(lr, beta1, beta2, eps, weight_decay)
        _check(lib().advisor_train_step(self.handle, _ptr(feat), _ptr(labels), feat.shape[0], _prec(precision),
                                        ctypes.cast(h, ctypes.c_void_p), _ptr(loss), _stream(stream)),
               "advisor_train_step")
        return loss

    def train_step_ex(self, feat, labels, precision="fp32", optimizer="rmsprop", loss_fn="rmse", lr=0.01,
                      alpha=0.99, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, loss=None, stream=None):
        """One step with a choice of optimizer ("adam" / "rmsprop") and loss ("mse" / "rmse")."""
        o = TrainOptions(optimizer={"adam": 0, "rmsprop": 1}[optimizer], loss={"mse": 0, "rmse": 1}[loss_fn],
                         lr=lr, beta1=beta1, beta2=beta2, alpha=alpha, eps=eps, weight_decay=weight_decay)
        _check(lib().advisor_train_step_ex(self.handle, _ptr(feat), _ptr(labels), feat.shape[0], _prec(precision),
                                           ctypes.byref(o), _ptr(loss), _stream(stream)), "advisor_train_step_ex")
        return loss

    def loss_grad(self, feat, labels, precision="fp32", stream=None):
        grad = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        _check(lib().advisor_loss_grad(self.handle, _ptr(feat), _ptr(labels), feat.shape[0], _prec(precision),
                                       _ptr(grad), _ptr(loss), _stream(stream)), "advisor_loss_grad")
        return loss, grad

    def set_profile_events(self, start=None, stop=None):
        """Bracket later tensor-core scorer launches with these torch.cuda.Events."""
        if start is None:
            _check(lib().advisor_model_set_profile_events(self.handle, None, None), "set_profile_events")
            return
        _check(lib().advisor_model_set_profile_events(self.handle, ctypes.c_void_p(start.cuda_event),
                                                      ctypes.c_void_p(stop.cuda_event)), "set_profile_events")

    # ---- training mode -------------------------------------------------------------

    def master(self) -> torch.Tensor:
        """The FP32 master parameters as a tensor view into the parameter block
        (per layer W[out][in] then b[out]).  After changing them in place, call
        repack() so that the scorers see the new values."""
        off = int(lib().advisor_model_master_offset(self.handle))
        return self.param_block[off:off + 4 * self.n_params].view(torch.float32)

    def repack(self, stream=None):
        _check(lib().advisor_model_repack(self.handle, _stream(stream)), "advisor_model_repack")

    def forward_saved(self, feat, precision="fp32", stream=None) -> torch.Tensor:
        y = torch.empty(feat.shape[0], dtype=torch.float32, device=self.device)
        _check(lib().advisor_forward_saved(self.handle, _ptr(feat), feat.shape[0], _prec(precision), _ptr(y),
                                           _stream(stream)), "advisor_forward_saved")
        return y

    def backward(self, dy, stream=None) -> torch.Tensor:
        dy = dy.contiguous().to(torch.float32)
        grad = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        _check(lib().advisor_backward(self.handle, _ptr(dy), dy.shape[0], _ptr(grad), _stream(stream)),
               "advisor_backward")
        return grad

    @property
    def adam_step(self) -> int:
        return int(lib().advisor_model_get_adam_step(self.handle))

    @adam_step.setter
    def adam_step(self, step: int):
        _check(lib().advisor_model_set_adam_step(self.handle, int(step)), "advisor_model_set_adam_step")

    def device_status(self, stream=None) -> int:
        return int(lib().advisor_get_device_status(self.handle, _stream(stream)))

    def check_wait_timeout(self, timeout_ns: int, stream=None):
        """Failure-detection self-test: a bounded device wait on a barrier nothing
        arrives at runs out after timeout_ns and records the timeout in the status
        word (advisor_model_check_wait_timeout); read it with device_status()."""
        _check(lib().advisor_model_check_wait_timeout(self.handle, int(timeout_ns), _stream(stream)),
               "advisor_model_check_wait_timeout")

    def calibrate_fp8(self, feat, stream=None):
        """Static per-tensor activation scales for FP8 scoring from a calibration
        sample of features (see advisor_model_calibrate_fp8)."""
        _check(lib().advisor_model_calibrate_fp8(self.handle, _ptr(feat), feat.shape[0], _stream(stream)),
               "advisor_model_calibrate_fp8")

    def calibrate_eps(self, feat, status=None, precision="bf16", safety=2.0):
        """Measured error bound of a precision against the FP64 scorer on a
        calibration sample: safety * max |score - fp64| over the valid rows."""
        y = self.score(feat, status, precision).double()
        y64 = self.score_fp64(feat, status)
        ok = torch.isfinite(y64)
        return float(safety * (y[ok] - y64[ok]).abs().max().item())


class Plan:
    """advisor_plan_rank: Model.rank captured into a CUDA graph, replayed by launch().

    The plan keeps the input and output tensors alive; launch() reads the
    current contents of `desc` and `offsets` and writes best / best_score /
    scores / status in place."""

    def __init__(self, model: Model, desc, offsets, precision="bf16", eps=-1.0, eps32=0.0, autotune=False,
                 stream=None, h_desc=None, n_stages=1, eps16=None):
        self.model = model
        self.desc, self.offsets, self.h_desc = desc, offsets, h_desc
        K = offsets.shape[0] - 1
        self.best = torch.empty(K, dtype=torch.int32, device=model.device)
        self.best_score = torch.empty(K, dtype=torch.float64, device=model.device)
        self.scores = torch.empty(desc.shape[0], dtype=torch.float32, device=model.device)
        self.status = torch.empty(desc.shape[0], dtype=torch.uint8, device=model.device)
        h = ctypes.c_void_p()
        e16 = -1.0 if eps16 is None else float(eps16)
        if h_desc is None:
            _check(lib().advisor_plan_rank_ex(model.handle, _ptr(desc), desc.shape[0], _ptr(offsets), K,
                                              _prec(precision), float(eps), e16, float(eps32), _ptr(self.best),
                                              _ptr(self.best_score), _ptr(self.scores), _ptr(self.status),
                                              1 if autotune else 0, _stream(stream), ctypes.byref(h)),
                   "advisor_plan_rank_ex")
        else:
            _check(lib().advisor_plan_rank_staged_ex(model.handle, _ptr(h_desc), _ptr(desc), desc.shape[0],
                                                     _ptr(offsets), K, _prec(precision), float(eps), e16,
                                                     float(eps32), _ptr(self.best), _ptr(self.best_score),
                                                     _ptr(self.scores), _ptr(self.status), int(n_stages),
                                                     1 if autotune else 0, _stream(stream), ctypes.byref(h)),
                   "advisor_plan_rank_staged_ex")
        self.handle = h

    def launch(self, stream=None):
        _check(lib().advisor_plan_launch(self.handle, _stream(stream)), "advisor_plan_launch")
        return self.best, self.best_score

    def info(self):
        c = LaunchConfig()
        us = ctypes.c_float()
        k = ctypes.c_int32()
        _check(lib().advisor_plan_info(self.handle, ctypes.byref(c), ctypes.byref(us), ctypes.byref(k)),
               "advisor_plan_info")
        return {"config": c.as_dict(), "replay_us": float(us.value), "kernels_per_replay": int(k.value)}

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.advisor_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLPFunction(torch.autograd.Function):
    """y = MLP(features) with the library's hand-written backward.

    apply(master, feat, model, precision="fp32"): `master` must be
    model.master() (the FP32 parameters the forward reads); its gradient comes
    from advisor_backward.  precision "bf16" / "fp16" runs the layer GEMMs on
    the tensor cores.  The features are integer inputs and get no gradient."""

    @staticmethod
    def forward(ctx, master, feat, model, precision="fp32"):
        ctx.model = model
        ctx.n = feat.shape[0]
        return model.forward_saved(feat, precision)

    @staticmethod
    def backward(ctx, dy):
        grad = ctx.model.backward(dy)
        return grad, None, None, None
