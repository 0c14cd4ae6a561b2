"""The C-ABI library builds, loads without a GPU and exports every function
include/advisor.h declares; host-side argument checks reject bad calls
without touching the device."""
import ctypes

import pytest

from paper_2301_03636_gb300 import advisor, build


@pytest.fixture(scope="module")
def L():
    build.build()
    return advisor.lib()


def test_exports_every_declared_function(L):
    names = advisor.header_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(L, n), n


def test_status_strings(L):
    for code in range(8):
        assert L.advisor_status_string(code)


def test_model_create_argument_checks(L):
    h = ctypes.c_void_p()

    def create(ws):
        arr = (ctypes.c_int32 * len(ws))(*ws)
        return L.advisor_model_create(ctypes.cast(arr, ctypes.c_void_p), len(ws), ctypes.byref(h))

    assert create([64, 256, 256, 256, 1]) == 0
    assert L.advisor_model_param_count(h) == 64 * 256 + 256 + 2 * (256 * 256 + 256) + 256 + 1
    assert L.advisor_model_param_bytes(h) > 0
    assert L.advisor_workspace_bytes(h, 1000, 10) > L.advisor_workspace_bytes(h, 10, 10)
    assert L.advisor_model_destroy(h) == 0
    assert create([64, 256, 2]) == 1        # output width must be 1
    assert create([48, 256, 1]) == 1        # F must be 32, 64 or 128
    assert create([64, 1]) == 1             # at least one hidden layer
    assert create([64, 2048, 1]) == 1       # hidden width limit


def test_extract_rejects_bad_arguments(L):
    s = None
    assert L.advisor_extract_features(None, 10, 64, None, None, s) == 1
    assert L.advisor_extract_features(None, 0, 64, None, None, s) == 0   # empty call is a no-op
    assert L.advisor_extract_features(None, 10, 48, None, None, s) == 1


def test_unbound_model_is_rejected(L):
    h = ctypes.c_void_p()
    arr = (ctypes.c_int32 * 4)(32, 128, 128, 1)
    assert L.advisor_model_create(ctypes.cast(arr, ctypes.c_void_p), 4, ctypes.byref(h)) == 0
    assert L.advisor_score_variants(h, ctypes.c_void_p(256), None, 10, 0, ctypes.c_void_p(256), None) == 1
    assert L.advisor_model_destroy(h) == 0


def test_newer_entry_points_reject_bad_arguments(L):
    """Argument checks of the staged, top-N, plan and self-test calls return
    ADVISOR_ERR_INVALID_ARGUMENT on the host, before anything is enqueued."""
    P, i64, i32, f32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float
    L = ctypes.CDLL(advisor.library_path())   # own function objects: the binding's argtypes stay as they are
    L.advisor_model_create.argtypes = [P, i32, P]
    L.advisor_model_destroy.argtypes = [P]
    L.advisor_rank_staged.argtypes = [P, P, P, i64, P, i64, i32, f32, f32, P, P, P, P, i32, P]
    L.advisor_rank_topn.argtypes = [P, P, i64, P, i64, i32, i32, f32, f32, P, P, P, P, P]
    L.advisor_model_check_wait_timeout.argtypes = [P, i64, P]
    L.advisor_plan_launch.argtypes = [P, P]
    L.advisor_get_rescore_counts.argtypes = [P, P, P]
    h = ctypes.c_void_p()
    arr = (ctypes.c_int32 * 4)(32, 128, 128, 1)
    assert L.advisor_model_create(ctypes.cast(arr, ctypes.c_void_p), 4, ctypes.byref(h)) == 0
    dev = ctypes.c_void_p(256)   # never dereferenced: every call below is refused first
    for stages in (0, 17):       # 1 .. ADVISOR_MAX_STAGES
        assert L.advisor_rank_staged(h, dev, dev, 10, dev, 1, 1, -1.0, 0.0, dev, dev, None, None, stages, None) == 1
    for n in (0, 129):           # 1 .. ADVISOR_MAX_TOP_N
        assert L.advisor_rank_topn(h, dev, 10, dev, 1, n, 1, -1.0, 0.0, dev, dev, None, None, None) == 1
    assert L.advisor_model_check_wait_timeout(None, 1000000, None) == 1
    assert L.advisor_model_check_wait_timeout(h, 1000000, None) == 1   # unbound model
    assert L.advisor_plan_launch(None, None) == 1
    assert L.advisor_get_rescore_counts(h, None, None) == 1
    assert L.advisor_model_destroy(h) == 0
