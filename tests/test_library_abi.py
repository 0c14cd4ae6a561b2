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
