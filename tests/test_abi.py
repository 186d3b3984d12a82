"""The C-ABI library loads and exports every symbol include/kcycle.h declares (CPU only).

No compute calls: only argument checks that return before any CUDA call is made.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "kcycle.h")).read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(mg_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def libk():
    from paper_2010_00626_b300 import build
    build.build()
    from paper_2010_00626_b300 import kcycle
    return kcycle


def test_header_declares_expected_entry_points():
    syms = declared_symbols()
    for name in ("mg_setup", "mg_kcycle", "mg_solve", "mg_pcg", "mg_destroy", "mg_kcycle_adjoint"):
        assert name in syms


def test_library_exports_every_declared_symbol(libk):
    lib = ctypes.CDLL(libk.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(declared_symbols()) <= set(libk.SIGNATURES)


def test_setup_rejects_bad_arguments_without_touching_the_gpu(libk):
    lib = libk._lib
    h = ctypes.c_void_p()
    bad = [
        (100, 1e-2, 0.5, 3, 2, 2),    # n not 2^k - 1
        (127, 1e-2, 0.5, 8, 2, 2),    # levels > k
        (127, 1e-2, 0.5, 2, 2, 2),    # coarsest grid 31 > 15
        (127, 0.0, 0.5, 7, 2, 2),     # eps <= 0
        (127, 1.5, 0.5, 7, 2, 2),     # eps > 1
        (127, float("nan"), 0.5, 7, 2, 2),
        (127, 1e-2, float("inf"), 7, 2, 2),
        (127, 1e-2, 0.5, 7, -1, 2),
        (127, 1e-2, 0.5, 7, 2, 9),
    ]
    for args in bad:
        assert lib.mg_setup(*args, ctypes.byref(h)) == -1, args
        assert not h.value
    assert lib.mg_kcycle(None, None, None, 1) == -5
    assert lib.mg_set_option(None, 9, 1.0) == -5      # MG_OPT_SMOOTHER on no handle
    assert lib.mg_batch_set_option(None, 9, 1.0) == -1
    n_l, ctas = ctypes.c_int(), ctypes.c_int()
    assert lib.mg_level_grid(None, 0, 0, ctypes.byref(n_l), ctypes.byref(ctas)) == -5
    assert lib.mg_destroy(None) == 0
    assert lib.mg_status_string(-1) == b"invalid argument"
