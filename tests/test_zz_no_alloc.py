"""The allocation-free residual norm against the handle-based one (needs a B300).

mg_residual_norm_noalloc serves callers that may not allocate device memory when they need the
number (a framework owns the memory pool, the host application forbids device allocation, or the
loop cannot take an allocation's device-wide synchronisation). Its scratch is a static device
array in the library, so this file is collected last: if it fails, every other test has run.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2010_00626_b300.inputs import rhs_normal, rhs_uniform

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12  # the tolerance the other residual-norm test uses


@pytest.mark.parametrize("n", [1, 7, 511, 4095])
def test_noalloc_residual_norm_matches_handle_entry_point_twice(lib, n):
    """n = 1: every neighbour is a boundary zero; n = 7: almost all of the fixed 592 blocks write a
    zero partial (49 points); 511 and 4095: every block sums points, 4095^2 over many grid strides."""
    import torch
    levels = max(1, int(round(math.log2(n + 1))) - 2)
    theta, eps = 1.3, 1e-4
    mg = lib.Multigrid(n, eps, theta, levels)
    stream = torch.cuda.current_stream().cuda_stream or lib.CUDA_STREAM_LEGACY
    for seed in (0, 1):  # two calls in a row: the second must not see the first's scratch
        v = torch.tensor(rhs_normal(n, 20 + seed) * (1.0 + seed), device="cuda")
        f = torch.tensor(rhs_uniform(n, 30 + seed), device="cuda")
        ref = mg.residual_norm(v, f)
        out = ctypes.c_double(-1.0)
        st = lib._lib.mg_residual_norm_noalloc(n, eps, theta, ctypes.c_void_p(v.data_ptr()),
                                               ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(stream),
                                               ctypes.byref(out))
        assert st == 0, lib._lib.mg_last_error()
        assert abs(out.value - ref) <= REL_TOL * ref, (seed, out.value, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    import torch
    v = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = ctypes.c_double()
    st = lib._lib.mg_residual_norm_noalloc(32767, 1e-2, 0.5, ctypes.c_void_p(v.data_ptr()),
                                           ctypes.c_void_p(v.data_ptr()), None, ctypes.byref(out))
    assert st == -1
    assert b"exceeds the maximum grid side" in lib._lib.mg_last_error()
    for eps, theta in ((0.0, 0.5), (1.5, 0.5), (1e-2, 2e4)):
        st = lib._lib.mg_residual_norm_noalloc(7, eps, theta, ctypes.c_void_p(v.data_ptr()),
                                               ctypes.c_void_p(v.data_ptr()), None, ctypes.byref(out))
        assert st == -1
        assert b"need 0 < eps <= 1" in lib._lib.mg_last_error()
