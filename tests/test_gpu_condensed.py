"""Condensed child calls (MG_OPT_CONDENSED_CHILDREN): the two calls that a call just above the
coarse-kernel level makes there, with everything below them, applied as one precomputed linear map
v = P_c f instead of the coarse kernel's walk (Algorithm 3's recursion is unchanged; only how
that subtree's linear map is evaluated). The map is the same linear map rounded differently, so
the FP64 cycle must keep the 1e-12 per-iterate parity with the oracle (norm-wise and element-wise)
either way, the FP32 cycle the calibrated FP32 bound, and the two evaluations must differ (the
path is really taken) by no more than rounding."""
import math

import numpy as np
import pytest

import oracle
from parity import rel, rel_elem, rel_l2
from paper_2010_00626_b300.inputs import KAPPA_W, rhs_normal, rhs_uniform

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-12
U32 = 2.0 ** -24


def dev(a, dtype="float64"):
    import torch
    return torch.tensor(a, dtype=getattr(torch, dtype), device="cuda")


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()


@pytest.mark.parametrize("n,levels,kappa", [(63, 6, 2), (127, 7, 3), (255, 8, KAPPA_W), (1023, 10, 4),
                                            (4095, 12, 4), (511, 9, 1)])
def test_fp64_cycles_condensed_and_walked_match_oracle(lib, n, levels, kappa):
    theta, eps = 1.9, 2e-4
    h = oracle.Hierarchy(n, levels, theta, eps)
    f = rhs_uniform(n, 11)
    k = levels + 1 if kappa == KAPPA_W else kappa
    out = {}
    for condense in (1, 0):
        mg = lib.Multigrid(n, eps, theta, levels)
        mg.set_option(lib.MG_OPT_CONDENSED_CHILDREN, condense)
        vd, fd = dev(np.zeros((n, n))), dev(f)
        v = np.zeros((n, n))
        for c in range(2 if n >= 4095 else 3):
            mg.kcycle(vd, fd, kappa)
            v = oracle.cycle(h, v, f, k)
            assert rel(host(vd), v) <= ITER_TOL, (condense, c)
        out[condense] = host(vd)
        mg.close()
    assert not np.array_equal(out[0], out[1])  # the condensed path was taken
    assert rel(out[1], out[0]) <= ITER_TOL


@pytest.mark.parametrize("n,levels,kappa", [(1023, 10, 3), (4095, 12, 4), (255, 8, 2)])
def test_fp32_cycles_condensed_within_calibrated_bound(lib, n, levels, kappa):
    """The FP32 maps are computed in FP64 and rounded once: the condensed FP32 cycle must stay
    within the bound of test_gpu_mixed (CAL_FACTOR x the oracle's own FP32 distance)."""
    from test_gpu_mixed import CAL_FACTOR, oracle_fp32_cycle
    theta, eps = 0.35, 1e-3
    h = oracle.Hierarchy(n, levels, theta, eps)
    f = rhs_normal(n, 12)
    ref = oracle.cycle(h, np.zeros((n, n)), f, kappa)
    cal = oracle_fp32_cycle(h, f, kappa)
    got = {}
    for condense in (1, 0):
        mg = lib.Multigrid(n, eps, theta, levels)
        mg.set_option(lib.MG_OPT_CONDENSED_CHILDREN, condense)
        v32 = dev(np.zeros((n, n)), "float32")
        mg.kcycle_f32(v32, dev(f, "float32"), kappa)
        got[condense] = host(v32)
        assert rel_l2(got[condense], ref) <= CAL_FACTOR * rel_l2(cal, ref) + 16 * U32, condense
        assert rel_elem(got[condense], ref) <= CAL_FACTOR * rel_elem(cal, ref) + 16 * U32, condense
        mg.close()
    assert not np.array_equal(got[0], got[1])


def test_condensed_solves_match_oracle_history_and_mixed_tolerance(lib):
    """Stand-alone FP64 solve (history within 1e-10 of the oracle's) and the mixed solve (the
    oracle recomputes the FP64 residual) with condensed child calls, 511^2."""
    n, levels, theta, eps, kappa = 511, 9, math.pi / 3, 1e-4, 3
    h = oracle.Hierarchy(n, levels, theta, eps)
    f = rhs_normal(n, 0)
    mg = lib.Multigrid(n, eps, theta, levels)
    assert mg.get_option(lib.MG_OPT_CONDENSED_CHILDREN) == 1
    xd = dev(np.zeros((n, n)))
    st, cycles, relres, hist = mg.solve(xd, dev(f), kappa, 1e-8, 2000)
    _, hist_or = oracle.solve(h, f, kappa, 1e-8, 2000)
    assert st == 0 and cycles == len(hist_or)
    for a, b in zip(hist, hist_or):
        assert abs(a - b) <= 1e-10 * b + 1e-13
    xm = dev(np.zeros((n, n)))
    st, iters, relres, _ = mg.solve_mixed(xm, dev(f), kappa, 1e-8, 2000)
    assert st == 0 and oracle.relres(h, host(xm), f) <= 1e-8 * (1 + 1e-6)
