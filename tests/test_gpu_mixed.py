"""Mixed precision (FP32 kappa-cycles inside FP64 iterative refinement) against the FP64 oracle.

The oracle computes in FP64, so the FP32 cycle is judged by how far it lands from the FP64 cycle,
and the refined solution by the criteria of the mixed-precision workload:
* binding: the oracle recomputes ||f - A x|| / ||f|| of the GPU result in FP64 and it is <= tol;
* stated: ||x - x*|| / ||x*|| against the oracle solved to 1e-13 (asserted only loosely, printed).

FP32 cycle bound. A worst-case bound for one FP32 cycle from zero is u32 * cond(A_l) relative
(u32 = 6e-8; for kappa > 1 the second coarse call at level l starts from a nonzero iterate and
forms its residual by cancellation), about 0.8 u32 n_l^2: 0.2 at 4095^2, no bound at all. The
bound used instead is calibrated on the oracle itself: the same oracle steps run on float32 data
(its work arrays take the input's dtype; FP32 stencils, the coarsest solve in FP64 as on the
device) give the size of FP32 rounding in exactly this cycle. The device's FP32 cycle must land
within CAL_FACTOR times that distance from the FP64 cycle, norm-wise and element-wise, plus a
floor of 16 u32. Two correct FP32 roundings of the same cycle differ from FP64 by similar amounts
(the dominant part is the smooth error of the coarse calls, of the same size for both); a wrong
stencil entry, transfer weight, recursion step or tile edge adds an error of order 1 in some
points and fails. Observed for the oracle: 1e-7 (kappa = 1) and 4e-4 to 5e-4 (kappa = 3, 4) at
1023^2.
"""
import math

import numpy as np
import pytest

import oracle
from parity import rel  # norm-wise and element-wise (tests/parity.py)
from paper_2010_00626_b300.inputs import KAPPA_W, rhs_normal, rhs_uniform

pytestmark = pytest.mark.gpu

F32_CYCLE_TOL = 1e-4  # loose sanity bound beside the calibrated one
CAL_FACTOR = 4.0
U32 = 2.0 ** -24


def oracle_fp32_cycle(h, f, kappa):
    """The oracle's cycle on float32 data: FP32 stencils, FP32 arrays, the coarsest solve in FP64
    rounded to FP32 (as the device does it)."""
    import copy
    h32 = copy.copy(h)
    h32.stencils = [s.astype(np.float32) for s in h.stencils]
    solve64 = h.coarsest_solve
    h32.coarsest_solve = lambda fc: solve64(fc.astype(np.float64)).astype(np.float32)
    return oracle.cycle(h32, np.zeros(f.shape, np.float32), f.astype(np.float32), kappa).astype(np.float64)


def dev(a, dtype="float64"):
    import torch
    return torch.tensor(a, dtype=getattr(torch, dtype), device="cuda")


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()




@pytest.mark.parametrize("n,levels,theta,eps,kappa", [
    (127, 7, math.pi / 6, 1e-2, 1), (127, 7, math.pi / 6, 1e-2, 3), (127, 7, math.pi / 6, 1e-2, KAPPA_W),
    (127, 6, math.pi / 6, 1e-2, 2), (255, 8, 2.2, 1e-5, 1), (255, 8, 2.2, 1e-5, 4), (255, 8, 2.2, 1e-5, KAPPA_W),
    (1023, 10, 0.7, 1e-3, 1), (1023, 10, 0.7, 1e-3, 3), (1023, 10, 0.7, 1e-3, 4), (2047, 11, 2.0, 1e-5, 3),
    (4095, 12, math.pi / 3, 1e-4, 1), (4095, 12, math.pi / 3, 1e-4, 3), (4095, 12, math.pi / 3, 1e-4, 4)])
def test_fp32_cycle_close_to_fp64_oracle(lib, n, levels, theta, eps, kappa):
    """One FP32 cycle from zero (the inner cycle of the mixed forms) against the FP64 oracle, within
    CAL_FACTOR times the distance of the oracle's own FP32 rendition (norm-wise and element-wise)."""
    from parity import rel_elem, rel_l2
    h = oracle.Hierarchy(n, levels, theta, eps)
    f = rhs_uniform(n, 0)
    k = levels + 1 if kappa == KAPPA_W else kappa
    mg = lib.Multigrid(n, eps, theta, levels)
    v32 = dev(np.zeros((n, n)), "float32")
    mg.kcycle_f32(v32, dev(f, "float32"), kappa)
    got = host(v32)
    ref = oracle.cycle(h, np.zeros((n, n)), f, k)
    cal = oracle_fp32_cycle(h, f, k)
    floor = 16 * U32
    l2, el = rel_l2(got, ref), rel_elem(got, ref)
    l2_cal, el_cal = rel_l2(cal, ref), rel_elem(cal, ref)
    print(f"n={n} kappa={kappa}: device {l2:.2e} / {el:.2e}, oracle FP32 {l2_cal:.2e} / {el_cal:.2e} (L2 / max)")
    assert l2 <= CAL_FACTOR * l2_cal + floor, (l2, l2_cal)
    assert el <= CAL_FACTOR * el_cal + floor, (el, el_cal)
    if k == 1 or n <= 255:
        assert rel(got, ref) <= F32_CYCLE_TOL


@pytest.mark.parametrize("n,levels,kappa", [(1023, 10, 3), (2047, 11, 1), (4095, 12, 4)])
def test_fp32_cycle_tensor_copy_passes_and_tile_passes_agree(lib, n, levels, kappa):
    """The large-level FP32 passes exist twice: persistent kernels fed by tensor copies (default)
    and the shared-memory tile / register-pipeline kernels (MG_OPT_TMA_PASSES = 0). Both must meet
    the calibrated FP32 bound against the FP64 oracle, and a few cycles of each stay together
    (a wrong tile edge in either would separate them element-wise)."""
    from parity import rel_elem, rel_l2
    theta, eps = 2.4, 3e-4
    h = oracle.Hierarchy(n, levels, theta, eps)
    f = rhs_uniform(n, 5)
    ref = oracle.cycle(h, np.zeros((n, n)), f, kappa)
    cal = oracle_fp32_cycle(h, f, kappa)
    mg = lib.Multigrid(n, eps, theta, levels)
    out = {}
    for tma in (1, 0):
        mg.set_option(lib.MG_OPT_TMA_PASSES, tma)
        v32 = dev(np.zeros((n, n)), "float32")
        mg.kcycle_f32(v32, dev(f, "float32"), kappa)
        got = host(v32)
        assert rel_l2(got, ref) <= CAL_FACTOR * rel_l2(cal, ref) + 16 * U32, tma
        assert rel_elem(got, ref) <= CAL_FACTOR * rel_elem(cal, ref) + 16 * U32, tma
        out[tma] = got
    assert mg.get_option(lib.MG_OPT_TMA_PASSES) == 0
    d = rel(out[1], out[0])
    print(f"n={n} kappa={kappa}: tensor-copy vs tile passes {d:.2e}")
    assert d <= 2 * CAL_FACTOR * rel_l2(cal, ref) + 16 * U32


@pytest.mark.parametrize("kappa", [1, 2, 3, KAPPA_W])
def test_mixed_solve_small_meets_tolerance_and_error(lib, kappa):
    n, levels, theta, eps = 127, 7, math.pi / 6, 1e-2
    h = oracle.Hierarchy(n, levels, theta, eps)
    f = rhs_uniform(n, 0)
    k = levels + 1 if kappa == KAPPA_W else kappa
    x_star, _ = oracle.solve(h, f, k, 1e-13, 1000)
    _, hist64 = oracle.solve(h, f, k, 1e-8, 1000)
    mg = lib.Multigrid(n, eps, theta, levels)
    xd = dev(np.zeros((n, n)))
    st, iters, relres, hist = mg.solve_mixed(xd, dev(f), kappa, 1e-8, 1000)
    x = host(xd)
    assert st == 0 and relres <= 1e-8
    assert oracle.relres(h, x, f) <= 1e-8 * (1 + 1e-6)          # binding criterion, FP64 oracle
    assert abs(iters - len(hist64)) <= max(2, len(hist64) // 5)  # FP32 cycles converge like FP64 ones
    err = rel(x, x_star)
    print(f"kappa={kappa}: {iters} iterations (FP64 cycles {len(hist64)}), error vs oracle {err:.2e}")
    assert err <= 1e-6


def test_mixed_solve_large(lib):
    """4095^2, 12 levels, theta=pi/3, eps=1e-4: the oracle recomputes the residual of the result."""
    n, levels, theta, eps = 4095, 12, math.pi / 3, 1e-4
    h = oracle.Hierarchy(n, levels, theta, eps)
    f = rhs_normal(n, 0)
    mg = lib.Multigrid(n, eps, theta, levels)
    xd = dev(np.zeros((n, n)))
    st, iters, relres, hist = mg.solve_mixed(xd, dev(f), 4, 1e-8, 3000)
    assert st == 0 and relres <= 1e-8
    assert oracle.relres(h, host(xd), f) <= 1e-8 * (1 + 1e-6)


def test_tensor_copy_wait_runs_out_and_reports_timeout(lib):
    """Bounded waits: with the test hook, one CTA of the FP32 tensor-copy pass A at level 0 arms its
    copy barrier for a tile whose copy is never issued. Its wait runs out after the limit, it
    records the timeout and returns; the solve reports MG_ERR_TIMEOUT (-4) once, and the same handle
    then solves as a fresh handle does, bit for bit (the context stays usable)."""
    import time
    n, levels, theta, eps = 1023, 10, math.pi / 3, 1e-4
    f = rhs_normal(n, 0)
    mg = lib.Multigrid(n, eps, theta, levels)
    mg.set_option(lib.MG_OPT_TEST_STALL_COPY, 3)
    assert mg.get_option(lib.MG_OPT_TEST_STALL_COPY) == 3
    t0 = time.perf_counter()
    with pytest.raises(lib.MultigridError, match=r"\(-4\)"):
        mg.solve_mixed(dev(np.zeros((n, n))), dev(f), 1, 1e-8, 1)
    waited = time.perf_counter() - t0
    mg.set_option(lib.MG_OPT_TEST_STALL_COPY, -1)
    xd = dev(np.zeros((n, n)))
    st, iters, relres, _ = mg.solve_mixed(xd, dev(f), 3, 1e-8, 300)
    fresh = lib.Multigrid(n, eps, theta, levels)
    xe = dev(np.zeros((n, n)))
    st2, iters2, relres2, _ = fresh.solve_mixed(xe, dev(f), 3, 1e-8, 300)
    print(f"timed-out solve took {waited:.2f} s; then {iters} iterations")
    assert st == 0 and st2 == 0 and iters == iters2 and relres == relres2
    assert np.array_equal(host(xd), host(xe))
    with pytest.raises(lib.MultigridError):
        mg.set_option(lib.MG_OPT_TEST_STALL_COPY, -2)


def test_mixed_solve_not_converged_and_bad_args(lib):
    n = 63
    mg = lib.Multigrid(n, 1e-4, 1.0, 6)
    f = rhs_uniform(n, 1)
    st, iters, relres, hist = mg.solve_mixed(dev(np.zeros((n, n))), dev(f), 1, 1e-12, 2)
    assert st == 1 and iters == 2 and len(hist) == 2
    with pytest.raises(lib.MultigridError):
        mg.solve_mixed(dev(np.zeros((n, n))), dev(f), 0, 1e-8, 5)


@pytest.mark.parametrize("kappa,flexible", [(1, True), (3, True), (3, False)])
def test_mixed_pcg_small(lib, kappa, flexible):
    n, levels, theta, eps = 255, 8, 2.0, 1e-3
    h = oracle.Hierarchy(n, levels, theta, eps)
    b = rhs_normal(n, 7)
    _, hist64 = oracle.pcg(h, b, kappa, 1e-10, 300, flexible=flexible)
    mg = lib.Multigrid(n, eps, theta, levels)
    xd = dev(np.zeros((n, n)))
    st, iters, relres, hist = mg.pcg(xd, dev(b), kappa, 1e-10, 300, flexible=flexible, mixed=True)
    assert st == 0 and relres <= 1e-10
    assert oracle.relres(h, host(xd), b) <= 1e-10 * (1 + 1e-5)
    assert abs(iters - len(hist64)) <= max(2, len(hist64) // 5)


def test_pcg_large_fp64_and_mixed(lib):
    """8191^2, 13 levels, theta from seed 0, eps=1e-5, kappa=3, tol 1e-10: FP64 and mixed MGCG;
    the oracle recomputes both residuals in FP64."""
    from paper_2010_00626_b300.inputs import pcg_theta
    n, levels, eps = 8191, 13, 1e-5
    theta = pcg_theta(0)
    h = oracle.Hierarchy(n, levels, theta, eps)
    b = rhs_normal(n, 0)
    mg = lib.Multigrid(n, eps, theta, levels)
    bd = dev(b)
    results = {}
    for mixed in (False, True):
        xd = dev(np.zeros((n, n)))
        st, iters, relres, _ = mg.pcg(xd, bd, 3, 1e-10, 1000, flexible=True, mixed=mixed, history=False)
        assert st == 0 and relres <= 1e-10
        assert oracle.relres(h, host(xd), b) <= 1e-10 * (1 + 1e-5)
        results[mixed] = iters
        del xd
    assert abs(results[True] - results[False]) <= max(2, results[False] // 5), results
