"""GPU parity of the alternating zebra line relaxation (Section 4, solvers 3-4) against the oracle.

The device solves every line with Thomas factors tabulated per level and a chunked scan, the
oracle with a banded LU per line: two orderings of the same exact solve, which agree to the
first-order forward error of a line solve, u * kappa_line (u = 2^-52 here, kappa_line the largest
condition number of a line operator over the levels and both directions, computed from the
oracle's stencils). Iterates must agree to max(1e-12, u * kappa_line): 1e-12 for the well
conditioned cases, up to about 4e-11 where the lines are nearly singular (theta = 0 or 90 degrees
with eps = 1e-5, kappa_line up to 1.8e5 at 4095^2). Histories and MGCG use the bounds of the
Jacobi tests with that iterate bound.
"""
import math

import numpy as np
import pytest

import oracle
from parity import rel  # norm-wise and element-wise (tests/parity.py)
from paper_2010_00626_b300.inputs import KAPPA_W, rhs_normal, rhs_uniform

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-12
HIST_TOL = 1e-10
U = 2.0 ** -52


def line_cond(h):
    """Largest condition number of the tridiagonal line operators tridiag(a, d, a) of the
    hierarchy: eigenvalues d + 2 a cos(j pi / (n + 1)), j = 1..n."""
    worst = 1.0
    for l, n in enumerate(h.sizes, start=1):
        st = h.stencil(l)
        d = st[1, 1]
        for a in (st[1, 0], st[0, 1]):
            lo = d - 2 * abs(a) * math.cos(math.pi / (n + 1))
            hi = d + 2 * abs(a) * math.cos(math.pi / (n + 1))
            worst = max(worst, hi / lo)
    return worst


def iter_tol(h):
    return max(ITER_TOL, U * line_cond(h))


def torch_dev(a):
    import torch
    return torch.tensor(a, dtype=torch.float64, device="cuda")


def to_np(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()




def hist_ok(h_gpu, h_orc, h, vs, f):
    anorm = np.abs(h.stencil(1)).sum()
    fn = np.linalg.norm(f)
    for k, (a, b) in enumerate(zip(h_gpu, h_orc)):
        floor = iter_tol(h) * anorm * np.linalg.norm(vs[k]) / fn
        assert abs(a - b) <= HIST_TOL * b + floor, (k, a, b)


DEG = math.pi / 180


@pytest.mark.parametrize("n,levels,theta,eps", [
    (127, 7, math.pi / 6, 1e-2), (127, 7, 0.0, 1e-5), (255, 8, 10 * DEG, 1e-5), (511, 9, 45 * DEG, 1e-5),
    (1023, 10, 80 * DEG, 1e-3), (1023, 10, 0.0, 1e-5), (1023, 10, 90 * DEG, 1e-5), (511, 6, 30 * DEG, 1e-4)])
def test_zebra_cycles_per_iterate(lib, n, levels, theta, eps):
    """Four cycles with counters 1, 3, 2, 4 from zero: lines of 511 and more points span
    several 512-point segments; 127 and 255 use chunks of 4 and 8 points; 31 and 63 one and two."""
    h = oracle.Hierarchy(n, levels, theta, eps, smoother="zebra")
    f = rhs_uniform(n, 0)
    mg = lib.Multigrid(n, eps, theta, levels, smoother="zebra")
    fd, vd = torch_dev(f), torch_dev(np.zeros((n, n)))
    v = np.zeros((n, n))
    for c, kappa in enumerate((1, 3, 2, 4)):
        v = oracle.cycle(h, v, f, kappa)
        mg.kcycle(vd, fd, kappa)
        err = rel(to_np(vd), v)
        assert err <= iter_tol(h), (c, err, iter_tol(h))


@pytest.mark.parametrize("n,levels,theta,eps", [(4095, 12, 0.0, 1e-5), (2047, 11, 60 * DEG, 1e-5)])
def test_zebra_large_one_cycle(lib, n, levels, theta, eps):
    """One kappa = 2 cycle from a nonzero start at the full sizes (eight and four segments per line)."""
    h = oracle.Hierarchy(n, levels, theta, eps, smoother="zebra")
    f = rhs_uniform(n, 1)
    v0 = rhs_normal(n, 2) * 1e-3
    mg = lib.Multigrid(n, eps, theta, levels, smoother="zebra")
    vd = torch_dev(v0)
    mg.kcycle(vd, torch_dev(f), 2)
    assert rel(to_np(vd), oracle.cycle(h, v0, f, 2)) <= iter_tol(h)


@pytest.mark.parametrize("coarse_n", [1, 3, 7, 15, 31, 63])
def test_zebra_coarse_threshold_does_not_change_iterates(lib, coarse_n):
    """The single-CTA coarse kernel runs its own line solves (one thread per line); moving the
    threshold moves levels between it and the line kernels."""
    n, levels, theta, eps = 63, 6, 1.1, 1e-3
    h = oracle.Hierarchy(n, levels, theta, eps, smoother="zebra")
    f = rhs_normal(n, 3)
    mg = lib.Multigrid(n, eps, theta, levels, coarse_n=coarse_n, smoother="zebra")
    fd, vd = torch_dev(f), torch_dev(np.zeros((n, n)))
    v = np.zeros((n, n))
    for kappa in (3, 1, 6, 2):
        v = oracle.cycle(h, v, f, kappa)
        mg.kcycle(vd, fd, kappa)
        assert rel(to_np(vd), v) <= iter_tol(h)


@pytest.mark.parametrize("nu", [(2, 2), (1, 1), (3, 1), (0, 2), (2, 0), (4, 4)])
def test_zebra_relaxation_counts(lib, nu):
    n, levels, theta, eps = 127, 7, 20 * DEG, 1e-4
    h = oracle.Hierarchy(n, levels, theta, eps, nu1=nu[0], nu2=nu[1], smoother="zebra")
    f = rhs_normal(n, 6)
    mg = lib.Multigrid(n, eps, theta, levels, nu1=nu[0], nu2=nu[1], smoother="zebra")
    fd = torch_dev(f)
    for kappa in (1, 3):
        vd = torch_dev(np.zeros((n, n)))
        mg.kcycle(vd, fd, kappa)
        assert rel(to_np(vd), oracle.cycle(h, np.zeros((n, n)), f, kappa)) <= iter_tol(h)


@pytest.mark.parametrize("n,levels", [(1, 1), (3, 2), (7, 3), (15, 4), (31, 5)])
def test_zebra_tiny_grids(lib, n, levels):
    theta, eps = 0.3, 1e-3
    h = oracle.Hierarchy(n, levels, theta, eps, smoother="zebra")
    f = rhs_uniform(n, 4)
    v0 = rhs_normal(n, 5) * 1e-3
    mg = lib.Multigrid(n, eps, theta, levels, smoother="zebra")
    fd, vd = torch_dev(f), torch_dev(v0)
    v = v0.copy()
    for kappa in (2, 4):
        v = oracle.cycle(h, v, f, kappa)
        mg.kcycle(vd, fd, kappa)
        assert rel(to_np(vd), v) <= iter_tol(h)


@pytest.mark.parametrize("theta", [10 * DEG, 45 * DEG, 0.0])
@pytest.mark.parametrize("kappa", [1, 2, 4, KAPPA_W])
def test_zebra_solve_history_matches_oracle(lib, theta, kappa):
    """Stand-alone solves at eps = 1e-5 (the Table 6 anisotropy) on 255^2."""
    n, levels, eps = 255, 8, 1e-5
    h = oracle.Hierarchy(n, levels, theta, eps, smoother="zebra")
    f = rhs_uniform(n, 0)
    k = levels + 1 if kappa == KAPPA_W else kappa
    v_or, hist_or = oracle.solve(h, f, k, 1e-8, 500)
    vs, v = [], np.zeros_like(f)
    for _ in range(len(hist_or)):
        v = oracle.cycle(h, v, f, k)
        vs.append(v)
    mg = lib.Multigrid(n, eps, theta, levels, smoother="zebra")
    vd = torch_dev(np.zeros((n, n)))
    st, cycles, relres, hist = mg.solve(vd, torch_dev(f), kappa, 1e-8, 500)
    assert st == 0 and cycles == len(hist_or)
    hist_ok(hist, hist_or, h, vs, f)
    assert rel(to_np(vd), v_or) <= iter_tol(h)
    assert oracle.relres(h, to_np(vd), f) <= 1e-8


@pytest.mark.parametrize("kappa,flexible", [(1, False), (4, False), (2, True), (KAPPA_W, False)])
def test_zebra_pcg_matches_oracle(lib, kappa, flexible):
    """MGCG with the zebra cycle (Table 7's solver). The cycle is not symmetric (x then y in both
    smoothing steps), which the flexible beta tolerates; both forms match the oracle."""
    n, levels, theta, eps = 255, 8, 30 * DEG, 1e-5
    h = oracle.Hierarchy(n, levels, theta, eps, smoother="zebra")
    b = rhs_uniform(n, 7)
    k = levels + 1 if kappa == KAPPA_W else kappa
    x_or, hist_or = oracle.pcg(h, b, k, 1e-10, 200, flexible=flexible)
    mg = lib.Multigrid(n, eps, theta, levels, smoother="zebra")
    xd = torch_dev(np.zeros((n, n)))
    st, iters, relres, hist = mg.pcg(xd, torch_dev(b), kappa, 1e-10, 200, flexible=flexible)
    assert st == 0 and iters == len(hist_or)
    for a, c in zip(hist, hist_or):
        assert abs(a - c) <= HIST_TOL * c + 1e-13
    assert rel(to_np(xd), x_or) <= 1e-10


def test_zebra_grid_aligned_anisotropy_large(lib):
    """theta = 0, eps = 1e-5 at 4095^2: damped point Jacobi cannot smooth this case (Section 4);
    the zebra cycle reaches 1e-8 in a handful of cycles, and the oracle confirms the residual."""
    n, levels = 4095, 12
    f = rhs_uniform(n, 0)
    mg = lib.Multigrid(n, 1e-5, 0.0, levels, smoother="zebra")
    vd = torch_dev(np.zeros((n, n)))
    st, cycles, relres, hist = mg.solve(vd, torch_dev(f), 4, 1e-8, 50)
    assert st == 0 and cycles <= 10
    h = oracle.Hierarchy(n, levels, 0.0, 1e-5, smoother="zebra")
    assert oracle.relres(h, to_np(vd), f) <= 1e-8


def test_zebra_mixed_precision_solve(lib):
    """FP32 zebra cycles inside FP64 iterative refinement: the FP64 residual reaches 1e-10 and the
    iteration count stays within two of the FP64 solve's."""
    n, levels, theta, eps = 1023, 10, 10 * DEG, 1e-5
    f = rhs_uniform(n, 8)
    mg = lib.Multigrid(n, eps, theta, levels, smoother="zebra")
    vd = torch_dev(np.zeros((n, n)))
    st64, c64, _, _ = mg.solve(vd, torch_dev(f), 3, 1e-10, 200)
    xd = torch_dev(np.zeros((n, n)))
    st32, c32, _, _ = mg.solve_mixed(xd, torch_dev(f), 3, 1e-10, 200)
    assert st64 == 0 and st32 == 0 and abs(c32 - c64) <= 2
    h = oracle.Hierarchy(n, levels, theta, eps, smoother="zebra")
    assert oracle.relres(h, to_np(xd), f) <= 1e-10


def test_zebra_rejects_adjoint_and_switches_back(lib):
    n, levels, theta, eps = 63, 6, 0.5, 1e-2
    mg = lib.Multigrid(n, eps, theta, levels, smoother="zebra")
    f = rhs_normal(n, 9)
    vd = torch_dev(np.zeros((n, n)))
    with pytest.raises(lib.MultigridError):
        mg.kcycle_adjoint(vd, torch_dev(f), 2)
    with pytest.raises(lib.MultigridError):
        mg.solve(vd, torch_dev(f), 2, 1e-8, 10, adjoint=True)
    assert mg.get_option(lib.MG_OPT_SMOOTHER) == 1
    mg.set_option(lib.MG_OPT_SMOOTHER, 0)   # back to damped Jacobi: the cached graphs are rebuilt
    h = oracle.Hierarchy(n, levels, theta, eps)
    vd = torch_dev(np.zeros((n, n)))
    mg.kcycle(vd, torch_dev(f), 3)
    assert rel(to_np(vd), oracle.cycle(h, np.zeros((n, n)), f, 3)) <= ITER_TOL
    with pytest.raises(lib.MultigridError):
        mg.set_option(lib.MG_OPT_SMOOTHER, 3)


@pytest.mark.parametrize("kappa", [1, 3, KAPPA_W])
@pytest.mark.parametrize("nu", [(2, 2), (0, 2), (2, 0)])
def test_zebra_counters_match_graph(lib, kappa, nu):
    n, levels = 1023, 10
    mg = lib.Multigrid(n, 1e-4, 0.4, levels, nu1=nu[0], nu2=nu[1], smoother="zebra")
    calls, launches, coarse = mg.counters(kappa)
    mg.kcycle(torch_dev(np.zeros((n, n))), torch_dev(rhs_normal(n, 0)), kappa)
    assert mg.get_option(lib.MG_OPT_LAUNCHES) == launches
