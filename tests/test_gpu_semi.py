"""GPU parity of y semi-coarsening with x-line zebra relaxation (Section 4, solvers 5-6).

Stencils are compared bit for bit: each semi-coarsened Galerkin entry is a sum of the fine entries
times powers of two, rounded once on both sides. Iterates are held to max(1e-12, 2^-52 kappa_x),
kappa_x the largest condition number of the x-line operators (the device's tabulated Thomas solve
and the oracle's banded LU are two roundings of the same exact solves; the derivation is in
tests/test_gpu_zebra.py).
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
DEG = math.pi / 180


def torch_dev(a):
    import torch
    return torch.tensor(a, dtype=torch.float64, device="cuda")


def to_np(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()




def iter_tol(h):
    worst = 1.0
    for l in range(1, h.levels + 1):
        st = h.stencil(l)
        d, a = st[1, 1], abs(st[1, 0])
        c = math.cos(math.pi / (h.n + 1))
        worst = max(worst, (d + 2 * a * c) / (d - 2 * a * c))
    return max(ITER_TOL, U * worst)


def semi(n, theta, eps, **kw):
    return oracle.Hierarchy(n, int(round(math.log2(n + 1))), theta, eps, smoother="xzebra", coarsening="y", **kw)


@pytest.mark.parametrize("n,theta,eps", [(63, 0.0, 1e-5), (127, 90 * DEG, 1e-5), (255, 45 * DEG, 1e-3),
                                         (1023, 10 * DEG, 1e-5), (4095, 30 * DEG, 1e-4)])
def test_semi_stencils_bitwise(lib, n, theta, eps):
    h = semi(n, theta, eps)
    mg = lib.Multigrid(n, eps, theta, h.levels, coarsening="y")
    st = mg.stencils()
    for l in range(h.levels):
        assert np.array_equal(st[l], h.stencils[l]), (l, st[l] - h.stencils[l])


@pytest.mark.parametrize("n,theta,eps", [(63, 0.0, 1e-5), (127, 90 * DEG, 1e-5), (255, 45 * DEG, 1e-3),
                                         (511, 10 * DEG, 1e-5), (1023, 80 * DEG, 1e-4)])
def test_semi_cycles_per_iterate(lib, n, theta, eps):
    """Four cycles with counters 1, 3, 2, 4 from zero; rows of 511 and more points span several
    512-point segments, and the coarsest level is a single row."""
    h = semi(n, theta, eps)
    f = rhs_uniform(n, 0)
    mg = lib.Multigrid(n, eps, theta, h.levels, coarsening="y")
    fd, vd = torch_dev(f), torch_dev(np.zeros((n, n)))
    v = np.zeros((n, n))
    for c, kappa in enumerate((1, 3, 2, 4)):
        v = oracle.cycle(h, v, f, kappa)
        mg.kcycle(vd, fd, kappa)
        err = rel(to_np(vd), v)
        assert err <= iter_tol(h), (c, err, iter_tol(h))


def test_semi_large_one_cycle(lib):
    n, theta, eps = 4095, 60 * DEG, 1e-5
    h = semi(n, theta, eps)
    f = rhs_uniform(n, 1)
    v0 = rhs_normal(n, 2) * 1e-3
    mg = lib.Multigrid(n, eps, theta, h.levels, coarsening="y")
    vd = torch_dev(v0)
    mg.kcycle(vd, torch_dev(f), 2)
    assert rel(to_np(vd), oracle.cycle(h, v0, f, 2)) <= iter_tol(h)


@pytest.mark.parametrize("nu", [(2, 2), (1, 1), (3, 1), (0, 2), (2, 0)])
def test_semi_relaxation_counts(lib, nu):
    n, theta, eps = 127, 20 * DEG, 1e-4
    h = semi(n, theta, eps, nu1=nu[0], nu2=nu[1])
    f = rhs_normal(n, 6)
    mg = lib.Multigrid(n, eps, theta, h.levels, nu1=nu[0], nu2=nu[1], coarsening="y")
    fd = torch_dev(f)
    for kappa in (1, 3):
        vd = torch_dev(np.zeros((n, n)))
        mg.kcycle(vd, fd, kappa)
        assert rel(to_np(vd), oracle.cycle(h, np.zeros((n, n)), f, kappa)) <= iter_tol(h)


@pytest.mark.parametrize("theta", [10 * DEG, 45 * DEG, 90 * DEG])
@pytest.mark.parametrize("kappa", [1, 2, 3, KAPPA_W])
def test_semi_solve_history_matches_oracle(lib, theta, kappa):
    n, eps = 255, 1e-5
    h = semi(n, theta, eps)
    f = rhs_uniform(n, 0)
    k = h.levels + 1 if kappa == KAPPA_W else kappa
    v_or, hist_or = oracle.solve(h, f, k, 1e-8, 500)
    vs, v = [], np.zeros_like(f)
    for _ in range(len(hist_or)):
        v = oracle.cycle(h, v, f, k)
        vs.append(v)
    mg = lib.Multigrid(n, eps, theta, h.levels, coarsening="y")
    vd = torch_dev(np.zeros((n, n)))
    st, cycles, relres, hist = mg.solve(vd, torch_dev(f), kappa, 1e-8, 500)
    assert st == 0 and cycles == len(hist_or)
    anorm, fn = np.abs(h.stencil(1)).sum(), np.linalg.norm(f)
    for i, (a, b) in enumerate(zip(hist, hist_or)):
        assert abs(a - b) <= HIST_TOL * b + iter_tol(h) * anorm * np.linalg.norm(vs[i]) / fn, (i, a, b)
    assert rel(to_np(vd), v_or) <= iter_tol(h)
    assert oracle.relres(h, to_np(vd), f) <= 1e-8


@pytest.mark.parametrize("kappa", [1, 2, 4])
def test_semi_pcg_matches_oracle(lib, kappa):
    """MGCG with the semi-coarsening cycle (Table 9's solver)."""
    n, theta, eps = 255, 30 * DEG, 1e-5
    h = semi(n, theta, eps)
    b = rhs_uniform(n, 7)
    x_or, hist_or = oracle.pcg(h, b, kappa, 1e-10, 200)
    mg = lib.Multigrid(n, eps, theta, h.levels, coarsening="y")
    xd = torch_dev(np.zeros((n, n)))
    st, iters, relres, hist = mg.pcg(xd, torch_dev(b), kappa, 1e-10, 200)
    assert st == 0 and iters == len(hist_or)
    for a, c in zip(hist, hist_or):
        assert abs(a - c) <= HIST_TOL * c + 1e-13
    assert rel(to_np(xd), x_or) <= 1e-10


@pytest.mark.parametrize("kappa", [1, 2, 3, KAPPA_W])
def test_semi_counters_match_graph(lib, kappa):
    n = 1023
    mg = lib.Multigrid(n, 1e-4, 0.4, 10, coarsening="y")
    calls, launches, coarse = mg.counters(kappa)
    k = 11 if kappa == KAPPA_W else kappa
    for l in range(10):
        assert calls[l] == sum(math.comb(l, j) for j in range(0, min(k - 1, l) + 1))
    assert coarse == 0
    mg.kcycle(torch_dev(np.zeros((n, n))), torch_dev(rhs_normal(n, 0)), kappa)
    assert mg.get_option(lib.MG_OPT_LAUNCHES) == launches


def test_semi_grid_aligned_both_ways_large(lib):
    """eps = 1e-5 with the strong direction along x (theta = 0) or y (90 degrees) at 4095^2:
    line relaxation covers the first, semi-coarsening the second."""
    n = 4095
    f = rhs_uniform(n, 0)
    for theta in (0.0, 90 * DEG):
        mg = lib.Multigrid(n, 1e-5, theta, 12, coarsening="y")
        vd = torch_dev(np.zeros((n, n)))
        st, cycles, relres, hist = mg.solve(vd, torch_dev(f), 2, 1e-8, 100)
        assert st == 0 and cycles <= 15, (theta, cycles)
        h = semi(n, theta, 1e-5)
        assert oracle.relres(h, to_np(vd), f) <= 1e-8


def test_semi_option_errors(lib):
    mg = lib.Multigrid(63, 1e-3, 0.4, 6)
    with pytest.raises(lib.MultigridError):
        lib.Multigrid(63, 1e-3, 0.4, 4, coarsening="y")        # levels must reach one row
    mg.set_option(lib.MG_OPT_COARSENING, 1)
    assert mg.get_option(lib.MG_OPT_SMOOTHER) == 2
    with pytest.raises(lib.MultigridError):
        mg.set_option(lib.MG_OPT_SMOOTHER, 0)
    with pytest.raises(lib.MultigridError):
        mg.set_option(lib.MG_OPT_COARSE_OP, 1)
    x, f = torch_dev(np.zeros((63, 63))), torch_dev(rhs_uniform(63, 0))
    with pytest.raises(lib.MultigridError):
        mg.solve_mixed(x, f, 2, 1e-8, 10)
    with pytest.raises(lib.MultigridError):
        mg.kcycle_adjoint(x, f, 2)
    mg.set_option(lib.MG_OPT_COARSENING, 0)                       # back to full coarsening, Jacobi
    assert mg.get_option(lib.MG_OPT_SMOOTHER) == 0
    h = oracle.Hierarchy(63, 6, 0.4, 1e-3)
    mg.kcycle(x, f, 3)
    assert rel(to_np(x), oracle.cycle(h, np.zeros((63, 63)), rhs_uniform(63, 0), 3)) <= ITER_TOL
