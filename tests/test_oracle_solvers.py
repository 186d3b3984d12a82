"""Pins of the oracle's solvers and gradients (CPU only).

* MGCG against scipy's preconditioned CG with the same kappa-cycle as preconditioner;
* parameter gradients against central finite differences of the loss through a dense solve;
* the stand-alone history against residuals recomputed from the iterates.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse.linalg as spla

import oracle
from paper_2010_00626_b300.inputs import rhs_normal, rhs_uniform


def dense_A(st, n):
    cols = []
    for k in range(n * n):
        e = np.zeros(n * n)
        e[k] = 1.0
        cols.append(oracle.apply_stencil(st, e.reshape(n, n)).ravel())
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("kappa", [1, 6])
def test_pcg_matches_scipy_cg_iterate_for_iterate(kappa):
    """Symmetric preconditioners (V and W): the oracle's MGCG is textbook PCG, so its
    iterates equal scipy's cg run with the same preconditioner for the same count."""
    n, levels = 63, 6
    h = oracle.Hierarchy(n, levels, math.pi / 3, 1e-3)
    b = rhs_normal(n, 11)
    st = h.stencil(1)
    A = spla.LinearOperator((n * n, n * n), matvec=lambda x: oracle.apply_stencil(st, x.reshape(n, n)).ravel())
    M = spla.LinearOperator((n * n, n * n),
                            matvec=lambda x: oracle.cycle(h, np.zeros((n, n)), x.reshape(n, n), kappa).ravel())
    for iters in (1, 3, 6):
        x_ref, _ = spla.cg(A, b.ravel(), rtol=1e-300, atol=0.0, maxiter=iters, M=M)
        x, hist = oracle.pcg(h, b, kappa, 1e-300, iters)
        assert len(hist) == iters
        assert np.linalg.norm(x.ravel() - x_ref) <= 1e-11 * np.linalg.norm(x_ref)


def test_pcg_converges_to_dense_solution_all_kappas():
    n, levels = 31, 5
    h = oracle.Hierarchy(n, levels, 1.1, 1e-4)
    b = rhs_uniform(n, 12)
    exact = scipy.linalg.solve(dense_A(h.stencil(1), n), b.ravel(), assume_a="pos").reshape(n, n)
    for kappa in (1, 2, 3, 5):
        for flexible in (False, True):
            x, hist = oracle.pcg(h, b, kappa, 1e-12, 200, flexible=flexible)
            assert hist[-1] <= 1e-12
            assert np.linalg.norm(x - exact) <= 1e-9 * np.linalg.norm(exact)
            assert np.isclose(hist[-1], oracle.relres(h, x, b), rtol=1e-6, atol=1e-15)


def test_solve_history_is_residual_of_iterates():
    n = 63
    h = oracle.Hierarchy(n, 6, math.pi / 6, 1e-2)
    f = rhs_uniform(n, 0)
    v, hist = oracle.solve(h, f, 3, 1e-300, 4)
    w = np.zeros_like(f)
    for k in range(4):
        w = oracle.cycle(h, w, f, 3)
        assert hist[k] == oracle.relres(h, w, f)
    assert np.array_equal(v, w)


@pytest.mark.parametrize("theta,eps", [(0.7, 1e-3), (math.pi / 6, 0.2)])
def test_param_grads_match_finite_differences(theta, eps):
    """L = 0.5 ||u - t||^2 with u = A(theta, eps)^{-1} f; central differences, h = 1e-6."""
    n = 15
    f = rhs_uniform(n, 13)
    t = rhs_normal(n, 14)

    def loss(th, ep):
        A = dense_A(oracle.fine_stencil(th, ep, n), n)
        u = scipy.linalg.solve(A, f.ravel(), assume_a="pos").reshape(n, n)
        return 0.5 * float(np.sum((u - t) ** 2)), u, A

    L0, u, A = loss(theta, eps)
    lam = scipy.linalg.solve(A.T, (u - t).ravel()).reshape(n, n)
    g_th, g_ep = oracle.param_grads(theta, eps, n, lam, u)
    d = 1e-6
    fd_th = (loss(theta + d, eps)[0] - loss(theta - d, eps)[0]) / (2 * d)
    fd_ep = (loss(theta, eps + d)[0] - loss(theta, eps - d)[0]) / (2 * d)
    assert abs(g_th - fd_th) <= 1e-6 * abs(fd_th)
    assert abs(g_ep - fd_ep) <= 1e-6 * abs(fd_ep)


def test_adjoint_solve_gives_lambda():
    """A is symmetric, so iterating the adjoint cycle on g solves A lambda = g."""
    n = 31
    h = oracle.Hierarchy(n, 5, 0.7, 1e-3)
    g = rhs_normal(n, 15)
    lam, hist = oracle.solve(h, g, 3, 1e-13, 300, adjoint=True)
    exact = scipy.linalg.solve(dense_A(h.stencil(1), n), g.ravel(), assume_a="pos").reshape(n, n)
    assert np.linalg.norm(lam - exact) <= 1e-10 * np.linalg.norm(exact)


def _dense_map(fn, n):
    cols = []
    for k in range(n * n):
        e = np.zeros(n * n)
        e[k] = 1.0
        cols.append(fn(e.reshape(n, n)).ravel())
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("kappa", [2, 3])
def test_symmetrised_preconditioner_is_symmetric_and_two_sided(kappa):
    """For 1 < kappa < levels the kappa-cycle B is not symmetric; M = B + B^T - B^T A B is, and its
    error propagator is (I - B^T A)(I - B A): a cycle followed by the adjoint cycle."""
    n, levels = 31, 5
    h = oracle.Hierarchy(n, levels, 0.7, 1e-2)
    A = dense_A(h.stencil(1), n)
    B = _dense_map(lambda r: oracle.cycle(h, np.zeros((n, n)), r, kappa), n)
    Bt = _dense_map(lambda r: oracle.cycle_adjoint(h, np.zeros((n, n)), r, kappa), n)
    M = _dense_map(lambda r: oracle.precondition(h, r, kappa, symmetric=True), n)
    scale = np.abs(M).max()
    assert np.abs(B - B.T).max() > 1e-6 * np.abs(B).max()          # B itself is not symmetric
    assert np.abs(M - M.T).max() <= 1e-12 * scale
    I = np.eye(n * n)
    assert np.abs((I - M @ A) - (I - Bt @ A) @ (I - B @ A)).max() <= 1e-12
    assert np.all(np.linalg.eigvalsh(0.5 * (M + M.T)) > 0)         # a valid CG preconditioner here


def test_symmetrised_pcg_converges_to_dense_solution():
    n, levels = 31, 5
    h = oracle.Hierarchy(n, levels, 1.1, 1e-4)
    b = rhs_uniform(n, 12)
    exact = scipy.linalg.solve(dense_A(h.stencil(1), n), b.ravel(), assume_a="pos").reshape(n, n)
    for kappa in (2, 3):
        x, hist = oracle.pcg(h, b, kappa, 1e-12, 200, symmetric=True)
        assert hist[-1] <= 1e-12
        assert np.linalg.norm(x - exact) <= 1e-9 * np.linalg.norm(exact)
