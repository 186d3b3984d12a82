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


@pytest.mark.parametrize("kappa", [1, 6])
def test_flexible_beta_equals_standard_for_symmetric_cycles(kappa):
    """Section 4's MGCG with a symmetric preconditioner B (the V- and W-cycles): in exact
    arithmetic PCG keeps r_{k+1} . B r_k = 0, so the flexible (Polak-Ribiere) beta,
    r_new.(z_new - z_old)/(r_old.z_old), equals the standard r_new.z_new/(r_old.z_old) and the two
    branches produce the same iterates up to rounding. A wrong sign, a wrong vector or a wrong
    denominator in the flexible branch changes beta by O(1) and fails this."""
    n, levels = 63, 6
    h = oracle.Hierarchy(n, levels, 0.4, 2e-3)
    b = rhs_normal(n, 13)
    for iters in (2, 5, 9):
        x_std, h_std = oracle.pcg(h, b, kappa, 1e-300, iters)
        x_flx, h_flx = oracle.pcg(h, b, kappa, 1e-300, iters, flexible=True)
        assert np.linalg.norm(x_flx - x_std) <= 1e-11 * np.linalg.norm(x_std), iters
        assert np.allclose(h_flx, h_std, rtol=1e-9, atol=0.0)
    # the orthogonality that makes the two agree, checked directly on the residuals after the
    # first and second iterations (after the first it holds for any B, since p_0 = z_0)
    r1, z1, r2 = _residuals_1_2(h, b, kappa)
    assert abs(float(np.sum(r2 * z1))) <= 1e-11 * np.linalg.norm(r2) * np.linalg.norm(z1)


def _residuals_1_2(h, b, kappa):
    st = h.stencil(1)
    x1, _ = oracle.pcg(h, b, kappa, 1e-300, 1)
    x2, _ = oracle.pcg(h, b, kappa, 1e-300, 2)
    r1 = b - oracle.apply_stencil(st, x1)
    return r1, oracle.precondition(h, r1, kappa), b - oracle.apply_stencil(st, x2)


def test_flexible_beta_differs_for_nonsymmetric_cycle_and_converges():
    """For 1 < kappa < levels the cycle is not symmetric (Section 4): r_{k+1} . B r_k no longer
    vanishes, so the two betas differ and the branch is really exercised; both still reach the
    dense solution."""
    n, levels, kappa = 63, 6, 2
    h = oracle.Hierarchy(n, levels, 0.4, 2e-3)
    b = rhs_normal(n, 13)
    x_std, _ = oracle.pcg(h, b, kappa, 1e-300, 4)
    x_flx, _ = oracle.pcg(h, b, kappa, 1e-300, 4, flexible=True)
    assert np.linalg.norm(x_flx - x_std) >= 1e-9 * np.linalg.norm(x_std)
    r1, z1, r2 = _residuals_1_2(h, b, kappa)
    assert abs(float(np.sum(r2 * z1))) >= 1e-8 * np.linalg.norm(r2) * np.linalg.norm(z1)


def _sine_mode(n, k, l):
    x = np.arange(1, n + 1) / (n + 1)
    return np.outer(np.sin(l * math.pi * x), np.sin(k * math.pi * x))  # [j, i]: x along i


@pytest.mark.parametrize("omega,sweeps", [(0.8, 1), (0.8, 2), (0.87, 3), (1.0, 1)])
def test_damped_jacobi_eigenvalues_of_five_point_laplacian(omega, sweeps):
    """theta = 0, eps = 1 is the five-point Laplacian (centre 4, the four neighbours -1, all over
    h^2). Its Dirichlet eigenvectors are sin(k pi x) sin(l pi y) with eigenvalue
    (4 - 2 cos(k pi h) - 2 cos(l pi h))/h^2, so one damped-Jacobi sweep with f = 0 multiplies such
    a mode by 1 - omega (1 - (cos(k pi h) + cos(l pi h))/2). Applying omega twice, dropping it or
    dividing by the wrong diagonal changes that factor."""
    n = 15
    h = oracle.Hierarchy(n, 4, 0.0, 1.0, omega=omega)
    hh = 1.0 / (n + 1)
    for k, l in ((1, 1), (3, 7), (15, 2), (8, 8)):
        e = _sine_mode(n, k, l)
        mu = 1.0 - omega * (1.0 - 0.5 * (math.cos(k * math.pi * hh) + math.cos(l * math.pi * hh)))
        out = oracle.relax(h, 1, e, np.zeros_like(e), sweeps)
        assert np.allclose(out, mu ** sweeps * e, rtol=0.0, atol=1e-13), (k, l)


def test_damped_jacobi_on_galerkin_level_of_laplacian():
    """The Galerkin operator of the Laplacian one level down is (1/H^2)[-1/4 -1/2 -1/4;
    -1/2 3 -1/2; -1/4 -1/2 -1/4]; it is diagonalised by the same sine modes with eigenvalue
    (3 - cos a - cos b - cos a cos b)/H^2, a = k pi H, b = l pi H. The hierarchy's relaxation at
    level 2 must therefore scale a mode by 1 - (omega/3)(3 - cos a - cos b - cos a cos b) per
    sweep (pins the level's stencil, the diagonal and omega together)."""
    n, omega = 31, 0.8
    h = oracle.Hierarchy(n, 4, 0.0, 1.0, omega=omega)
    nc = h.sizes[1]
    H = 1.0 / (nc + 1)
    for k, l in ((1, 2), (5, 5), (15, 1)):
        e = _sine_mode(nc, k, l)
        a, b = k * math.pi * H, l * math.pi * H
        mu = 1.0 - (omega / 3.0) * (3.0 - math.cos(a) - math.cos(b) - math.cos(a) * math.cos(b))
        out = oracle.relax(h, 2, e, np.zeros_like(e), 2)
        assert np.allclose(out, mu ** 2 * e, rtol=0.0, atol=1e-12), (k, l)


def test_one_jacobi_sweep_equals_dense_iteration_matrix():
    """One sweep of the oracle's damped Jacobi on a 7^2 rotated anisotropic problem equals the
    dense (I - omega D^-1 A) v + omega D^-1 f, with A assembled column by column and D its
    diagonal."""
    n, omega = 7, 0.8
    st = oracle.fine_stencil(1.1, 3e-2, n)
    A = dense_A(st, n)
    D = np.diag(A)
    v = rhs_normal(n, 21)
    f = rhs_uniform(n, 22)
    want = v.ravel() - omega * (A @ v.ravel()) / D + omega * f.ravel() / D
    got = oracle.jacobi(st, v, f, omega, 1)
    assert np.allclose(got.ravel(), want, rtol=1e-14, atol=1e-14 * np.abs(want).max())
    two = oracle.jacobi(st, v, f, omega, 2).ravel()
    want2 = want - omega * (A @ want) / D + omega * f.ravel() / D
    assert np.allclose(two, want2, rtol=1e-13, atol=1e-13 * np.abs(want2).max())
