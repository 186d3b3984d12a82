"""Pins of the oracle's discretisation, transfers and Galerkin operator (CPU only).

Each pin checks the oracle against something other than itself: the continuous operator
-div(K grad u) on quadratics (the nine-point formula is exact there), the textbook Galerkin
stencil of the 5-point Laplacian, dense matrix products, and exactness of the transfers
on polynomials.
"""
import math

import numpy as np
import pytest

import oracle

CASES = [(0.0, 1.0), (math.pi / 6, 1e-2), (math.pi / 3, 1e-4), (0.7, 1e-3), (2.5, 0.3)]


def diffusion_tensor(theta, eps):
    """K = R(theta) diag(1, eps) R(theta)^T: strong diffusion along angle theta."""
    c, s = math.cos(theta), math.sin(theta)
    rot = np.array([[c, -s], [s, c]])
    return rot @ np.diag([1.0, eps]) @ rot.T


def grid(n):
    h = 1.0 / (n + 1)
    x = (np.arange(n) + 1) * h
    return np.meshgrid(x, x)  # X[j, i] = x_i, Y[j, i] = y_j


@pytest.mark.parametrize("theta,eps", CASES)
@pytest.mark.parametrize("abc", [(1, 0, 0), (0, 1, 0), (0, 0, 1), (0.3, -0.7, 1.1)])
def test_fine_stencil_exact_on_quadratics(theta, eps, abc):
    """Section 4 stencil (top row = north, A = S/h^2) reproduces -div(K grad u) exactly
    for u = a x^2 + b xy + c y^2, with K built from the rotation, not from the table."""
    n = 31
    a, b, c = abc
    X, Y = grid(n)
    u = a * X * X + b * X * Y + c * Y * Y
    K = diffusion_tensor(theta, eps)
    expected = -(2 * a * K[0, 0] + 2 * b * K[0, 1] + 2 * c * K[1, 1])
    Au = oracle.apply_stencil(oracle.fine_stencil(theta, eps, n), u)[1:-1, 1:-1]
    scale = 8.0 * (n + 1) ** 2 * np.max(np.abs(u))  # size of the cancelling terms
    assert np.max(np.abs(Au - expected)) <= 1e-13 * scale


def test_fine_stencil_symmetric_and_zero_row_sum():
    for theta, eps in CASES:
        st = oracle.fine_stencil(theta, eps, 15)
        assert np.allclose(st, st[::-1, ::-1], rtol=0, atol=1e-12 * np.abs(st).max())
        assert abs(st.sum()) <= 1e-13 * np.abs(st).max()


def test_apply_dirichlet_is_dense_matrix_of_stencil_neighbours():
    """Brute force: A as an explicit double loop over grid points and their neighbours."""
    n = 7
    st = oracle.fine_stencil(0.7, 1e-3, n)
    v = np.random.default_rng(3).standard_normal((n, n))
    out = np.zeros((n, n))
    for j in range(n):
        for i in range(n):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    jj, ii = j + dy, i + dx
                    if 0 <= jj < n and 0 <= ii < n:
                        out[j, i] += st[1 + dy, 1 + dx] * v[jj, ii]
    assert np.allclose(oracle.apply_stencil(st, v), out, rtol=1e-14, atol=1e-12)


def dense(op, shape_in):
    """Dense matrix of a linear grid operator, by columns on unit vectors."""
    size = shape_in[0] * shape_in[1]
    cols = []
    for k in range(size):
        e = np.zeros(size)
        e[k] = 1.0
        cols.append(op(e.reshape(shape_in)).ravel())
    return np.stack(cols, axis=1)


def test_restriction_is_quarter_prolongation_transpose():
    """Full weighting = P^T / 4 (the adjoint pair named in Section 4)."""
    P = dense(oracle.prolong_bilinear, (7, 7))
    R = dense(oracle.restrict_fw, (15, 15))
    assert P.shape == (225, 49) and R.shape == (49, 225)
    assert np.array_equal(R, P.T / 4.0)


def test_prolongation_exact_on_bilinear_functions():
    m = 7
    n = 2 * m + 1
    Xc, Yc = grid(m)
    Xf, Yf = grid(n)
    g = lambda X, Y: 0.4 + 1.3 * X - 0.8 * Y + 2.1 * X * Y
    # a bilinear function does not vanish on the boundary; compare only where no
    # boundary value enters: fine points whose coarse neighbours are all interior
    pf = oracle.prolong_bilinear(g(Xc, Yc))
    assert np.allclose(pf[1:-1, 1:-1], g(Xf, Yf)[1:-1, 1:-1], rtol=0, atol=1e-14)


def test_restriction_exact_on_linear_functions():
    n = 15
    Xf, Yf = grid(n)
    Xc, Yc = grid(7)
    g = lambda X, Y: 0.4 + 1.3 * X - 0.8 * Y
    assert np.allclose(oracle.restrict_fw(g(Xf, Yf)), g(Xc, Yc), rtol=0, atol=1e-14)


@pytest.mark.parametrize("theta,eps", CASES)
def test_galerkin_equals_dense_rap_including_boundary_rows(theta, eps):
    """Dense R A P on 15^2 -> 7^2 equals the constant coarse stencil on every row."""
    nf, nc = 15, 7
    st = oracle.fine_stencil(theta, eps, nf)
    A = dense(lambda v: oracle.apply_stencil(st, v), (nf, nf))
    P = dense(oracle.prolong_bilinear, (nc, nc))
    R = dense(oracle.restrict_fw, (nf, nf))
    Ac = R @ A @ P
    stc = oracle.galerkin_stencil(st)
    Ac_st = dense(lambda v: oracle.apply_stencil(stc, v), (nc, nc))
    assert np.max(np.abs(Ac - Ac_st)) <= 1e-14 * np.abs(Ac).max()
    assert np.allclose(Ac, Ac.T, rtol=0, atol=1e-14 * np.abs(Ac).max())


def test_galerkin_of_laplacian_is_textbook_stencil():
    """eps=1, theta=0 is the 5-point Laplacian; its Galerkin coarse operator with full
    weighting and bilinear interpolation is (1/H^2)[-1/4 -1/2 -1/4; -1/2 3 -1/2; ...]."""
    n = 31
    H = 2.0 / (n + 1)
    stc = oracle.galerkin_stencil(oracle.fine_stencil(0.0, 1.0, n))
    expect = np.array([[-0.25, -0.5, -0.25], [-0.5, 3.0, -0.5], [-0.25, -0.5, -0.25]]) / H ** 2
    assert np.allclose(stc, expect, rtol=1e-14, atol=0)


@pytest.mark.parametrize("theta,eps", CASES)
def test_galerkin_consistent_on_quadratics(theta, eps):
    """Two Galerkin steps stay consistent with -div(K grad u) at the coarse spacing."""
    n = 63
    st = oracle.fine_stencil(theta, eps, n)
    for m in (31, 15):
        st = oracle.galerkin_stencil(st)
        X, Y = grid(m)
        K = diffusion_tensor(theta, eps)
        u = 0.3 * X * X - 0.7 * X * Y + 1.1 * Y * Y
        expected = -(2 * 0.3 * K[0, 0] - 2 * 0.7 * K[0, 1] + 2 * 1.1 * K[1, 1])
        Au = oracle.apply_stencil(st, u)[1:-1, 1:-1]
        assert np.max(np.abs(Au - expected)) <= 1e-12 * np.abs(st).sum() * np.abs(u).max()


def test_stencil_derivatives_match_central_differences():
    n, d = 31, 1e-6
    for theta, eps in CASES:
        dth, dep = oracle.fine_stencil_derivatives(theta, eps, n)
        fd_th = (oracle.fine_stencil(theta + d, eps, n) - oracle.fine_stencil(theta - d, eps, n)) / (2 * d)
        fd_ep = (oracle.fine_stencil(theta, eps + d, n) - oracle.fine_stencil(theta, eps - d, n)) / (2 * d)
        scale = (n + 1) ** 2
        assert np.max(np.abs(dth - fd_th)) <= 1e-7 * scale
        assert np.max(np.abs(dep - fd_ep)) <= 1e-7 * scale


def test_level_sizes():
    assert oracle.level_sizes(127, 7) == [127, 63, 31, 15, 7, 3, 1]
    assert oracle.level_sizes(4095, 12)[-1] == 1
    assert oracle.level_sizes(127, 6)[-1] == 3
    with pytest.raises(ValueError):
        oracle.Hierarchy(100, 3, 0.1, 0.1)
    with pytest.raises(ValueError):
        oracle.Hierarchy(127, 8, 0.1, 0.1)


def _galerkin_exact(S):
    """R A P of a 3x3 stencil in exact rational arithmetic (independent of the oracle)."""
    from fractions import Fraction as Fr
    hat = {-1: Fr(1, 2), 0: Fr(1), 1: Fr(1, 2)}
    out = [[Fr(0)] * 3 for _ in range(3)]
    for Dy in (-1, 0, 1):
        for Dx in (-1, 0, 1):
            acc = Fr(0)
            for ay in (-1, 0, 1):
                for ax in (-1, 0, 1):
                    r = Fr(1, 4) * hat[ay] * hat[ax]
                    for by in (-1, 0, 1):
                        for bx in (-1, 0, 1):
                            y, x = ay + by - 2 * Dy, ax + bx - 2 * Dx
                            if abs(y) <= 1 and abs(x) <= 1:
                                acc += r * S[by + 1][bx + 1] * hat[y] * hat[x]
            out[Dy + 1][Dx + 1] = acc
    return out


@pytest.mark.parametrize("theta,eps", [(math.pi / 3, 1e-4), (math.pi / 6, 1e-2), (0.7, 1e-3)])
def test_hierarchy_stencils_match_exact_galerkin(theta, eps):
    """12 levels: the oracle's coarse stencils equal the exact rational Galerkin chain of the
    fine stencil with its centre set to -(sum of the others) to a few ulp per level."""
    from fractions import Fraction as Fr
    n, levels = 4095, 12
    h = oracle.Hierarchy(n, levels, theta, eps)
    fine = [[Fr(float(v)) for v in row] for row in h.stencils[0]]
    zs = [row[:] for row in fine]
    zs[1][1] = -(sum(sum(r) for r in zs) - zs[1][1])
    for l in range(1, levels):
        zs = _galerkin_exact(zs)
        exact = np.array([[float(v) for v in r] for r in zs])
        scale = np.abs(exact).max()
        # each level adds a few ulp in components the Galerkin map does not amplify
        assert np.max(np.abs(h.stencils[l] - exact)) <= 16 * (l + 1) * np.finfo(float).eps * scale, l
        assert abs(h.stencils[l].sum()) <= 16 * np.finfo(float).eps * scale


def test_cos_sin_correctly_rounded_against_libm():
    """The oracle's cos/sin are within 1 ulp of libm and equal to it almost always."""
    rng = np.random.default_rng(0)
    angles = [math.pi / 6, math.pi / 3, 0.7, 0.0, math.pi / 4, 2.5] + list(rng.uniform(0, math.pi, 100))
    same = 0
    for a in angles:
        c, s = oracle.cos_sin(float(a))
        assert abs(c - math.cos(a)) <= np.spacing(abs(math.cos(a))) and abs(s - math.sin(a)) <= np.spacing(abs(math.sin(a)))
        same += (c == math.cos(a)) and (s == math.sin(a))
    assert same >= len(angles) - 3
    assert oracle.cos_sin(0.0) == (1.0, 0.0)


def test_galerkin_exact_matches_float_probing():
    """The exactly rounded Galerkin stencil equals R A P applied in FP64 up to rounding."""
    for theta, eps in CASES:
        st = oracle.fine_stencil(theta, eps, 63)
        e = np.zeros((5, 5))
        e[2, 2] = 1.0
        col = oracle.restrict_fw(oracle.apply_stencil(st, oracle.prolong_bilinear(e)))
        probe = np.array([[col[2 - dy, 2 - dx] for dx in (-1, 0, 1)] for dy in (-1, 0, 1)])
        assert np.max(np.abs(oracle.galerkin_stencil(st) - probe)) <= 16 * np.finfo(float).eps * np.abs(st).max()


# --------------------------------------------------------------------------------------------
# Semi-coarsening along y (Section 4, solvers 5-6)
# --------------------------------------------------------------------------------------------

def test_semi_restriction_is_half_prolongation_transpose():
    nyf, nx = 15, 9
    P = dense(oracle.prolong_y, ((nyf - 1) // 2, nx))
    R = dense(oracle.restrict_fw_y, (nyf, nx))
    assert np.array_equal(R, P.T / 2)


def test_semi_transfers_exact_on_linear_functions_of_y():
    nyf, nx = 15, 5
    y = (np.arange(nyf) + 1) / (nyf + 1)
    yc = (np.arange(7) + 1) / 8
    g = lambda yy, x: (0.3 - 1.7 * yy)[:, None] * (1.0 + x)[None, :]
    x = np.linspace(0.1, 0.9, nx)
    assert np.allclose(oracle.restrict_fw_y(g(y, x)), g(yc, x), rtol=0, atol=1e-14)
    # interior fine rows (every coarse neighbour interior) are reproduced exactly
    assert np.allclose(oracle.prolong_y(g(yc, x))[1:-1], g(y, x)[1:-1], rtol=0, atol=1e-14)


@pytest.mark.parametrize("theta,eps", CASES)
def test_semi_galerkin_equals_dense_rap(theta, eps):
    """Dense R_y A P_y on 15 rows -> 7 rows (9 columns kept) equals the constant coarse stencil on
    every row, boundary rows and columns included."""
    nyf, nyc, nx = 15, 7, 9
    st = oracle.fine_stencil(theta, eps, 15)
    A = dense(lambda v: oracle.apply_stencil(st, v), (nyf, nx))
    P = dense(oracle.prolong_y, (nyc, nx))
    R = dense(oracle.restrict_fw_y, (nyf, nx))
    Ac = R @ A @ P
    stc = oracle.galerkin_stencil_y(st)
    Ac_st = dense(lambda v: oracle.apply_stencil(stc, v), (nyc, nx))
    assert np.max(np.abs(Ac - Ac_st)) <= 1e-14 * np.abs(Ac).max()
    assert np.allclose(Ac, Ac.T, rtol=0, atol=1e-14 * np.abs(Ac).max())


def test_semi_galerkin_of_laplacian_closed_form():
    """eps=1, theta=0 is the 5-point Laplacian (1/h^2)[0 -1 0; -1 4 -1; 0 -1 0]. With linear
    interpolation in y and R = P^T / 2, the x part becomes (-u_xx) x (1/2) P^T P = rows
    [1/8, 3/4, 1/8] and the y part (1/2)(1-D Galerkin [-1/2, 1, -1/2]): in all
    (1/h^2)[-1/8 0 -1/8; -3/4 2 -3/4; -1/8 0 -1/8]."""
    n = 31
    h = 1.0 / (n + 1)   # fine spacing: semi-coarsening keeps h in x (the y spacing doubles)
    stc = oracle.galerkin_stencil_y(oracle.fine_stencil(0.0, 1.0, n))
    expect = np.array([[-0.125, 0.0, -0.125], [-0.75, 2.0, -0.75], [-0.125, 0.0, -0.125]]) / h ** 2
    assert np.allclose(stc, expect, rtol=1e-14, atol=1e-14 / h ** 2)


def test_semi_hierarchy_coarsest_is_one_row_solved_exactly():
    n = 31
    h = oracle.Hierarchy(n, 5, 0.4, 1e-3, smoother="xzebra", coarsening="y")
    assert h.sizes == [31, 15, 7, 3, 1]
    f = np.random.default_rng(3).standard_normal((1, n))
    x = h.coarsest_solve(f)
    assert x.shape == (1, n)
    r = f - oracle.apply_stencil(h.stencil(5), x)
    assert np.max(np.abs(r)) <= 1e-12 * np.abs(f).max()
    with pytest.raises(ValueError):
        oracle.Hierarchy(n, 4, 0.4, 1e-3, smoother="xzebra", coarsening="y")


# --------------------------------------------------------------------------------------------
# Convection-diffusion (the non-symmetric problem Section 5 proposes): upwind convection
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("bx,by", [(30.0, 10.0), (-20.0, 5.0), (7.0, -40.0), (-3.0, -3.0)])
def test_upwind_convection_exact_on_linear_and_quadratic(bx, by):
    """Linear u: the diffusion part vanishes and one-sided differences are exact, so A u = b . grad u
    at interior points. u = x^2 (or y^2): the one-sided difference of x^2 is 2x - h (backward) or
    2x + h (forward), so A u = -2 K_xx + bx (2x -/+ h) exactly."""
    n, theta, eps = 15, 0.6, 0.1
    h = 1.0 / (n + 1)
    st = oracle.convection_stencil(oracle.fine_stencil(theta, eps, n), bx, by, n)
    X, Y = grid(n)
    inner = (slice(1, -1), slice(1, -1))
    lin = 0.3 + 1.7 * X - 0.4 * Y
    Au = oracle.apply_stencil(st, lin)
    assert np.allclose(Au[inner], bx * 1.7 + by * (-0.4), rtol=0, atol=1e-9 * np.abs(st).max())
    K = diffusion_tensor(theta, eps)
    quad = X ** 2
    expect = -2 * K[0, 0] + bx * (2 * X - np.sign(bx) * h)
    assert np.allclose(oracle.apply_stencil(st, quad)[inner], expect[inner], rtol=0, atol=1e-9 * np.abs(st).max())


@pytest.mark.parametrize("bx,by", [(30.0, 10.0), (-20.0, 5.0)])
def test_galerkin_of_nonsymmetric_equals_dense_rap(bx, by):
    nf, nc = 15, 7
    st = oracle.convection_stencil(oracle.fine_stencil(0.7, 1e-2, nf), bx, by, nf)
    A = dense(lambda v: oracle.apply_stencil(st, v), (nf, nf))
    assert np.abs(A - A.T).max() > 1.0                              # not symmetric
    P = dense(oracle.prolong_bilinear, (nc, nc))
    R = dense(oracle.restrict_fw, (nf, nf))
    Ac = R @ A @ P
    stc = oracle.galerkin_stencil(st)
    Ac_st = dense(lambda v: oracle.apply_stencil(stc, v), (nc, nc))
    assert np.max(np.abs(Ac - Ac_st)) <= 1e-14 * np.abs(Ac).max()
