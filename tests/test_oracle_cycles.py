"""Pins of the oracle's cycles (CPU only).

* recursion counts against the closed forms of Proposition 2.2, Proposition 2.4 and
  Lemma 2.9 (coarsest calls carry counter kappa - j, C(n-1, j) times);
* Proposition 2.1: kappa=1 is the V-cycle, kappa=2 the F-cycle, kappa>=n the W-cycle,
  iterate for iterate against separately written Algorithms 1 and 2;
* convergence to the dense direct solution;
* the symmetry statement of Section 4 (V and W symmetric from a zero start, 1<kappa<n not)
  and the adjoint cycle by the dot-product test.
"""
import math
from collections import Counter

import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2010_00626_b300.inputs import rhs_uniform


def level_calls_closed(kappa, level):
    """Proposition 2.2."""
    return sum(math.comb(level - 1, j) for j in range(0, min(kappa - 1, level - 1) + 1))


def total_calls_closed(kappa, n):
    """Proposition 2.4."""
    return sum(math.comb(n, j) for j in range(1, min(kappa, n) + 1))


def small_hierarchy(n=31, levels=None, theta=math.pi / 6, eps=1e-2, nu1=2, nu2=2):
    levels = levels or int(round(math.log2(n + 1)))
    return oracle.Hierarchy(n, levels, theta, eps, nu1=nu1, nu2=nu2)


@pytest.mark.parametrize("levels", [1, 2, 3, 4, 5, 6])
def test_recursion_counts_match_closed_forms(levels):
    h = small_hierarchy(63, levels)
    f = rhs_uniform(63, 0)
    for kappa in range(1, levels + 3):
        rec = oracle.CallRecorder(levels)
        oracle.cycle(h, np.zeros_like(f), f, kappa, rec)
        for lvl in range(1, levels + 1):
            assert rec.per_level[lvl] == level_calls_closed(kappa, lvl)
        assert sum(rec.per_level) == total_calls_closed(kappa, levels)
        # Lemma 2.9: C(n-1, j) coarsest calls with counter kappa - j
        seen = Counter(rec.coarsest_counters)
        expect = {kappa - j: math.comb(levels - 1, j) for j in range(0, min(kappa - 1, levels - 1) + 1)}
        assert dict(seen) == expect


def test_total_calls_examples():
    """Section 1: a W-cycle with ten levels makes 2^10 - 1 calls; Corollary 2.5."""
    assert total_calls_closed(10, 10) == 1023
    assert total_calls_closed(1, 12) == 12
    assert [total_calls_closed(k, 12) for k in (1, 2, 3, 4, 5, 12)] == [12, 78, 298, 793, 1585, 4095]


@pytest.mark.parametrize("n", [31, 63])
def test_kappa_one_is_v_cycle_bitwise(n):
    h = small_hierarchy(n)
    f = rhs_uniform(n, 1)
    v1 = v2 = np.zeros_like(f)
    for _ in range(3):
        v1 = oracle.cycle(h, v1, f, 1)
        v2 = oracle.gamma_cycle(h, 1, v2, f, 1)
        assert np.array_equal(v1, v2)


@pytest.mark.parametrize("n", [31, 63])
def test_kappa_two_is_f_cycle_bitwise(n):
    h = small_hierarchy(n)
    f = rhs_uniform(n, 2)
    v1 = v2 = np.zeros_like(f)
    for _ in range(3):
        v1 = oracle.cycle(h, v1, f, 2)
        v2 = oracle.f_cycle(h, 1, v2, f)
        assert np.array_equal(v1, v2)


@pytest.mark.parametrize("n", [31, 63])
def test_kappa_at_least_levels_is_w_cycle_bitwise(n):
    h = small_hierarchy(n)
    f = rhs_uniform(n, 3)
    for kappa in (h.levels, h.levels + 3):
        v1 = v2 = np.zeros_like(f)
        for _ in range(2):
            v1 = oracle.cycle(h, v1, f, kappa)
            v2 = oracle.gamma_cycle(h, 1, v2, f, 2)
            assert np.array_equal(v1, v2)


def test_kappa_between_is_neither_v_nor_w():
    h = small_hierarchy(63)
    f = rhs_uniform(63, 4)
    z = np.zeros_like(f)
    v3 = oracle.cycle(h, z, f, 3)
    assert not np.allclose(v3, oracle.gamma_cycle(h, 1, z, f, 1))
    assert not np.allclose(v3, oracle.gamma_cycle(h, 1, z, f, 2))


def dense_matrix_of(h):
    n = h.n
    cols = []
    for k in range(n * n):
        e = np.zeros(n * n)
        e[k] = 1.0
        cols.append(oracle.apply_stencil(h.stencil(1), e.reshape(n, n)).ravel())
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("n,levels", [(3, 2), (7, 3), (15, 4), (31, 5), (15, 3), (31, 3)])
def test_solve_reaches_dense_direct_solution(n, levels):
    h = small_hierarchy(n, levels, theta=math.pi / 3, eps=1e-2)
    f = rhs_uniform(n, 5)
    A = dense_matrix_of(h)
    exact = scipy.linalg.solve(A, f.ravel(), assume_a="pos").reshape(n, n)
    v, hist = oracle.solve(h, f, 3, 1e-14, 500)
    assert hist[-1] <= 1e-14
    assert np.linalg.norm(v - exact) <= 1e-12 * np.linalg.norm(exact)
    # history entries are the residuals of the iterates
    assert hist == sorted(hist, reverse=True) or hist[-1] < hist[0]


def test_one_level_is_exact_in_one_cycle():
    h = small_hierarchy(7, 1)
    f = rhs_uniform(7, 6)
    A = dense_matrix_of(h)
    v = oracle.cycle(h, np.zeros_like(f), f, 1)
    assert np.allclose(A @ v.ravel(), f.ravel(), rtol=0, atol=1e-13 * np.abs(f).max())


def cycle_matrix(h, kappa, adjoint=False):
    n = h.n
    step = oracle.cycle_adjoint if adjoint else oracle.cycle
    cols = []
    for k in range(n * n):
        e = np.zeros(n * n)
        e[k] = 1.0
        cols.append(step(h, np.zeros((n, n)), e.reshape(n, n), kappa).ravel())
    return np.stack(cols, axis=1)


def test_v_and_w_cycles_symmetric_others_not():
    """Section 4: with symmetric Jacobi, nu1 = nu2 and R the adjoint of P, the V- and
    W-cycle matrices from a zero start are symmetric; for 1 < kappa < n they are not."""
    h = small_hierarchy(15, 4, theta=math.pi / 3, eps=1e-3)
    # kappa = n-1 is symmetric too: its only difference from W is a second call at level
    # n-1 that repeats an exact coarsest solve and so changes nothing (Section 1 remark).
    for kappa in (1, 3, 4, 7):
        B = cycle_matrix(h, kappa)
        assert np.max(np.abs(B - B.T)) <= 1e-13 * np.abs(B).max()
        assert np.all(np.linalg.eigvalsh(0.5 * (B + B.T)) > 0)
    for kappa in (2,):
        B = cycle_matrix(h, kappa)
        assert np.max(np.abs(B - B.T)) > 1e-6 * np.abs(B).max()


@pytest.mark.parametrize("nu", [(2, 2), (1, 3), (0, 2)])
def test_adjoint_cycle_is_transpose(nu):
    h = small_hierarchy(15, 4, theta=0.7, eps=1e-3, nu1=nu[0], nu2=nu[1])
    for kappa in (1, 2, 3, 4):
        B = cycle_matrix(h, kappa)
        Bt = cycle_matrix(h, kappa, adjoint=True)
        assert np.max(np.abs(Bt - B.T)) <= 1e-13 * np.abs(B).max()


def test_adjoint_dot_product_large():
    h = small_hierarchy(63, 6, theta=0.7, eps=1e-3)
    rng = np.random.default_rng(9)
    x, y = rng.standard_normal((2, 63, 63))
    z = np.zeros((63, 63))
    for kappa in (2, 3, 5):
        lhs = np.sum(x * oracle.cycle(h, z, y, kappa))
        rhs = np.sum(oracle.cycle_adjoint(h, z, x, kappa) * y)
        assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_cycle_from_nonzero_start_is_affine():
    """v_out = v + B (f - A v): the cycle is the stationary iteration of its zero-start map."""
    h = small_hierarchy(31, 5)
    rng = np.random.default_rng(10)
    v, f = rng.standard_normal((2, 31, 31))
    for kappa in (1, 3):
        lhs = oracle.cycle(h, v, f, kappa)
        rhs = v + oracle.cycle(h, np.zeros_like(v), oracle.residual(h.stencil(1), v, f), kappa)
        assert np.allclose(lhs, rhs, rtol=0, atol=1e-12 * np.abs(lhs).max())


def test_coarsest_dense_when_levels_short():
    """levels < k: the coarsest grid is larger than 1x1 and solved exactly (3x3 here)."""
    h = small_hierarchy(127, 6, theta=math.pi / 6, eps=1e-2)
    assert h.sizes[-1] == 3
    f = rhs_uniform(3, 7)
    v = h.coarsest_solve(f)
    assert np.allclose(oracle.apply_stencil(h.stencils[-1], v), f, rtol=0, atol=1e-13 * np.abs(f).max())


def test_rediscretized_hierarchy_and_error_protocol():
    """Rediscretized coarse operators are the Section 4 stencil with the coarse h; the error
    protocol (f = 0) is the same cycle iteration, so its history is the iterate norm ratio and the
    solution tends to zero."""
    n, levels = 63, 6
    h = oracle.Hierarchy(n, levels, math.pi / 4, 1e-2, coarse_op="rediscretized")
    for lvl, m in enumerate(h.sizes):
        assert np.array_equal(h.stencils[lvl], oracle.fine_stencil(math.pi / 4, 1e-2, m))
    v0 = np.random.default_rng(2).uniform(-1, 1, (n, n))
    v, hist = oracle.solve_error_reduction(h, v0, 3, 1e-8, 500)
    assert hist[-1] <= 1e-8 and np.linalg.norm(v) <= 1e-8 * np.linalg.norm(v0)
    w = v0.copy()
    for _ in range(3):
        w = oracle.cycle(h, w, np.zeros_like(v0), 3)
    assert np.isclose(np.linalg.norm(w) / np.linalg.norm(v0), hist[2], rtol=1e-14)
    with pytest.raises(ValueError):
        oracle.Hierarchy(15, 3, 0.1, 0.1, coarse_op="other")


def _zebra_brute(st, v, f, axis):
    """Line Gauss-Seidel in zebra order with explicit loops and a dense solve per line."""
    n = v.shape[0]
    v = v.copy()
    for parity in (0, 1):
        for L in range(parity, n, 2):
            A = np.zeros((n, n))
            b = np.zeros(n)
            for p in range(n):
                i, j = (p, L) if axis == "x" else (L, p)
                b[p] = f[j, i]
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        ii, jj = i + dx, j + dy
                        if not (0 <= ii < n and 0 <= jj < n):
                            continue
                        on_line = (jj == L) if axis == "x" else (ii == L)
                        if on_line:
                            A[p, ii if axis == "x" else jj] += st[1 + dy, 1 + dx]
                        else:
                            b[p] -= st[1 + dy, 1 + dx] * v[jj, ii]
            x = np.linalg.solve(A, b)
            for p in range(n):
                if axis == "x":
                    v[L, p] = x[p]
                else:
                    v[p, L] = x[p]
    return v


@pytest.mark.parametrize("axis", ["x", "y"])
def test_zebra_lines_match_brute_force_and_zero_last_residual(axis):
    n = 15
    st = oracle.galerkin_stencil(oracle.fine_stencil(0.7, 1e-3, 31))  # a general 9-point stencil
    rng = np.random.default_rng(8)
    v, f = rng.standard_normal((2, n, n))
    got = oracle.zebra_lines(st, v, f, axis)
    ref = _zebra_brute(st, v, f, axis)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.abs(ref).max()
    r = oracle.residual(st, got, f)
    odd = r[1::2, :] if axis == "x" else r[:, 1::2]  # the lines solved last satisfy their equations
    assert np.max(np.abs(odd)) <= 1e-12 * np.abs(f).max() * np.abs(st).sum()


def test_zebra_cycles_solve_grid_aligned_anisotropy():
    """theta = 0, eps = 1e-4: strong coupling along x. Zebra kappa-cycles reach the dense solution
    quickly; damped point Jacobi cycles stall (the case Section 4 uses line relaxation for)."""
    n, levels = 31, 5
    hz = oracle.Hierarchy(n, levels, 0.0, 1e-4, smoother="zebra")
    hj = oracle.Hierarchy(n, levels, 0.0, 1e-4)
    f = rhs_uniform(n, 11)
    vz, histz = oracle.solve(hz, f, 2, 1e-10, 200)
    vj, histj = oracle.solve(hj, f, 2, 1e-10, 200)
    assert histz[-1] <= 1e-10 and len(histz) < 40
    assert len(histj) > 3 * len(histz)
    A = dense_matrix_of(hz)
    exact = scipy.linalg.solve(A, f.ravel(), assume_a="pos").reshape(n, n)
    assert np.linalg.norm(vz - exact) <= 1e-9 * np.linalg.norm(exact)


@pytest.mark.parametrize("axis", ["x", "y"])
def test_zebra_exact_when_lines_decouple(axis):
    """With no coupling between lines (a 1-D operator along the lines), one relaxation along the
    lines is the exact solve, whatever the starting guess."""
    n = 31
    st = np.zeros((3, 3))
    st[1, 1], st[1, 0], st[1, 2] = 2.3, -1.0, -1.0
    if axis == "y":
        st = st.T.copy()
    rng = np.random.default_rng(12)
    v0, f = rng.standard_normal((2, n, n))
    got = oracle.zebra_lines(st, v0, f, axis)
    T = np.diag(np.full(n, 2.3)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1)
    exact = np.linalg.solve(T, f.T).T if axis == "x" else np.linalg.solve(T, f)
    assert np.max(np.abs(got - exact)) <= 1e-13 * np.abs(exact).max()


def test_zebra_two_relaxations_are_one_per_direction():
    """nu = 2 is an x relaxation followed by a y relaxation (Section 4's alternating form)."""
    n, levels = 15, 3
    h = oracle.Hierarchy(n, levels, 0.4, 1e-3, smoother="zebra")
    rng = np.random.default_rng(13)
    v, f = rng.standard_normal((2, n, n))
    st = h.stencil(1)
    both = oracle.relax(h, 1, v, f, 2)
    manual = oracle.zebra_lines(st, oracle.zebra_lines(st, v, f, "x"), f, "y")
    assert np.array_equal(both, manual)
    with pytest.raises(ValueError):
        oracle.Hierarchy(n, levels, 0.4, 1e-3, smoother="sor")
    with pytest.raises(ValueError):
        oracle.cycle_adjoint(h, v, f, 2)


@pytest.mark.parametrize("theta", [0.0, math.pi / 2, math.pi / 4, 0.3])
def test_semi_coarsening_cycles_robust_for_any_angle(theta):
    """x-line zebra with y semi-coarsening (Section 4, solvers 5-6) at eps = 1e-5: strong coupling
    along x is handled by the line solves, along y by the coarsening, so both grid-aligned cases
    converge quickly; the cycles reach the dense solution."""
    n, levels = 31, 5
    h = oracle.Hierarchy(n, levels, theta, 1e-5, smoother="xzebra", coarsening="y")
    f = rhs_uniform(n, 14)
    v, hist = oracle.solve(h, f, 2, 1e-10, 200)
    assert hist[-1] <= 1e-10 and len(hist) < 60
    A = dense_matrix_of(h)
    exact = scipy.linalg.solve(A, f.ravel(), assume_a="pos").reshape(n, n)
    assert np.linalg.norm(v - exact) <= 1e-9 * np.linalg.norm(exact)


def test_semi_coarsening_levels_keep_every_column():
    n, levels = 15, 4
    h = oracle.Hierarchy(n, levels, 0.5, 1e-3, smoother="xzebra", coarsening="y")
    rec = oracle.CallRecorder(levels)
    shapes = []
    orig = oracle.mg.relax

    def spy(hh, level, v, f, sweeps):
        shapes.append((level, v.shape))
        return orig(hh, level, v, f, sweeps)

    oracle.mg.relax = spy
    try:
        oracle.cycle(h, np.zeros((n, n)), rhs_uniform(n, 1), 2, rec)
    finally:
        oracle.mg.relax = orig
    assert {lv: s for lv, s in shapes} == {1: (15, 15), 2: (7, 15), 3: (3, 15)}
    assert rec.per_level[1:] == [1, 2, 3, 4]   # the F-cycle counts of Algorithm 3, as with full coarsening


@pytest.mark.parametrize("bx,by", [(30.0, 10.0), (-50.0, 20.0)])
def test_convection_diffusion_cycles_reach_dense_solution(bx, by):
    """The kappa-cycle on the non-symmetric upwind convection-diffusion operator (damped Jacobi,
    upwind operators rediscretized on every level, LU at the coarsest level) converges to the
    dense solution. (Galerkin products of the upwind operator lose the upwind structure on the
    coarse grids, where the cell Peclet number doubles per level, and Jacobi diverges there.)"""
    n, levels = 31, 5
    h = oracle.Hierarchy(n, levels, math.pi / 6, 1e-2, bx=bx, by=by, coarse_op="rediscretized")
    f = rhs_uniform(n, 15)
    A = dense_matrix_of(h)
    assert np.abs(A - A.T).max() > 1.0
    exact = scipy.linalg.solve(A, f.ravel()).reshape(n, n)
    for kappa in (1, 3):
        v, hist = oracle.solve(h, f, kappa, 1e-10, 300)
        assert hist[-1] <= 1e-10 and len(hist) < 40
        assert np.linalg.norm(v - exact) <= 1e-8 * np.linalg.norm(exact)
    g = oracle.Hierarchy(n, levels, math.pi / 6, 1e-2, bx=bx, by=by)   # Galerkin: diverges
    with np.errstate(all="ignore"):
        assert not oracle.solve(g, f, 1, 1e-10, 30)[1][-1] <= 1.0
