"""Differentiable solve: the hand-written backward (adjoint kappa-cycles + parameter gradients)
against the FP64 oracle's adjoint and against central finite differences (h = 1e-6, FP64).

Central differences of L = 0.5||u - t||^2 are evaluated without cancellation as
L(p+h) - L(p-h) = (u+ - u-) . ((u+ + u-)/2 - t), the same difference computed stably (the loss
itself is about 5e5 at 1023^2, so subtracting two rounded loss values would bury a 1e-6 step).
Tolerance 1e-6 relative for gradients. In solve mode the forward and adjoint solves run to 1e-12
(finite-difference solves to 1e-13) so solver error stays below it; in fixed-cycle mode the map
f -> u is linear and its transpose is k adjoint cycles from zero, so dL/df is exact.
"""
import math

import numpy as np
import pytest

import oracle
from parity import rel  # norm-wise and element-wise (tests/parity.py)
from paper_2010_00626_b300.inputs import rhs_normal, rhs_uniform

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-6


def t64(a, grad=False):
    import torch
    return torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=grad)


def central_difference(u_plus, u_minus, target, h):
    """(L(p+h) - L(p-h)) / 2h for L = 0.5||u - t||^2, evaluated without cancellation."""
    up, um = u_plus.cpu().numpy(), u_minus.cpu().numpy()
    return float(np.sum((up - um) * (0.5 * (up + um) - target))) / (2 * h)


def loss_and_grads(solve, f, theta, eps, target, **kw):
    import torch
    fd = t64(f, True)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    ep = torch.tensor(eps, dtype=torch.float64, requires_grad=True)
    u = solve(fd, th, ep, **kw)
    L = 0.5 * ((u - t64(target)) ** 2).sum()
    L.backward()
    return float(L.detach()), fd.grad.detach().cpu().numpy(), float(th.grad), float(ep.grad), u.detach().cpu().numpy()


def test_gradients_match_oracle_adjoint_63(lib):
    from paper_2010_00626_b300.autograd import kcycle_solve
    n, levels, theta, eps = 63, 6, 0.7, 1e-3
    f, target = rhs_uniform(n, 2), rhs_normal(n, 1)
    L, gf, gth, gep, u = loss_and_grads(kcycle_solve, f, theta, eps, target, levels=levels, kappa=3, tol=1e-12)
    h = oracle.Hierarchy(n, levels, theta, eps)
    u_or, _ = oracle.solve(h, f, 3, 1e-13, 1000)
    lam, _ = oracle.solve(h, u_or - target, 3, 1e-13, 1000, adjoint=True)
    ref_th, ref_ep = oracle.param_grads(theta, eps, n, lam, u_or)
    assert rel(gf, lam) <= GRAD_TOL
    assert abs(gth - ref_th) <= GRAD_TOL * abs(ref_th)
    assert abs(gep - ref_ep) <= GRAD_TOL * abs(ref_ep)


@pytest.mark.parametrize("theta,eps", [(0.7, 1e-3), (math.pi / 6, 0.05)])
def test_parameter_gradients_match_finite_differences(lib, theta, eps):
    from paper_2010_00626_b300.autograd import kcycle_solve
    import torch
    n, levels = 127, 7
    f, target = rhs_uniform(n, 3), rhs_normal(n, 4)
    _, _, gth, gep, _ = loss_and_grads(kcycle_solve, f, theta, eps, target, levels=levels, kappa=3, tol=1e-12)
    d = 1e-6

    def U(th, ep):
        with torch.no_grad():
            return kcycle_solve(t64(f), torch.tensor(th, dtype=torch.float64), torch.tensor(ep, dtype=torch.float64),
                                levels, kappa=3, tol=1e-13)
    fd_th = central_difference(U(theta + d, eps), U(theta - d, eps), target, d)
    fd_ep = central_difference(U(theta, eps + d), U(theta, eps - d), target, d)
    assert abs(gth - fd_th) <= GRAD_TOL * abs(fd_th), (gth, fd_th)
    assert abs(gep - fd_ep) <= GRAD_TOL * abs(fd_ep), (gep, fd_ep)


def test_fixed_cycles_1023_df_is_exact_transpose(lib):
    """1023^2, theta=0.7, eps=1e-3, 10 kappa=3 cycles, u_target ~ N(0,1) seed 1."""
    from paper_2010_00626_b300.autograd import kcycle_solve
    import torch
    n, levels, theta, eps, kappa = 1023, 10, 0.7, 1e-3, 3
    f, target = rhs_uniform(n, 0), rhs_normal(n, 1)
    L0, gf, _, _, u = loss_and_grads(kcycle_solve, f, theta, eps, target, levels=levels, kappa=kappa, cycles=10)
    # oracle: 10 cycles forward, 10 adjoint cycles on g = u - target
    h = oracle.Hierarchy(n, levels, theta, eps)
    v = np.zeros_like(f)
    for _ in range(10):
        v = oracle.cycle(h, v, f, kappa)
    assert rel(u, v) <= 1e-12
    g, lam = v - target, np.zeros_like(f)
    for _ in range(10):
        lam = oracle.cycle_adjoint(h, lam, g, kappa)
    assert rel(gf, lam) <= 1e-10
    # directional central differences of the (quadratic) loss along seeded random directions
    rng = np.random.default_rng(5)
    hstep = 1e-6

    def Uf(ff):
        with torch.no_grad():
            return kcycle_solve(t64(ff), torch.tensor(theta, dtype=torch.float64),
                                torch.tensor(eps, dtype=torch.float64), levels, kappa=kappa, cycles=10)
    for _ in range(8):
        dlt = rng.standard_normal((n, n))
        fd = central_difference(Uf(f + hstep * dlt), Uf(f - hstep * dlt), target, hstep)
        assert abs(float(np.sum(gf * dlt)) - fd) <= GRAD_TOL * abs(fd)


def test_adjoint_solve_entry_point(lib):
    import torch
    n, levels, theta, eps = 255, 8, 1.2, 1e-2
    g = rhs_normal(n, 6)
    mg = lib.Multigrid(n, eps, theta, levels)
    lam = t64(np.zeros((n, n)))
    st, cycles, relres, hist = mg.solve(lam, t64(g), 2, 1e-10, 500, adjoint=True)
    h = oracle.Hierarchy(n, levels, theta, eps)
    lam_or, hist_or = oracle.solve(h, g, 2, 1e-10, 500, adjoint=True)
    assert st == 0 and cycles == len(hist_or)
    torch.cuda.synchronize()
    assert rel(lam.cpu().numpy(), lam_or) <= 1e-12
