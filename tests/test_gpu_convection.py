"""GPU parity for the non-symmetric convection-diffusion problem (Section 5's proposed test):
-div(K grad u) + b . grad u with upwind convection, damped-Jacobi kappa-cycles on the general
(non-symmetric) stencil kernels. Stencils bit for bit, iterates to 1e-12, histories as in
tests/test_gpu_parity.py."""
import math

import numpy as np
import pytest

import oracle
from parity import rel  # norm-wise and element-wise (tests/parity.py)
from paper_2010_00626_b300.inputs import KAPPA_W, rhs_normal, rhs_uniform

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-12
HIST_TOL = 1e-10
CASES = [(127, 7, math.pi / 6, 1e-2, (30.0, 10.0)), (255, 8, 1.0, 1e-3, (-200.0, 50.0)),
         (1023, 10, 0.3, 1.0, (500.0, -800.0)), (511, 6, 2.0, 1e-1, (-5.0, -5.0))]


def torch_dev(a):
    import torch
    return torch.tensor(a, dtype=torch.float64, device="cuda")


def to_np(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()




def make(lib, n, levels, theta, eps, b, coarse_op="rediscretized"):
    h = oracle.Hierarchy(n, levels, theta, eps, bx=b[0], by=b[1], coarse_op=coarse_op)
    mg = lib.Multigrid(n, eps, theta, levels, convection=b, coarse_op=coarse_op)
    return h, mg


@pytest.mark.parametrize("coarse_op", ["rediscretized", "galerkin"])
@pytest.mark.parametrize("n,levels,theta,eps,b", CASES)
def test_convection_stencils_bitwise(lib, n, levels, theta, eps, b, coarse_op):
    h, mg = make(lib, n, levels, theta, eps, b, coarse_op)
    st = mg.stencils()
    for l in range(levels):
        assert np.array_equal(st[l], h.stencils[l]), (l, st[l] - h.stencils[l])


@pytest.mark.parametrize("n,levels,theta,eps,b", CASES)
def test_convection_cycles_per_iterate(lib, n, levels, theta, eps, b):
    h, mg = make(lib, n, levels, theta, eps, b)
    f = rhs_uniform(n, 0)
    fd, vd = torch_dev(f), torch_dev(np.zeros((n, n)))
    v = np.zeros((n, n))
    for c, kappa in enumerate((1, 3, 2, 4)):
        v = oracle.cycle(h, v, f, kappa)
        mg.kcycle(vd, fd, kappa)
        err = rel(to_np(vd), v)
        assert err <= ITER_TOL, (c, err)


@pytest.mark.parametrize("kappa", [1, 2, 3, KAPPA_W])
def test_convection_solve_history_matches_oracle(lib, kappa):
    n, levels, theta, eps, b = 255, 8, math.pi / 6, 1e-2, (100.0, -60.0)
    h, mg = make(lib, n, levels, theta, eps, b)
    f = rhs_uniform(n, 3)
    k = levels + 1 if kappa == KAPPA_W else kappa
    v_or, hist_or = oracle.solve(h, f, k, 1e-10, 300)
    vs, v = [], np.zeros_like(f)
    for _ in range(len(hist_or)):
        v = oracle.cycle(h, v, f, k)
        vs.append(v)
    vd = torch_dev(np.zeros((n, n)))
    st, cycles, relres, hist = mg.solve(vd, torch_dev(f), kappa, 1e-10, 300)
    assert st == 0 and cycles == len(hist_or)
    anorm, fn = np.abs(h.stencil(1)).sum(), np.linalg.norm(f)
    for i, (a, c) in enumerate(zip(hist, hist_or)):
        assert abs(a - c) <= HIST_TOL * c + ITER_TOL * anorm * np.linalg.norm(vs[i]) / fn, (i, a, c)
    assert rel(to_np(vd), v_or) <= ITER_TOL
    assert oracle.relres(h, to_np(vd), f) <= 1e-10


def test_convection_apply_and_residual_norm(lib):
    n, levels, theta, eps, b = 127, 7, 0.4, 1e-2, (-70.0, 30.0)
    h, mg = make(lib, n, levels, theta, eps, b)
    v, f = rhs_normal(n, 4), rhs_uniform(n, 5)
    out = torch_dev(np.zeros((n, n)))
    mg.apply(torch_dev(v), out)
    ref = oracle.apply_stencil(h.stencil(1), v)
    assert rel(to_np(out), ref) <= 1e-14
    assert abs(mg.residual_norm(torch_dev(v), torch_dev(f)) - np.linalg.norm(f - ref)) <= 1e-13 * np.linalg.norm(f - ref)


def test_convection_rejections(lib):
    n = 63
    mg = lib.Multigrid(n, 1e-2, 0.5, 6, convection=(10.0, 5.0), coarse_op="rediscretized")
    x, b = torch_dev(np.zeros((n, n))), torch_dev(rhs_uniform(n, 0))
    for call in (lambda: mg.pcg(x, b, 2, 1e-8, 10), lambda: mg.solve_mixed(x, b, 2, 1e-8, 10),
                 lambda: mg.kcycle_adjoint(x, b, 2), lambda: mg.set_option(lib.MG_OPT_SMOOTHER, 1)):
        with pytest.raises(lib.MultigridError):
            call()
    assert mg.get_option(lib.MG_OPT_CONV_X) == 10.0 and mg.get_option(lib.MG_OPT_CONV_Y) == 5.0
    mg.set_option(lib.MG_OPT_CONV_X, 0.0)
    mg.set_option(lib.MG_OPT_CONV_Y, 0.0)                    # back to the symmetric problem
    h = oracle.Hierarchy(n, 6, 0.5, 1e-2, coarse_op="rediscretized")
    mg.kcycle(x, b, 3)
    assert rel(to_np(x), oracle.cycle(h, np.zeros((n, n)), rhs_uniform(n, 0), 3)) <= ITER_TOL
