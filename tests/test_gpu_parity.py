"""GPU parity: the CUDA path through the C ABI against the FP64 oracle (needs a B300).

Tolerances (floating point):
* iterates: ||v_gpu - v_oracle|| / ||v_oracle|| <= 1e-12 after every cycle;
* relative-residual histories: |rho_gpu - rho_oracle| <= 1e-10 rho_oracle + floor_k, where
  floor_k = 1e-12 ||A||_inf ||v_k||_2 / ||f||_2 is the residual change that the 1e-12 iterate
  bound allows (it only matters once rho nears the FP64 rounding floor);
* stencils: bit for bit (each entry is rounded once from an exactly defined value; a one-ulp
  row-sum difference would act on smooth modes like a zeroth-order term of relative size
  ulp(c0)/lambda_min, about 1e-10 at 4095^2, which is why this is exact rather than a tolerance);
* MGCG: as the stand-alone histories with 1e-10, and x within 1e-10.
Integers (call counts, cycle counts) are compared exactly.
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
        floor = ITER_TOL * anorm * np.linalg.norm(vs[k]) / fn
        assert abs(a - b) <= HIST_TOL * b + floor, (k, a, b)


def kappa_eff(kappa, levels):
    return levels + 1 if kappa == KAPPA_W else kappa


@pytest.mark.parametrize("n,levels,theta,eps", [
    (127, 7, math.pi / 6, 1e-2), (127, 6, math.pi / 6, 1e-2), (4095, 12, math.pi / 3, 1e-4),
    (1023, 10, 0.7, 1e-3), (63, 4, 2.5, 0.3), (8191, 13, 2.998934482165474, 1e-5),
    (255, 8, 0.0, 1.0), (255, 8, math.pi / 2, 1e-3)])
def test_stencils_match_oracle(lib, n, levels, theta, eps):
    """Every stencil entry is rounded once from an exactly defined value on both sides
    (correctly rounded cos/sin, exact Galerkin sums, zero-row-sum centres), so the device
    stencils equal the oracle's bit for bit at every level."""
    mg = lib.Multigrid(n, eps, theta, levels)
    h = oracle.Hierarchy(n, levels, theta, eps)
    st = mg.stencils()
    for l in range(levels):
        assert np.array_equal(st[l], h.stencils[l]), (l, st[l] - h.stencils[l])


@pytest.mark.parametrize("levels", [7, 6])
@pytest.mark.parametrize("kappa", [1, 2, 3, KAPPA_W])
def test_small_standalone_per_iterate(lib, levels, kappa):
    """127^2, theta=pi/6, eps=1e-2, nu=2+2, omega=0.8, f~U(-1,1) seed 0, v0=0, 20 cycles."""
    n, theta, eps = 127, math.pi / 6, 1e-2
    h = oracle.Hierarchy(n, levels, theta, eps)
    f = rhs_uniform(n, 0)
    mg = lib.Multigrid(n, eps, theta, levels)
    fd, vd = torch_dev(f), torch_dev(np.zeros((n, n)))
    v = np.zeros((n, n))
    k = kappa_eff(kappa, levels)
    for c in range(20):
        v = oracle.cycle(h, v, f, k)
        mg.kcycle(vd, fd, kappa)
        err = rel(to_np(vd), v)
        assert err <= ITER_TOL, (c, err)


@pytest.mark.parametrize("coarse_n", [1, 3, 7, 15, 31, 63])
def test_coarse_threshold_does_not_change_iterates(lib, coarse_n):
    n, levels, theta, eps = 63, 6, 1.1, 1e-3
    h = oracle.Hierarchy(n, levels, theta, eps)
    f = rhs_normal(n, 3)
    mg = lib.Multigrid(n, eps, theta, levels, coarse_n=coarse_n)
    fd, vd = torch_dev(f), torch_dev(np.zeros((n, n)))
    v = np.zeros((n, n))
    for kappa in (3, 1, 6, 2):
        for _ in range(2):
            v = oracle.cycle(h, v, f, kappa)
            mg.kcycle(vd, fd, kappa)
            assert rel(to_np(vd), v) <= ITER_TOL


@pytest.mark.parametrize("n,levels", [(255, 8), (511, 9), (1023, 10), (511, 6), (3, 2), (1, 1), (7, 3)])
def test_ragged_and_degenerate_sizes(lib, n, levels):
    """Sizes whose tiles end in a ragged tail, coarsest grids above 1x1, and tiny grids."""
    theta, eps = 0.9, 5e-3
    h = oracle.Hierarchy(n, levels, theta, eps)
    f = rhs_uniform(n, 4)
    v0 = rhs_normal(n, 5) * 1e-3
    mg = lib.Multigrid(n, eps, theta, levels)
    fd, vd = torch_dev(f), torch_dev(v0)
    v = v0.copy()
    for kappa in (2, 4):
        v = oracle.cycle(h, v, f, kappa)
        mg.kcycle(vd, fd, kappa)
        assert rel(to_np(vd), v) <= ITER_TOL


@pytest.mark.parametrize("nu", [(2, 2), (1, 3), (0, 2), (3, 0)])
def test_smoothing_counts_and_adjoint(lib, nu):
    n, levels, theta, eps = 127, 7, 0.7, 1e-3
    h = oracle.Hierarchy(n, levels, theta, eps, nu1=nu[0], nu2=nu[1])
    f = rhs_normal(n, 6)
    mg = lib.Multigrid(n, eps, theta, levels, nu1=nu[0], nu2=nu[1])
    fd = torch_dev(f)
    for kappa in (1, 3):
        vd = torch_dev(np.zeros((n, n)))
        mg.kcycle(vd, fd, kappa)
        assert rel(to_np(vd), oracle.cycle(h, np.zeros((n, n)), f, kappa)) <= ITER_TOL
        vd = torch_dev(np.zeros((n, n)))
        mg.kcycle_adjoint(vd, fd, kappa)
        assert rel(to_np(vd), oracle.cycle_adjoint(h, np.zeros((n, n)), f, kappa)) <= ITER_TOL


@pytest.mark.parametrize("kappa", [1, 2, 3, KAPPA_W])
def test_solve_history_matches_oracle(lib, kappa):
    n, levels, theta, eps = 127, 7, math.pi / 6, 1e-2
    h = oracle.Hierarchy(n, levels, theta, eps)
    f = rhs_uniform(n, 0)
    k = kappa_eff(kappa, levels)
    v_or, hist_or = oracle.solve(h, f, k, 1e-8, 300)
    vs, v = [], np.zeros_like(f)
    for _ in range(len(hist_or)):
        v = oracle.cycle(h, v, f, k)
        vs.append(v)
    mg = lib.Multigrid(n, eps, theta, levels)
    vd = torch_dev(np.zeros((n, n)))
    st, cycles, relres, hist = mg.solve(vd, torch_dev(f), kappa, 1e-8, 300)
    assert st == 0 and cycles == len(hist_or)
    hist_ok(hist, hist_or, h, vs, f)
    assert rel(to_np(vd), v_or) <= ITER_TOL
    assert oracle.relres(h, to_np(vd), f) <= 1e-8


def test_solve_not_converged_status(lib):
    n, levels = 63, 6
    mg = lib.Multigrid(n, 1e-4, 1.0, levels)
    f = rhs_uniform(n, 1)
    st, cycles, relres, hist = mg.solve(torch_dev(np.zeros((n, n))), torch_dev(f), 1, 1e-14, 3)
    assert st == 1 and cycles == 3 and relres > 1e-14 and len(hist) == 3


def test_solve_host_buffers(lib):
    n, levels, theta, eps = 255, 8, 0.4, 1e-2
    h = oracle.Hierarchy(n, levels, theta, eps)
    f = rhs_uniform(n, 2)
    v = np.zeros((n, n))
    mg = lib.Multigrid(n, eps, theta, levels)
    st, cycles, relres = mg.solve_host(v, f, 3, 1e-9, 200)
    assert st == 0 and relres <= 1e-9
    assert oracle.relres(h, v, f) <= 1e-9
    v_or, hist_or = oracle.solve(h, f, 3, 1e-9, 200)
    assert cycles == len(hist_or)
    assert rel(v, v_or) <= ITER_TOL


@pytest.mark.parametrize("kappa,flexible", [(1, False), (3, False), (2, True), (KAPPA_W, False)])
def test_pcg_matches_oracle(lib, kappa, flexible):
    n, levels, theta, eps = 255, 8, 2.0, 1e-3
    h = oracle.Hierarchy(n, levels, theta, eps)
    b = rhs_normal(n, 7)
    k = kappa_eff(kappa, levels)
    x_or, hist_or = oracle.pcg(h, b, k, 1e-10, 200, flexible=flexible)
    mg = lib.Multigrid(n, eps, theta, levels)
    xd = torch_dev(np.zeros((n, n)))
    st, iters, relres, hist = mg.pcg(xd, torch_dev(b), kappa, 1e-10, 200, flexible=flexible)
    assert st == 0 and iters == len(hist_or)
    for a, c in zip(hist, hist_or):
        assert abs(a - c) <= HIST_TOL * c + 1e-15, (a, c)
    assert rel(to_np(xd), x_or) <= 1e-10
    assert oracle.relres(h, to_np(xd), b) <= 1e-10


def test_apply_and_residual_norm(lib):
    n, levels, theta, eps = 511, 9, 1.3, 1e-4
    h = oracle.Hierarchy(n, levels, theta, eps)
    v, f = rhs_normal(n, 8), rhs_uniform(n, 9)
    mg = lib.Multigrid(n, eps, theta, levels)
    out = torch_dev(np.zeros((n, n)))
    mg.apply(torch_dev(v), out)
    Av = oracle.apply_stencil(h.stencil(1), v)
    assert rel(to_np(out), Av) <= 1e-14 * np.abs(h.stencil(1)).sum() * np.linalg.norm(v) / np.linalg.norm(Av) + 1e-15
    r = mg.residual_norm(torch_dev(v), torch_dev(f))
    assert abs(r - np.linalg.norm(f - Av)) <= 1e-12 * r


def test_param_grads_match_oracle(lib):
    n, levels, theta, eps = 255, 8, 0.7, 1e-3
    lam, u = rhs_normal(n, 10), rhs_normal(n, 11)
    mg = lib.Multigrid(n, eps, theta, levels)
    g = mg.param_grads(torch_dev(lam), torch_dev(u))
    ref = oracle.param_grads(theta, eps, n, lam, u)
    for a, b in zip(g, ref):
        assert abs(a - b) <= 1e-10 * abs(b)


@pytest.mark.parametrize("kappa", [1, 2, 3, 4, 5, KAPPA_W])
def test_counters_match_closed_forms(lib, kappa):
    n, levels = 4095, 12
    mg = lib.Multigrid(n, 1e-4, math.pi / 3, levels)
    calls, launches, coarse = mg.counters(kappa)
    k = kappa_eff(kappa, levels)
    for l in range(levels):
        assert calls[l] == sum(math.comb(l, j) for j in range(0, min(k - 1, l) + 1))
    assert sum(calls) == sum(math.comb(levels, j) for j in range(1, min(k, levels) + 1))
    # the graph of one cycle launches exactly the counted kernels
    v, f = torch_dev(np.zeros((n, n))), torch_dev(rhs_normal(n, 0))
    mg.kcycle(v, f, kappa)
    assert mg.get_option(lib.MG_OPT_LAUNCHES) == launches


def test_level_grid_reports_the_launch_shapes(lib):
    """CTAs per pass launch at 4095^2: 64x32 tiles at 4095 and 2047 (about two waves), 32^2 at 1023,
    one tile per SM at 511 and 255 (FP64: 12^2 tiles of 44^2 and 22^2 on 148 SMs), 8^2 below, one
    coarse-kernel CTA at 15^2 and below. FP32:
    the persistent tensor-copy passes at 4095, 2047 and 1023 (one CTA per SM: 2240, 576 and 288
    tiles of 120 columns), the FP32 coarse kernel from 31^2; with MG_OPT_TMA_PASSES = 0 pass B as
    the register pipelines at 4095 (35 strips of 120 columns, 4 per CTA, chunks of 64 rows) and the
    shared-memory tiles of 112 x 16 at 2047. The level just above the coarse kernel runs its calls
    as one cluster launch: 16 CTAs of 8^2 tiles at 31^2 (FP64 with the coarse kernel at 15^2), of
    16^2 tiles at 63^2 (FP32); without the fused calls 64 CTAs at 63^2 (FP32). With the default FP64
    coarse kernel at 31^2, the 63^2 level keeps its 64 tiles (a fused call would need at most 16)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count

    def one_per_sm(n, old):  # the smallest even edge with at most one tile per SM, where built
        tiles = lambda b: ((n + b - 1) // b) ** 2
        b = next(b for b in range(2, 66, 2) if tiles(b) <= sms or b == 64)
        return tiles(b) if b in (44, 22) and tiles(b) <= sms else old

    wide = [one_per_sm(511, 16 * 16), one_per_sm(255, 16 * 16)]
    assert sms != 148 or wide == [144, 144]
    default = lib.Multigrid(4095, 1e-4, math.pi / 3, 12)
    grid = [default.level_grid(l)[1] for l in range(12)]
    # the 127^2 and 63^2 levels inside the persistent deep launches (one or two CTAs per SM)
    assert grid[:5] == [64 * 128, 32 * 64, 32 * 32] + wide and grid[7:] == [1] * 5
    assert grid[5] == grid[6] and grid[5] in (sms, 2 * sms)
    default.set_option(lib.MG_OPT_DEEP_CALLS, 0)
    assert [default.level_grid(l)[1] for l in range(5, 8)] == [16 * 16, 8 * 8, 1]
    mg = lib.Multigrid(4095, 1e-4, math.pi / 3, 12, coarse_n=15)
    mg.set_option(lib.MG_OPT_DEEP_CALLS, 0)
    fp64 = [mg.level_grid(l) for l in range(12)]
    assert [c for _, c in fp64] == [64 * 128, 32 * 64, 32 * 32] + wide + [16 * 16, 8 * 8, 4 * 4, 1, 1, 1, 1]
    assert [m for m, _ in fp64] == [2 ** (12 - l) - 1 for l in range(12)]
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    fp32 = [mg.level_grid(l, fp32=True)[1] for l in range(12)]
    assert fp32[5] == 16 * 16 and fp32[6] == 16 and fp32[7:] == [1] * 5
    assert all(0 < c <= 3 * sms for c in fp32[:3])
    mg.set_option(lib.MG_OPT_FUSED_CALL, 2)
    assert mg.level_grid(6)[1] == 16 and mg.level_grid(5, fp32=True)[1] == 16
    mg.set_option(lib.MG_OPT_TMA_PASSES, 0)
    assert [mg.level_grid(l, fp32=True)[1] for l in range(2)] == [9 * 64, 19 * 128]
    mg.set_option(lib.MG_OPT_FUSED_CALL, 0)
    assert mg.level_grid(6, fp32=True)[1] == 64 and mg.level_grid(7)[1] == 16
    zebra = lib.Multigrid(127, 1e-4, math.pi / 3, 7, smoother="zebra")
    with pytest.raises(lib.MultigridError):
        zebra.level_grid(0)


def test_bad_arguments(lib):
    mg = lib.Multigrid(31, 1e-2, 0.5, 5)
    v, f = torch_dev(np.zeros((31, 31))), torch_dev(rhs_uniform(31, 0))
    with pytest.raises(lib.MultigridError):
        mg.kcycle(v, f, 0)
    with pytest.raises(lib.MultigridError):
        mg.solve(v, f, 1, 0.0, 10)
    with pytest.raises(lib.MultigridError):
        mg.pcg(v, f, 1, 1e-8, 0)
    with pytest.raises(lib.MultigridError):
        mg.set_option(lib.MG_OPT_COARSE_N, 5)


@pytest.mark.parametrize("kappa", [1, 4, KAPPA_W])
def test_large_one_cycle_matches_oracle(lib, kappa):
    """4095^2, 12 levels, theta=pi/3, eps=1e-4, f~N(0,1): the first cycle, whole array."""
    n, levels, theta, eps = 4095, 12, math.pi / 3, 1e-4
    h = oracle.Hierarchy(n, levels, theta, eps)
    f = rhs_normal(n, 0)
    mg = lib.Multigrid(n, eps, theta, levels)
    vd = torch_dev(np.zeros((n, n)))
    mg.kcycle(vd, torch_dev(f), kappa)
    v = oracle.cycle(h, np.zeros((n, n)), f, kappa_eff(kappa, levels))
    assert rel(to_np(vd), v) <= ITER_TOL


def test_large_solve_reaches_tolerance(lib):
    """4095^2 solve to 1e-8 with kappa=4; the oracle recomputes the residual of the result."""
    n, levels, theta, eps = 4095, 12, math.pi / 3, 1e-4
    h = oracle.Hierarchy(n, levels, theta, eps)
    f = rhs_normal(n, 0)
    mg = lib.Multigrid(n, eps, theta, levels)
    vd = torch_dev(np.zeros((n, n)))
    st, cycles, relres, hist = mg.solve(vd, torch_dev(f), 4, 1e-8, 3000)
    assert st == 0 and relres <= 1e-8
    assert all(b < a for a, b in zip(hist, hist[1:]))
    assert oracle.relres(h, to_np(vd), f) <= 1e-8 * (1 + 1e-6)


@pytest.mark.parametrize("kappa", [1, 2, 3, 4, 5, KAPPA_W])
def test_large_solve_matches_oracle_cycle_counts(lib, kappa):
    """4095^2 solves against the oracle's own full-size runs (tests/golden, written by
    oracle/full_size_cycles.py): identical cycle counts and residual histories."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", f"large_standalone_cycles_k{kappa_eff(kappa, 12)}.json")
    if not os.path.exists(path):
        pytest.skip("no oracle run stored for this counter")
    g = json.load(open(path))
    n, levels = g["n"], g["levels"]
    mg = lib.Multigrid(n, g["eps"], g["theta"], levels)
    vd = torch_dev(np.zeros((n, n)))
    st, cycles, relres, hist = mg.solve(vd, torch_dev(rhs_normal(n, 0)), kappa, g["tol"], max(3000, g["cycles"] + 100))
    assert st == 0 and cycles == g["cycles"]
    # iterates agree to 1e-12, so the histories agree to that bound relative to the early
    # residuals, which is far below 1e-10 of the late ones
    for a, b in zip(hist, g["history"]):
        assert abs(a - b) <= HIST_TOL * b + 1e-12 * g["history"][0], (a, b)


def test_large_vcycle_history_matches_oracle_first_200_cycles(lib):
    """4095^2 V-cycles (kappa = 1, the slowest counter: 4115 cycles to 1e-8, Table 4's first row)
    against the oracle's own first 200 cycles of the same solve (tests/golden, written by
    oracle/full_size_cycles.py --first 200): the residual history cycle by cycle."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "large_standalone_first200_k1.json")))
    n, levels = g["n"], g["levels"]
    mg = lib.Multigrid(n, g["eps"], g["theta"], levels)
    vd = torch_dev(np.zeros((n, n)))
    st, cycles, relres, hist = mg.solve(vd, torch_dev(rhs_normal(n, 0)), 1, 1e-300, g["cycles"])
    assert st == 1 and cycles == g["cycles"] == 200
    for a, b in zip(hist, g["history"]):
        assert abs(a - b) <= HIST_TOL * b + 1e-12 * g["history"][0], (a, b)


def test_largest_grid_solve(lib):
    """16383^2 (14 levels, the paper's largest): kappa=3 solve to 1e-8; the oracle recomputes the
    residual of the result (a property that holds at any size)."""
    n, levels, theta, eps = 16383, 14, math.pi / 3, 1e-4
    f = rhs_normal(n, 0)
    mg = lib.Multigrid(n, eps, theta, levels)
    vd = torch_dev(np.zeros((n, n)))
    st, cycles, relres, hist = mg.solve(vd, torch_dev(f), 3, 1e-8, 3000, history=False)
    assert st == 0 and relres <= 1e-8
    st_fine = oracle.fine_stencil(theta, eps, n)
    r = f - oracle.apply_stencil(st_fine, to_np(vd))
    assert np.linalg.norm(r) / np.linalg.norm(f) <= 1e-8 * (1 + 1e-6)


def test_rediscretized_hierarchy_and_error_protocol(lib):
    """Coarse operators rediscretized (Section 4 stencil at each coarse h): stencils bit for bit,
    iterates to 1e-12; the error-reduction protocol (f = 0, random start, ||v_k|| / ||v_0||) gives
    the oracle's cycle count and history."""
    n, levels, theta, eps = 255, 8, math.pi / 4, 1e-3
    h = oracle.Hierarchy(n, levels, theta, eps, coarse_op="rediscretized")
    mg = lib.Multigrid(n, eps, theta, levels)
    mg.set_option(lib.MG_OPT_COARSE_OP, 1)
    st = mg.stencils()
    for l in range(levels):
        assert np.array_equal(st[l], h.stencils[l]), l
    f = rhs_uniform(n, 3)
    vd, v = torch_dev(np.zeros((n, n))), np.zeros((n, n))
    for kappa in (1, 3, 9):
        v = oracle.cycle(h, v, f, kappa)
        mg.kcycle(vd, torch_dev(f), kappa)
        assert rel(to_np(vd), v) <= ITER_TOL
    v0 = np.random.default_rng(4).uniform(-1.0, 1.0, (n, n))
    _, hist_or = oracle.solve_error_reduction(h, v0, 3, 1e-8, 2000)
    mg.set_option(lib.MG_OPT_STOP, 1)
    st_, cycles, red, hist = mg.solve(torch_dev(v0), torch_dev(np.zeros((n, n))), 3, 1e-8, 2000)
    assert st_ == 0 and cycles == len(hist_or) and red <= 1e-8
    for a, b in zip(hist, hist_or):
        assert abs(a - b) <= HIST_TOL * b + ITER_TOL


@pytest.mark.parametrize("kappa", [2, 3, 4])
def test_symmetrised_pcg_matches_oracle(lib, kappa):
    """MGCG with M = B + B^T - B^T A B (a cycle, the residual, an adjoint cycle)."""
    n, levels, theta, eps = 255, 8, 0.7, 1e-4
    h = oracle.Hierarchy(n, levels, theta, eps)
    b = rhs_uniform(n, 7)
    x_or, hist_or = oracle.pcg(h, b, kappa, 1e-10, 200, symmetric=True)
    mg = lib.Multigrid(n, eps, theta, levels)
    mg.set_option(lib.MG_OPT_PRECOND, 1)
    xd = torch_dev(np.zeros((n, n)))
    st, iters, relres, hist = mg.pcg(xd, torch_dev(b), kappa, 1e-10, 200)
    assert st == 0 and iters == len(hist_or)
    for a, c in zip(hist, hist_or):
        assert abs(a - c) <= HIST_TOL * c + 1e-13
    assert rel(to_np(xd), x_or) <= 1e-10
    with pytest.raises(lib.MultigridError):
        mg.pcg(xd, torch_dev(b), kappa, 1e-10, 200, mixed=True)
    mg.set_option(lib.MG_OPT_SMOOTHER, 1)
    with pytest.raises(lib.MultigridError):
        mg.pcg(xd, torch_dev(b), kappa, 1e-10, 200)
