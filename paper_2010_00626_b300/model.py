"""Run-time model of the kappa-cycle (Section 3) and kappa pre-selection.

Paper form (eq. 3.1, Table 3):  T = alpha * N_gpuCalls + beta * N_ops, with
  levelCalls(kappa, l)  = sum_{j=0}^{min(kappa-1, l-1)} C(l-1, j)           (Proposition 2.2)
  totalCalls(kappa, n)  = sum_{j=1}^{min(kappa, n)} C(n, j)                   (Proposition 2.4)
  N_gpuCalls(kappa, n)  = (5+nu) totalCalls(kappa, n-1) + totalCalls(kappa, n) - totalCalls(kappa, n-1)
  N_ops(kappa, n)       = (2^n - 1)^2 * 2 (1 - 3^-kappa)                       (eq. 3.3)
alpha and beta come from a least-squares fit over measured per-cycle times (eq. 3.2); the turning
point n_tp where alpha N_gpuCalls = beta N_ops follows the Appendix's fixed-point iteration.

B300 form: this implementation launches two fused kernels per fine-level call, serves every call
at or below the coarse threshold inside one persistent kernel, and runs each call at the level just
above the threshold (not the finest) with its subtree as one cluster launch, so the per-call
overhead splits into a launch term and a coarse-call term:
  T = alpha_f * N_fine_launches + alpha_c * N_coarse_calls + beta * N_ops.
kappa pre-selection: argmin_kappa T(kappa) * ceil(log(tol) / log(rho_kappa)), with rho_kappa the
contraction per cycle estimated from the first cycles' residual history.
"""
from __future__ import annotations

import math

import numpy as np

W_COUNTER = 10 ** 6  # stands for kappa = infinity (the W-cycle) in these formulas


def level_calls(kappa: int, level: int) -> int:
    """Proposition 2.2 (level 1 finest)."""
    return sum(math.comb(level - 1, j) for j in range(0, min(kappa - 1, level - 1) + 1))


def total_calls(kappa: int, n: int) -> int:
    """Proposition 2.4."""
    return sum(math.comb(n, j) for j in range(1, min(kappa, n) + 1))


def n_gpu_calls(kappa: int, n: int, nu: int) -> int:
    """Kernel launches per cycle of the paper's implementation (Algorithm 4, Table 3)."""
    return (5 + nu) * total_calls(kappa, n - 1) + total_calls(kappa, n) - total_calls(kappa, n - 1)


def c_kappa(kappa: int) -> float:
    """C(kappa) = 2 (1 - 3^-kappa) of Table 3 (f(kappa, 1/4) of eq. 2.3)."""
    return 2.0 * (1.0 - 3.0 ** (-min(kappa, 60)))


def n_ops(kappa: int, n: int) -> float:
    """N_ops of Table 3: (2^n - 1)^2 C(kappa)."""
    return (2 ** n - 1) ** 2 * c_kappa(kappa)


def predict_paper(alpha: float, beta: float, kappa: int, n: int, nu: int) -> float:
    """Eq. 3.1: predicted time of one cycle (units of alpha and beta)."""
    return alpha * n_gpu_calls(kappa, n, nu) + beta * n_ops(kappa, n)


def fit_paper(samples, nu: int):
    """Eq. 3.2: least-squares (alpha, beta) from samples [(kappa, n, time), ...]."""
    A = np.array([[n_gpu_calls(k, n, nu), n_ops(k, n)] for k, n, _ in samples], dtype=float)
    t = np.array([s[2] for s in samples], dtype=float)
    (alpha, beta), *_ = np.linalg.lstsq(A, t, rcond=None)
    return float(alpha), float(beta)


def turning_point(alpha: float, beta: float, kappa: int, nu: int, iters: int = 20):
    """Appendix: iterate n <- log2(1 + sqrt((alpha/beta) N_gpuCalls(kappa, n) / C(kappa))) from n = 2;
    N_gpuCalls is evaluated on the real-valued n through the polynomial of Proposition 2.4
    (or 2^n - 1 for the W-cycle). Returns (n_tp, N_tp = (2^n_tp - 1)^2)."""
    def total_real(k, x):
        if k >= W_COUNTER:
            return 2.0 ** x - 1.0
        tot = 0.0
        for j in range(1, k + 1):  # C(x, j) as the degree-j polynomial x(x-1)...(x-j+1)/j!
            term = 1.0
            for i in range(j):
                term *= (x - i)
            tot += term / math.factorial(j)
        return tot

    def calls_real(k, x):
        return (5 + nu) * total_real(k, x - 1) + total_real(k, x) - total_real(k, x - 1)

    x = 2.0
    for _ in range(iters):
        x = math.log2(1.0 + math.sqrt((alpha / beta) * calls_real(kappa, x) / c_kappa(kappa)))
    return x, (2.0 ** x - 1.0) ** 2


# ------------------------------------------------------------------------------------------- B300
def b300_counts(kappa: int, levels: int, coarse_level: int, fused: bool = True):
    """(fine launches, coarse calls) of one cycle here: 2 launches per call on levels above the
    coarse threshold (0-based level < coarse_level), every call at or below it inside the coarse
    kernel; with fused calls, 1 launch per call at 0-based level coarse_level - 1 when that is not
    level 0 (pass A, the coarse walk and pass B in one cluster launch)."""
    top = min(coarse_level, levels)
    fine = sum((1 if fused and l == coarse_level - 1 and l >= 1 else 2) * level_calls(kappa, l + 1)
               for l in range(top))
    coarse = sum(level_calls(kappa, l + 1) for l in range(coarse_level, levels))
    return fine, coarse


def fit_b300(samples):
    """Least squares (alpha_f, alpha_c, beta) from [(fine_launches, coarse_calls, n_ops, time)]."""
    A = np.array([[s[0], s[1], s[2]] for s in samples], dtype=float)
    t = np.array([s[3] for s in samples], dtype=float)
    coef, *_ = np.linalg.lstsq(A, t, rcond=None)
    return tuple(float(c) for c in coef)


def predict_b300(params, kappa: int, levels: int, coarse_level: int, n_fine: int) -> float:
    af, ac, beta = params
    fine, coarse = b300_counts(kappa, levels, coarse_level)
    return af * fine + ac * coarse + beta * n_fine * n_fine * c_kappa(kappa)


def contraction(history, skip: int = 2) -> float:
    """Geometric-mean residual contraction per cycle over the history after `skip` cycles."""
    h = [x for x in history if x > 0]
    if len(h) < skip + 2:
        return h[-1] / h[0] if len(h) >= 2 else 0.5
    return (h[-1] / h[skip]) ** (1.0 / (len(h) - 1 - skip))


def preselect_kappa(time_per_cycle: dict, rho: dict, tol: float):
    """argmin_kappa time_per_cycle[kappa] * ceil(log(tol) / log(rho[kappa])); returns (kappa, table)."""
    table = {}
    for k, t in time_per_cycle.items():
        r = min(max(rho[k], 1e-16), 1 - 1e-12)
        table[k] = t * math.ceil(math.log(tol) / math.log(r))
    return min(table, key=table.get), table
