"""Seeded synthetic inputs shared by the tests, the bench and the oracle-side checks.

Holds no multigrid arithmetic: only random right-hand sides, parameter draws and the
workload definitions (grid sizes, angles, anisotropies, cycle counters) of the
rotated anisotropic diffusion problems the solver is measured on. Every array comes from
``numpy.random.default_rng(seed)`` (PCG64), row-major, float64, index [j, i] with i the
x index and j the y index.
"""
from __future__ import annotations

import math

import numpy as np

KAPPA_W = 0x7FFFFFFF  # any counter >= the number of levels gives the W-cycle (Proposition 2.1)


def rhs_uniform(n: int, seed: int = 0) -> np.ndarray:
    """f ~ U(-1, 1) on the n x n interior grid."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(n, n))


def rhs_normal(n: int, seed: int = 0) -> np.ndarray:
    """f ~ N(0, 1) on the n x n interior grid."""
    return np.random.default_rng(seed).standard_normal((n, n))


def levels_for(n: int) -> int:
    """Number of factor-2 levels down to a 1x1 coarsest grid for n = 2^k - 1 (k levels)."""
    k = int(round(math.log2(n + 1)))
    if (1 << k) - 1 != n:
        raise ValueError("n must be 2^k - 1")
    return k


# Workloads (all synthetic; the paper's test problems are synthetic PDEs, Section 4).
SMALL = dict(name="small standalone 127^2", n=127, levels=7, theta=math.pi / 6, eps=1e-2,
             nu1=2, nu2=2, omega=0.8, rhs="uniform", seed=0, cycles=20, kappas=(1, 2, 3, KAPPA_W))
LARGE = dict(name="large standalone 4095^2", n=4095, levels=12, theta=math.pi / 3, eps=1e-4,
             nu1=2, nu2=2, omega=0.8, rhs="normal", seed=0, tol=1e-8, kappas=(1, 2, 3, 4, 5, KAPPA_W))
PCG_LARGE = dict(name="MGCG 8191^2", n=8191, levels=13, eps=(1e-3, 1e-5), nu1=2, nu2=2, omega=0.8,
                 rhs="normal", seeds=(0, 1, 2, 3, 4), tol=1e-10, kappas=(1, 2, 3, 4))
AUTOGRAD = dict(name="differentiable 1023^2", n=1023, levels=10, theta=0.7, eps=1e-3, kappa=3,
                cycles=10, tol=1e-10, target_seed=1, fd_n=63)


def pcg_theta(seed: int) -> float:
    """theta ~ U[0, pi) for the MGCG workload, one draw per seed."""
    return float(np.random.default_rng(seed).uniform(0.0, math.pi))


def batched_instances(count: int = 256, seed: int = 0, sizes=(127, 255, 511, 1023)):
    """Batched workload: per instance (n, theta, eps, f-seed).

    n uniform over ``sizes``; theta ~ U[0, pi); log10(eps) ~ U[-5, -1]; the right-hand
    side of instance i is ``rhs_uniform(n, seed * 100003 + i + 1)``.
    """
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=count)
    thetas = rng.uniform(0.0, math.pi, size=count)
    epss = 10.0 ** rng.uniform(-5.0, -1.0, size=count)
    return [dict(n=int(ns[i]), theta=float(thetas[i]), eps=float(epss[i]), seed=seed * 100003 + i + 1)
            for i in range(count)]
