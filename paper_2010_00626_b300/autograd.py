"""Differentiable kappa-cycle solve: a torch.autograd.Function over the C ABI.

forward:  u = A(theta, eps)^{-1} f by the stand-alone kappa-cycle solver (to ``tol``), or the
          result of exactly ``cycles`` cycles from zero.
backward: lambda = A^{-T} g by adjoint kappa-cycles (mg_solve_adjoint, or ``cycles`` adjoint
          cycles from zero, the exact transpose of the forward map in that mode); then
          dL/df = lambda and dL/dp = -lambda^T (dA/dp) u for p = theta, eps (mg_param_grads).
          In fixed-cycle mode dL/dtheta and dL/deps are the implicit-function approximation.
torch provides device memory and streams only; every step runs in the library's kernels.
"""
from __future__ import annotations

import torch

from . import kcycle

_cache: dict = {}


def _handle(n, levels, theta, eps, nu1, nu2):
    key = (n, levels, float(theta), float(eps), nu1, nu2)
    mg = _cache.get(key)
    if mg is None:
        if len(_cache) >= 4:
            _cache.pop(next(iter(_cache))).close()
        mg = kcycle.Multigrid(n, float(eps), float(theta), levels, nu1, nu2)
        _cache[key] = mg
    return mg


class KCycleSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, theta, eps, levels, kappa, tol, max_cycles, cycles, nu1, nu2):
        n = f.shape[-1]
        mg = _handle(n, levels, float(theta), float(eps), nu1, nu2)
        f = f.contiguous()
        u = torch.zeros_like(f)
        if cycles is None:
            st, _, rel, _ = mg.solve(u, f, kappa, tol, max_cycles, history=False)
            if st != kcycle.MG_OK:
                raise kcycle.MultigridError(f"forward solve did not reach {tol} (relres {rel})")
        else:
            for _ in range(cycles):
                mg.kcycle(u, f, kappa)
        ctx.save_for_backward(u)
        ctx.mg, ctx.kappa, ctx.tol, ctx.max_cycles, ctx.cycles = mg, kappa, tol, max_cycles, cycles
        return u

    @staticmethod
    def backward(ctx, g):
        (u,) = ctx.saved_tensors
        mg = ctx.mg
        g = g.contiguous()
        lam = torch.zeros_like(g)
        if ctx.cycles is None:
            st, _, rel, _ = mg.solve(lam, g, ctx.kappa, ctx.tol, ctx.max_cycles, history=False, adjoint=True)
            if st != kcycle.MG_OK:
                raise kcycle.MultigridError(f"adjoint solve did not reach {ctx.tol} (relres {rel})")
        else:
            for _ in range(ctx.cycles):
                mg.kcycle_adjoint(lam, g, ctx.kappa)
        dth, dep = mg.param_grads(lam, u)
        dtype = torch.float64
        return (lam, torch.tensor(dth, dtype=dtype, device=g.device), torch.tensor(dep, dtype=dtype, device=g.device),
                None, None, None, None, None, None, None)


def kcycle_solve(f, theta, eps, levels, kappa=3, tol=1e-10, max_cycles=10000, cycles=None, nu1=2, nu2=2):
    """u = A(theta, eps)^{-1} f, differentiable in f, theta and eps.

    theta and eps should be float64 tensors (a float32 tensor would round the angle); f is a
    float64 CUDA tensor of shape (n, n)."""
    return KCycleSolve.apply(f, theta, eps, levels, kappa, tol, max_cycles, cycles, nu1, nu2)
