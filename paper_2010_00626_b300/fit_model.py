"""Fit the Section 3 run-time model to this GPU and pre-select kappa.

    python -m paper_2010_00626_b300.fit_model [--max-levels 13] [--reps 3]

Measures the FP64 per-cycle time of the 2^L - 1 grid (theta = pi/4, eps = 1e-4, as in Section
3.1's tests) for L = 4..max-levels and kappa in {1, 2, 3, 4, W} with CUDA events around graph
launches, then fits T = alpha N_gpuCalls + beta N_ops (eq. 3.2, the paper's counts) and the B300
form T = alpha_f N_fine_launches + alpha_c N_coarse_calls + beta N_ops, and prints one JSON line
with the parameters, the relative prediction errors (as in Table 2) and the turning points (as in
Table 1).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2010_00626_b300 import model  # noqa: E402

KAPPAS = (1, 2, 3, 4, model.W_COUNTER)


def measure(max_levels=13, reps=3, kappas=KAPPAS, theta=math.pi / 4, eps=1e-4):
    """[(kappa, L, ms_per_cycle, fine_launches, coarse_calls)] for L = 4..max_levels."""
    import torch
    from paper_2010_00626_b300 import kcycle
    from paper_2010_00626_b300.inputs import rhs_normal
    out = []
    for L in range(4, max_levels + 1):
        n = 2 ** L - 1
        mg = kcycle.Multigrid(n, eps, theta, L)
        mg.set_option(kcycle.MG_OPT_DEEP_CALLS, 0)  # the launch-by-launch form whose launches the model counts
        f = torch.tensor(rhs_normal(n, 0), device="cuda")
        v = torch.zeros_like(f)
        lc = None
        for k in kappas:
            kk = min(k, kcycle.MG_KAPPA_W)
            mg.kcycle(v, f, kk)  # builds the graph
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                mg.kcycle(v, f, kk)
            b.record()
            torch.cuda.synchronize()
            if lc is None:  # first level handled by the coarse kernel
                lc = next((l for l in range(L) if _is_coarse(mg, l)), L - 1)
            fine_launches, coarse_calls = model.b300_counts(k, L, lc)
            out.append((k, L, a.elapsed_time(b) / reps, fine_launches, coarse_calls))
        mg.close()
    return out


def _is_coarse(mg, level):
    from paper_2010_00626_b300 import kcycle
    n_l = (mg.n + 1) // (2 ** level) - 1
    return n_l <= mg.get_option(kcycle.MG_OPT_COARSE_N)


def fit(samples, nu=4):
    paper = model.fit_paper([(k, L, t) for k, L, t, _, _ in samples], nu)
    b300 = model.fit_b300([(fl, cc, model.n_ops(k, L), t) for k, L, t, fl, cc in samples])
    errors = {}
    for k, L, t, fl, cc in samples:
        pred = b300[0] * fl + b300[1] * cc + b300[2] * model.n_ops(k, L)
        errors.setdefault("W" if k >= model.W_COUNTER else str(k), {})[L] = round((pred - t) / t, 4)
    tp = {("W" if k >= model.W_COUNTER else str(k)): round(model.turning_point(paper[0], paper[1], k, nu)[0], 2)
          for k in KAPPAS}
    return {"paper_form": {"alpha_ms": paper[0], "beta_ms": paper[1], "turning_point_levels": tp},
            "b300_form": {"alpha_fine_launch_ms": b300[0], "alpha_coarse_call_ms": b300[1], "beta_ms": b300[2],
                          "relative_errors": errors}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--max-levels", type=int, default=13)
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    samples = measure(args.max_levels, args.reps)
    res = fit(samples)
    res["samples"] = [{"kappa": ("W" if k >= model.W_COUNTER else k), "levels": L, "ms": round(t, 4)}
                      for k, L, t, _, _ in samples]
    print(json.dumps(res))


if __name__ == "__main__":
    main()
