"""Write the oracle's stand-alone solve of the 4095^2 problem (12 levels, theta=pi/3, eps=1e-4,
f ~ N(0,1) seed 0, v0 = 0, nu1 = nu2 = 2, omega = 0.8) as a golden file: its residual history and
the cycles it needs to reach a 1e-8 relative residual.

    python -m oracle.full_size_cycles KAPPA                 -> tests/golden/large_standalone_cycles_k<KAPPA>.json
    python -m oracle.full_size_cycles KAPPA --first N       -> tests/golden/large_standalone_first<N>_k<KAPPA>.json
                                                               (the first N cycles only, tolerance not applied)

Calls only oracle/ and the seeded input generator. Slow (minutes to hours per kappa on one core).
"""
import json
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2010_00626_b300.inputs import rhs_normal  # noqa: E402


def main():
    kappa = int(sys.argv[1])
    first = int(sys.argv[sys.argv.index("--first") + 1]) if "--first" in sys.argv else None
    n, levels, theta, eps, tol = 4095, 12, math.pi / 3, 1e-4, 1e-8
    h = oracle.Hierarchy(n, levels, theta, eps)
    f = rhs_normal(n, 0)
    t0 = time.time()
    if first:
        _, hist = oracle.solve(h, f, kappa, 0.0, first)
        name = f"large_standalone_first{first}_k{kappa}.json"
    else:
        _, hist = oracle.solve(h, f, kappa, tol, 20000)
        name = f"large_standalone_cycles_k{kappa}.json"
    out = dict(workload="large standalone 4095^2", n=n, levels=levels, theta=theta, eps=eps,
               tol=None if first else tol, kappa=kappa, cycles=len(hist), history=hist,
               seconds=time.time() - t0, written_by="oracle/full_size_cycles.py")
    path = os.path.join(ROOT, "tests", "golden", name)
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(path, len(hist), out["seconds"])


if __name__ == "__main__":
    main()
