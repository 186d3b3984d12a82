"""Run a fixed number of kappa-cycles on one synthetic problem through the C ABI, for profiling.

    python -m paper_2010_00626_b300.run_cycles --n 4095 --levels 12 --kappa 4 --cycles 1 \
        [--smoother zebra] [--coarsening y] [--theta 1.0471975511965976] [--eps 1e-4] [--fp32] [--solve]
        [--mixed]

The right-hand side is f ~ N(0, 1) (seed 0) and the start v = 0. With --fp32 the cycles are the
FP32 cycles of the mixed forms (mg_kcycle_f32). Prints one JSON line with the wall time; the
numbers meant for reports come from CUDA events in bench.py, this only drives a profiler.
"""
import argparse
import json
import math
import time


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=4095)
    ap.add_argument("--levels", type=int, default=0, help="0: down to 1x1")
    ap.add_argument("--kappa", type=int, default=4)
    ap.add_argument("--cycles", type=int, default=1)
    ap.add_argument("--theta", type=float, default=math.pi / 3)
    ap.add_argument("--eps", type=float, default=1e-4)
    ap.add_argument("--smoother", default="jacobi", choices=["jacobi", "zebra", "xzebra"])
    ap.add_argument("--coarsening", default="full", choices=["full", "y"])
    ap.add_argument("--fp32", action="store_true")
    ap.add_argument("--mixed", action="store_true", help="run the FP32 cycle of the mixed solve launch by launch on "
                                                          "the handle's own FP32 arrays (16-byte pitches), as "
                                                          "mg_profile_cycle does")
    ap.add_argument("--solve", action="store_true", help="run the launches of stand-alone solve cycles (with the "
                                                         "stopping test's norm) one by one, as mg_profile_cycle "
                                                         "does, instead of bare cycles (a solve's own graph has "
                                                         "conditional nodes, whose kernels profilers skip)")
    args = ap.parse_args()

    import torch

    from paper_2010_00626_b300 import build
    build.build()
    from paper_2010_00626_b300 import kcycle
    from paper_2010_00626_b300.inputs import rhs_normal

    n = args.n
    levels = args.levels or int(round(math.log2(n + 1)))
    mg = kcycle.Multigrid(n, args.eps, args.theta, levels, smoother=args.smoother, coarsening=args.coarsening)
    dt = torch.float32 if args.fp32 else torch.float64
    f = torch.tensor(rhs_normal(n, 0), device="cuda").to(dt)
    v = torch.zeros_like(f)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.cycles if args.solve else 0):
        mg.profile_cycle(v, f, args.kappa, with_norm=True)
    for _ in range(args.cycles if args.mixed else 0):
        mg.profile_cycle(v, f, args.kappa, fp32=True)
    for _ in range(0 if (args.solve or args.mixed) else args.cycles):
        if args.fp32:
            mg.kcycle_f32(v, f, args.kappa)
        else:
            mg.kcycle(v, f, args.kappa)
    torch.cuda.synchronize()
    print(json.dumps({"n": n, "levels": levels, "kappa": args.kappa, "cycles": args.cycles,
                      "smoother": args.smoother, "coarsening": args.coarsening, "fp32": args.fp32,
                      "solve": args.solve, "mixed": args.mixed,
                      "wall_ms": 1e3 * (time.perf_counter() - t0)}))


if __name__ == "__main__":
    main()
