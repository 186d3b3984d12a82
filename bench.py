"""Benchmark: milliseconds to a 1e-8 relative residual for the kappa-cycle stand-alone solver.

Workload (synthetic, shaped like the paper's Section 4 tests): 4095^2 interior grid, 12 levels,
theta = pi/3, eps = 1e-4, f ~ N(0,1) (seed = rank), v0 = 0, nu1 = nu2 = 2, omega = 0.8, Galerkin
coarse operators, FP64 throughout. One step = one solve to 1e-8 with the step's kappa (default
4) through the C ABI (one CUDA-graph launch with an on-device stopping test).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--kappa K] [--impl reference]

Prints one JSON line. Under torchrun (N > 1) each rank solves its own problem (replicas); the
step time is the maximum over ranks and rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2010_00626_b300.inputs import KAPPA_W, LARGE, rhs_normal  # noqa: E402

METRIC = "ms to 1e-8 rel. residual per kappa (FP64 vs mixed/batched) and % of HBM peak"
WORKLOAD = "large standalone 4095^2 (12 levels, theta=pi/3, eps=1e-4, FP64)"
NOMINAL_FP64_TFLOPS = 1.25  # nominal B300 FP64 rate
# Measured DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum, one ncu capture) of one level-0
# pass A launch of a solve cycle at 4095^2, keyed by the SHA-256 of the kernel source it was taken
# on (kernels.cuh from its start to the pass B section: the shared helpers and pass A): when that
# text changes the figure no longer describes the kernel and is reported as null until a new
# capture replaces it.
PASS_A_L0_TRAFFIC = {"source": "paper_2010_00626_b300/csrc/kernels.cuh", "until": "// Pass B: v <- v + P v_c",
                     "sha256": "4bc1574b89893c8218c12cfb6e265967970d9dfc870582efd8c56923a292db58",
                     "bytes": 268_414_976 + 133_147_136}


# The same for the FP32 tensor-copy passes at level 0 of the mixed solve's FP32 cycle (4095^2), keyed
# by the whole of tma_f32.cuh.
TMA_L0_TRAFFIC = {
    "pass_a": {"source": "paper_2010_00626_b300/csrc/tma_f32.cuh", "sha256": "aedf126f506700bace586c5478c5e794744bdcbc7feb452e929347050a973443",
               "bytes": 67_187_200 + 33_016_064},
    "pass_b": {"source": "paper_2010_00626_b300/csrc/tma_f32.cuh", "sha256": "aedf126f506700bace586c5478c5e794744bdcbc7feb452e929347050a973443",
               "bytes": 151_072_512 + 37_347_072},
}


def source_digest(entry):
    """SHA-256 of the kernel source text an entry's figure was measured on."""
    import hashlib
    try:
        with open(os.path.join(ROOT, entry["source"])) as fh:
            text = fh.read()
    except OSError:
        return None
    end = text.find(entry["until"]) if entry.get("until") else -1
    return hashlib.sha256((text[:end] if end >= 0 else text).encode()).hexdigest()


def measured_traffic(entry):
    """The stored DRAM bytes of `entry` if its kernel source is unchanged since the capture, else None."""
    if not entry.get("sha256"):
        return None
    return entry["bytes"] if source_digest(entry) == entry["sha256"] else None


def host_cpu():
    """CPU model and logical core count of the host the oracle runs on."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"cpu_model": model, "nproc": os.cpu_count()}


def bench_config(kappa, world=1):
    """The workload description both arms print (the same keys and values)."""
    cfg = LARGE
    out = {"workload": WORKLOAD, "n": cfg["n"], "levels": cfg["levels"], "theta": cfg["theta"], "eps": cfg["eps"],
           "kappa": kname(kappa), "tol": 1e-8, "nu1": cfg["nu1"], "nu2": cfg["nu2"], "omega": cfg["omega"],
           "l2": "inputs larger than L2 (each 4095^2 FP64 array is 134 MB)"}
    if world > 1:
        out["parallelism"] = f"replicas x{world}"
    return out


def kname(k):
    return "W" if k >= 1000 else str(k)


# ------------------------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------ oracle CPU arm
def oracle_cycles_to_tol(kappa):
    """Cycles the oracle needs to reach 1e-8 on this workload, from the golden file written by
    oracle/full_size_cycles.py (calls only the oracle); None when not recorded."""
    path = os.path.join(ROOT, "tests", "golden", f"large_standalone_cycles_k{kappa}.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh)["cycles"]
    return None


def time_oracle_cycles(kappa, ncycles):
    """Wall ms per oracle cycle on the host cores, timed over `ncycles` cycles from v0 = 0."""
    import oracle
    cfg = LARGE
    h = oracle.Hierarchy(cfg["n"], cfg["levels"], cfg["theta"], cfg["eps"])
    f = rhs_normal(cfg["n"], 0)
    v = np.zeros_like(f)
    t0 = time.perf_counter()
    for _ in range(ncycles):
        v = oracle.cycle(h, v, f, kappa)
    return 1e3 * (time.perf_counter() - t0) / ncycles


def _oracle_replica(kappa, seed, barrier, out):
    """One oracle cycle on its own 4095^2 problem, started together with the other replicas."""
    import oracle
    cfg = LARGE
    h = oracle.Hierarchy(cfg["n"], cfg["levels"], cfg["theta"], cfg["eps"])
    f = rhs_normal(cfg["n"], seed)
    v = np.zeros_like(f)
    barrier.wait()
    t0 = time.perf_counter()
    oracle.cycle(h, v, f, kappa)
    out.put(1e3 * (time.perf_counter() - t0))


def oracle_all_cores(kappa, cycles):
    """The oracle on every host core at once. It is single-threaded (numpy stencil operations),
    so one problem cannot use more than one core; the host's cores are used by as many independent
    replicas (one process each, spawned, each on its own f) as there are cores, bounded by memory
    (about 2 GB per replica at 4095^2). Each replica times one kappa-cycle; reported: the median
    per-replica ms to 1e-8 (ms per cycle x cycles) and the host's throughput in problems per hour."""
    import multiprocessing as mp
    nproc = os.cpu_count() or 1
    try:
        import psutil
        mem_cap = max(1, int(psutil.virtual_memory().available / 2e9))
    except Exception:
        mem_cap = nproc
    procs_n = max(1, min(nproc, mem_cap))
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(procs_n), ctx.SimpleQueue()
    procs = [ctx.Process(target=_oracle_replica, args=(kappa, 1000 + i, barrier, out)) for i in range(procs_n)]
    for p in procs:
        p.start()
    ms = sorted(out.get() for _ in range(procs_n))
    for p in procs:
        p.join()
    med = ms[len(ms) // 2]
    return {"value": med * cycles, "unit": "ms", "cores": procs_n, "kind": "oracle",
            "sample": (f"{procs_n} concurrent replicas (one process per core, own f each), one kappa={kname(kappa)} "
                       f"oracle cycle each on the 4095^2 problem; value = median ms per cycle "
                       f"({med:.0f}) x {cycles} cycles to 1e-8; slowest replica {ms[-1]:.0f} ms per cycle"),
            "problems_per_hour": procs_n * 3.6e6 / (ms[-1] * cycles)}


def cpu_cores_used():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([1] + [int(i.get("num_threads", 1)) for i in info if i.get("internal_api") != "openmp"])
    except Exception:
        return 1


def run_reference(args, rank, world):
    if rank != 0:
        return
    kappa = args.kappa
    cycles = oracle_cycles_to_tol(kappa)
    samples = []
    for _ in range(args.warmup):
        time_oracle_cycles(kappa, 1)
    for _ in range(args.steps):
        samples.append(time_oracle_cycles(kappa, 1))
    ms_cycle = statistics.mean(samples)
    value = ms_cycle * cycles if cycles else None
    sample = (f"each step one kappa={kname(kappa)} oracle cycle on the 4095^2 problem from v0=0; value = mean ms per "
              f"cycle x {cycles} cycles, the oracle's own count to 1e-8 (tests/golden)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_cycle, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(kappa, world), "cycles": cycles, "ms_per_cycle": ms_cycle,
            "cpu_baseline": {"value": value, "unit": "ms", "cores": cpu_cores_used(), "kind": "oracle",
                             "sample": sample, **host_cpu()},
            "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks_of(x, world, device):
    """The largest x over the ranks of the default process group (NCCL with device "cuda", gloo with
    "cpu"): a replicated run reports its slowest rank's step time."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------------ GPU arm
def dp_ops_per_point(kind, nu, norm):
    """FP64 operations per fine point the method needs in one launch (no halo recomputation):
    Jacobi 10 (4 adds, 1 mul, 5 fma, or the residual form: 9 for f - A v and 1 fma), residual 9,
    full weighting 9 per coarse point (2.25 per fine), bilinear interpolation + correction 3 on
    average, one fma per squared residual of a norm; flops count an fma as 2."""
    jac_ops, jac_flops = 10, 15
    res_ops, res_flops = 9, 14
    fw_ops, fw_flops = 9 / 4, 11 / 4
    pr_ops, pr_flops = 3, 3
    if kind == 0:  # with norm: the first sweep's residual squared and summed (one fma)
        return (nu * jac_ops + res_ops + fw_ops + (1 if norm else 0),
                nu * jac_flops + res_flops + fw_flops + (2 if norm else 0))
    ops = pr_ops + nu * jac_ops + (res_ops + 1 if norm else 0)
    flops = pr_flops + nu * jac_flops + (res_flops + 2 if norm else 0)
    return ops, flops


def bytes_per_point(kind, norm):
    """Algorithmic HBM bytes per fine point of one fused pass (each field read or written once)."""
    return 8 + 8 + 8 + 2 if kind == 0 else 8 + 8 + 2 + 8


REF_TOL = 1e-12  # tolerance of the FP64 reference solutions of the error statements


def error_vs_fp64(mg, x, f, x_star):
    """Quality of a mixed-precision result x, stated per result: its relative residual recomputed
    in FP64 on the device (mg_residual_norm, the FP64 kernel whose parity with the oracle the tests
    pin) and its relative error against x_star, the FP64 solve of the same problem to REF_TOL,
    norm-wise and element-wise."""
    import torch
    rr = mg.residual_norm(x, f) / float(torch.linalg.vector_norm(f))
    d = x - x_star
    return {"relres_fp64": rr,
            "rel_error_l2": float(torch.linalg.vector_norm(d) / torch.linalg.vector_norm(x_star)),
            "rel_error_max": float(d.abs().max() / x_star.abs().max())}


# launch kinds of mg_profile_cycle
PROFILE_KINDS = {0: "pass_a", 1: "pass_b", 2: "coarse", 3: "residual", 4: "lines_x", 5: "lines_y",
                 6: "call",  # call: pass A, the coarse walk and pass B of one call in one cluster launch
                 7: "deep"}  # deep: a call with every call below it in one persistent cooperative launch


def per_level_report(mg, prof, fp32, fp64_peak_ops, hbm_peak, norm_l0, sms, kappa, l0_zero):
    """Per level of one profiled cycle (a CUDA event pair around every launch, replayed from a graph
    as a solve runs it): launches,
    microseconds per launch, CTAs per launch (mg_level_grid), algorithmic bytes and FP64 operations
    per launch (each field read or written once; no halo recomputation; a pass A that starts from
    zero reads no v and its first sweep is one operation: the first call below each parent call, and
    level 0 when l0_zero), the achieved HBM GB/s and FP64 op/s with their fractions of the measured
    peaks, and the time during which SMs hold no CTA (a launch of c < 148 CTAs leaves 148 - c SMs
    without work)."""
    ms, kind, level = prof
    esz = 4 if fp32 else 8
    rows, idle_ms, total_ms, coarse_ms, coarse_idle = {}, 0.0, 0.0, 0.0, 0.0
    for t, k, l in zip(ms, kind, level):
        key = (int(l), int(k))
        r = rows.setdefault(key, [0, 0.0])
        r[0] += 1
        r[1] += float(t)
    grids = {}
    out = []
    calls = mg.counters(kappa)[0]
    for (l, k), (cnt, t) in sorted(rows.items()):
        if l not in grids:
            grids[l] = mg.level_grid(l, fp32=fp32)
        n_l, ctas = grids[l]
        busy = min(ctas, sms)
        idle = t * (sms - busy) / sms
        total_ms += t
        idle_ms += idle
        if ctas < sms:
            coarse_ms += t
            coarse_idle += idle
        e = {"level": l, "n": n_l, "kind": PROFILE_KINDS.get(k, str(k)),
             "launches": cnt, "us_per_launch": round(1e3 * t / cnt, 2), "ctas": ctas}
        if k in (0, 1):
            pts = n_l * n_l
            # pass A: v, f read, relaxed v written, coarse f written (a quarter); pass B: relaxed v,
            # f read, coarse v read (a quarter), v written
            nbytes = pts * esz * 3.25
            ops = dp_ops_per_point(k, 2, norm_l0 and k == 0 and l == 0)[0] * pts
            if k == 0:
                # from zero the first sweep is v = w f: one operation instead of ten, and no v read
                zero = ((1 if l0_zero else 0) if l == 0 else calls[l - 1]) / max(calls[l], 1)
                nbytes -= pts * esz * zero
                ops -= 9 * pts * zero
            sec = 1e-3 * t / cnt
            e["gb_s"] = round(nbytes / sec / 1e9, 1)
            e["hbm_frac"] = round(nbytes / sec / 1e9 / hbm_peak, 4)
            if not fp32:
                e["fp64_frac"] = round(ops / sec / fp64_peak_ops, 4)
        out.append(e)
    return {"levels": out,
            "sm_idle": {"ms_per_cycle": round(idle_ms, 4), "frac_of_cycle": round(idle_ms / total_ms, 4),
                        "launches_below_one_wave_ms": round(coarse_ms, 4),
                        "idle_within_those_ms": round(coarse_idle, 4),
                        "note": "launches timed with CUDA event pairs inside a graph replay; an SM idles while a launch has fewer "
                                "CTAs than SMs (the coarse levels and the one-CTA coarse kernel)"}}


PAPER_TABLE6 = {"10": {"2": 589, "3": 274, "4": 206, "W": 193}, "45": {"2": 1725, "3": 706, "4": 463, "W": 385}}
PAPER_TABLE7 = {"10": {"4": 36}, "45": {"4": 53}}
PAPER_TABLE8 = {"10": {"1": 1705, "2": 371, "3": 187, "4": 148}, "45": {"2": 1093, "3": 410, "4": 254}}
PAPER_TABLE9 = {"10": {"2": 45}, "45": {"2": 79}}


def zebra_tables(n, levels, tol, v0_host, f, settings, coarsening="full", mgcg_kappa=4):
    """Zebra line relaxation with Galerkin coarse operators at eps = 1e-5 (Section 4): alternating
    x/y relaxation with full coarsening (solvers 3-4, Tables 6-7), or x-line relaxation with
    semi-coarsening along y (coarsening="y", solvers 5-6, Tables 8-9). Stand-alone cycles from a
    random start with f = 0 until the L2 error (the iterate) is reduced by 1e8 (the tables'
    protocol), and MGCG with the `mgcg_kappa` cycle on f ~ N(0, 1) to `tol` relative residual
    (mg_pcg starts from x0 = 0, so the f = 0 protocol does not apply to it)."""
    import torch
    from paper_2010_00626_b300 import kcycle
    semi = coarsening == "y"
    relax = ("x-line zebra (nu=2+2, both along x), semi-coarsening along y" if semi else
             "alternating zebra x then y (nu=2+2: one relaxation per direction)")
    out = {"setting": (f"{n}^2, {levels} levels, eps=1e-5, {relax}, Galerkin coarse operators; stand-alone: "
                       "f=0, v0~U(-1,1) seed 12345, ||v_k||/||v_0|| <= 1e-8; MGCG: f~N(0,1) seed 0, x0=0, "
                       f"relres <= {tol:g}")}
    if semi:
        out.update({"paper_table8_cycles_16383_rtx3090": PAPER_TABLE8, "paper_table9_iters_16383_rtx3090": PAPER_TABLE9})
    else:
        out.update({"paper_table6_cycles_16383_rtx3090": PAPER_TABLE6, "paper_table7_iters_16383_rtx3090": PAPER_TABLE7})
    v0 = torch.tensor(v0_host, device="cuda")
    zero = torch.zeros_like(v0)
    for deg, kappas in settings:
        mz = kcycle.Multigrid(n, 1e-5, math.radians(deg), levels, 2, 2, smoother="zebra", coarsening=coarsening)
        mz.set_option(kcycle.MG_OPT_STOP, 1)
        row = {}
        for k in kappas:
            vv = v0.clone()
            mz.solve(vv, zero, k, 1e-8, 1, history=False)  # builds the graph
            vv = v0.clone()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            st_z, cyc_z, red_z, _ = mz.solve(vv, zero, k, 1e-8, 20000, history=False)
            b.record()
            torch.cuda.synchronize()
            row[kname(k)] = {"cycles": cyc_z, "ms": round(a.elapsed_time(b), 1),
                             "ms_per_cycle": round(a.elapsed_time(b) / max(cyc_z, 1), 3), "status": st_z}
        mz.set_option(kcycle.MG_OPT_STOP, 0)
        x = torch.zeros_like(v0)
        mz.pcg(x, f, mgcg_kappa, tol, 1, history=False)
        x.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        st_c, it_c, rel_c, _ = mz.pcg(x, f, mgcg_kappa, tol, 2000, history=False)
        b.record()
        torch.cuda.synchronize()
        row[f"mgcg_k{mgcg_kappa}"] = {"iterations": it_c, "ms": round(a.elapsed_time(b), 1), "relres": rel_c,
                                      "status": st_c}
        out[f"{deg}deg"] = row
        mz.close()
    return out


def profile_run(argv):
    """Profiler driver: a fixed number of kappa-cycles on one synthetic problem through the C ABI,
    with no timing of its own (the numbers meant for reports come from CUDA events in the main
    bench; this only gives ncu the launches to capture).

        python bench.py --profile-run --n 4095 --kappa 4 --cycles 1 [--levels L] [--theta T] [--eps E]
            [--smoother jacobi|zebra|xzebra] [--coarsening full|y] [--fp32 | --mixed | --solve]

    f ~ N(0, 1) seed 0, v = 0. --fp32: FP32 cycles (mg_kcycle_f32); --mixed: the FP32 cycle of
    mg_solve_mixed launch by launch on the handle's own FP32 arrays (mg_profile_cycle); --solve:
    the launches of stand-alone solve cycles (with the stopping test's norm) one by one, as
    mg_profile_cycle runs them (a solve's own graph has conditional nodes, whose kernels
    profilers skip). Prints one JSON line with the wall time."""
    ap = argparse.ArgumentParser(prog="bench.py --profile-run")
    ap.add_argument("--n", type=int, default=4095)
    ap.add_argument("--levels", type=int, default=0, help="0: down to 1x1")
    ap.add_argument("--kappa", type=int, default=4)
    ap.add_argument("--cycles", type=int, default=1)
    ap.add_argument("--theta", type=float, default=math.pi / 3)
    ap.add_argument("--eps", type=float, default=1e-4)
    ap.add_argument("--smoother", default="jacobi", choices=["jacobi", "zebra", "xzebra"])
    ap.add_argument("--coarsening", default="full", choices=["full", "y"])
    ap.add_argument("--fp32", action="store_true")
    ap.add_argument("--mixed", action="store_true")
    ap.add_argument("--solve", action="store_true")
    args = ap.parse_args(argv)

    import torch

    from paper_2010_00626_b300 import build
    build.build()
    from paper_2010_00626_b300 import kcycle

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
                      "solve": args.solve, "mixed": args.mixed, "wall_ms": 1e3 * (time.perf_counter() - t0)}))


def main():
    if "--profile-run" in sys.argv[1:]:
        return profile_run([a for a in sys.argv[1:] if a != "--profile-run"])
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--kappa", type=int, default=4)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-sweep", action="store_true", help="skip the per-kappa sweep")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--paper-scale", action="store_true",
                    help="also run the zebra Table 6/7 setting at the paper's 16383^2 (about a minute)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return max_over_ranks_of(x, world, "cuda")

    from paper_2010_00626_b300 import build
    build.build()
    from paper_2010_00626_b300 import kcycle

    cfg = LARGE
    n, levels, tol, kappa = cfg["n"], cfg["levels"], 1e-8, args.kappa
    mg = kcycle.Multigrid(n, cfg["eps"], cfg["theta"], levels, cfg["nu1"], cfg["nu2"])
    f_host = rhs_normal(n, rank)
    f = torch.tensor(f_host, device="cuda")
    v = torch.zeros_like(f)
    max_cycles = 20000

    def step():
        v.zero_()
        return mg.solve(v, f, kappa, tol, max_cycles, history=False)

    for _ in range(args.warmup):
        st, cycles, rel, _ = step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        barrier()
        e0.record()
        for _ in range(args.steps):
            st, cycles, rel, _ = step()
        e1.record()
        barrier()
    ms_step = max_over_ranks(e0.elapsed_time(e1) / args.steps)
    assert st == 0 and rel <= tol, (st, rel)
    launches_cycle = mg.counters(kappa)[1]
    gpu_launches = args.steps * (2 + 1 + cycles * (launches_cycle + 1))

    # ---------------------------------------------------------------- per-launch profile
    prof_ms, prof_kind, prof_level = None, None, None
    for _ in range(3):
        prof_ms, prof_kind, prof_level = mg.profile_cycle(v, f, kappa, with_norm=True, graph=True)
    share = {}
    for t, k, l in zip(prof_ms, prof_kind, prof_level):
        key = (int(k), int(l))
        share[key] = share.get(key, 0.0) + float(t)
    total = sum(share.values())
    top = max(share, key=share.get)
    kinds = PROFILE_KINDS
    # the finest-level pass A: the dominant fused kernel of the FP64 path
    dom = (0, 0)
    dom_ms = [float(t) for t, k, l in zip(prof_ms, prof_kind, prof_level) if (k, l) == dom]
    dom_avg = sum(dom_ms) / len(dom_ms)
    # the solve's level-0 pass A also forms the stopping test's residual norm in its first sweep
    ops, flops = dp_ops_per_point(0, cfg["nu1"], True)
    pts = n * n
    achieved_tflops = flops * pts / (dom_avg * 1e-3) / 1e12
    # the FP64 pipe issues add, mul and fma at one rate: the ALU roofline counts FP64 operations
    # against this device's measured FP64 operation rate (DFMA throughput probe, run live)
    fp64_peak_ops = kcycle.fp64_rate()
    achieved_ops = ops * pts / (dom_avg * 1e-3)
    bytes_alg = bytes_per_point(0, False) * pts
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    hbm_achieved = bytes_alg / (dom_avg * 1e-3) / 1e9
    roofline = {"bound": "alu", "kernel": "pass_a level 0 (4095^2, FP64; two sweeps, residual, full weighting, "
                                          "and the stopping test's residual norm)",
                "achieved": achieved_ops / 1e12,
                "peak": fp64_peak_ops / 1e12, "unit": "T FP64 op/s", "frac": achieved_ops / fp64_peak_ops,
                "peak_source": "measured live: FP64 FMA throughput probe (mg_fp64_rate); add/mul/fma count as one",
                "algorithmic_ops_per_point": ops, "ms_per_launch": dom_avg,
                "tflops_fma2": achieved_tflops, "frac_of_nominal_1.25_tflops": achieved_tflops / NOMINAL_FP64_TFLOPS,
                "traffic": measured_traffic(PASS_A_L0_TRAFFIC) if n == 4095 else None,
                "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch, taken on the "
                                   "kernel source with the recorded SHA-256 (null once that source changed)"),
                "hbm": {"achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_achieved / hbm_peak,
                        "algorithmic_bytes": bytes_alg}}
    cycle_share = {f"{kinds[k]}@L{l}": round(t / total, 4) for (k, l), t in sorted(share.items(), key=lambda x: -x[1])[:8]}
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    per_level = per_level_report(mg, (prof_ms, prof_kind, prof_level), False, fp64_peak_ops, hbm_peak, True, sms,
                                 kappa, False)
    per_level["cycle"] = f"FP64 kappa={kname(kappa)} stand-alone solve cycle"
    per_level["fine_dof_per_s"] = n * n / (ms_step / cycles * 1e-3)

    # ---------------------------------------------------------------- end to end (host buffers)
    e2e = None
    if rank == 0 or world > 1:
        fh_pin = torch.tensor(f_host).pin_memory()
        vh_pin = torch.zeros_like(fh_pin).pin_memory()
        vh_np, fh_np = vh_pin.numpy(), fh_pin.numpy()
        mg.solve_host(vh_np, fh_np, kappa, tol, max_cycles)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            vh_np[:] = 0.0
            st2, c2, r2 = mg.solve_host(vh_np, fh_np, kappa, tol, max_cycles)
        e2e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0) / args.steps)
        e2e = {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 2 * 8 * n * n, "d2h_bytes_per_step": 8 * n * n}

    # ---------------------------------------------------------------- per-kappa sweep
    per_kappa = {}
    if not args.no_sweep:
        for k in (1, 2, 3, 4, 5, KAPPA_W):
            v.zero_()
            mg.solve(v, f, k, tol, 1, history=False)  # builds the graph
            v.zero_()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            st_k, cyc_k, rel_k, _ = mg.solve(v, f, k, tol, max_cycles, history=False)
            b.record()
            torch.cuda.synchronize()
            ms_k = a.elapsed_time(b)
            per_kappa[kname(k)] = {"ms": round(ms_k, 3), "cycles": cyc_k, "ms_per_cycle": round(ms_k / cyc_k, 4),
                                   "relres": rel_k, "status": st_k}

    # ---------------------------------------------------------------- mixed precision (FP32 cycles + FP64 IR)
    per_kappa_mixed = {}
    if not args.no_sweep:
        # the reference solution for the error statements: the FP64 solve to 1e-12 (its residual
        # levels off near 6e-13 at this size, so a tighter tolerance is not reachable)
        x_star = torch.zeros_like(f)
        st_s, cyc_s, rel_s, _ = mg.solve(x_star, f, kappa, REF_TOL, 3000, history=False)
        per_kappa_mixed["reference_solution"] = {"what": f"FP64 kappa={kname(kappa)} solve", "tol": REF_TOL,
                                                 "cycles": cyc_s, "relres": rel_s, "status": st_s}
        for k in (1, 2, 3, 4, 5, KAPPA_W):
            v.zero_()
            mg.solve_mixed(v, f, k, tol, 1, history=False)  # builds the graph and the FP32 levels
            v.zero_()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            st_k, it_k, rel_k, _ = mg.solve_mixed(v, f, k, tol, max_cycles, history=False)
            b.record()
            torch.cuda.synchronize()
            ms_k = a.elapsed_time(b)
            per_kappa_mixed[kname(k)] = {"ms": round(ms_k, 3), "iterations": it_k,
                                         "ms_per_iteration": round(ms_k / it_k, 4), "relres": rel_k, "status": st_k,
                                         "error_vs_fp64": error_vs_fp64(mg, v, f, x_star)}
        # the same statement for the FP64 solve to the same tolerance: a relative residual of tol
        # bounds the error only through cond(A), for either form
        v.zero_()
        mg.solve(v, f, kappa, tol, max_cycles, history=False)
        per_kappa_mixed["fp64_solve_same_tol"] = {"kappa": kname(kappa), "tol": tol,
                                                  "error_vs_fp64": error_vs_fp64(mg, v, f, x_star)}
        del x_star

    # ---------------------------------------------------------------- run-time model (Section 3) and kappa pre-selection
    model_report = None
    if not args.no_sweep and world == 1:
        from paper_2010_00626_b300 import fit_model, model
        samples = fit_model.measure(max_levels=12, reps=2)
        fitted = fit_model.fit(samples)
        bf = fitted["b300_form"]
        params = (bf["alpha_fine_launch_ms"], bf["alpha_coarse_call_ms"], bf["beta_ms"])
        lc = next(l for l in range(levels) if (n + 1) // (2 ** l) - 1 <= mg.get_option(kcycle.MG_OPT_COARSE_N))
        pred_cycle, rho = {}, {}
        for k in (1, 2, 3, 4, 5, KAPPA_W):
            kk = model.W_COUNTER if k == KAPPA_W else k
            pred_cycle[kname(k)] = model.predict_b300(params, kk, levels, lc, n)
            # asymptotic contraction: the first cycles remove the oscillatory error quickly, so the
            # rate is taken over cycles 40..80, when the slowest modes dominate
            v.zero_()
            _, _, _, hist80 = mg.solve(v, f, k, 1e-300, 80)
            rho[kname(k)] = model.contraction(hist80, skip=40)
        best_pred, table = model.preselect_kappa(pred_cycle, rho, tol)
        measured = {k: d["ms"] for k, d in per_kappa.items()}
        model_report = {"fit": {"paper_alpha_ms": fitted["paper_form"]["alpha_ms"],
                                "paper_beta_ms": fitted["paper_form"]["beta_ms"],
                                "turning_point_levels": fitted["paper_form"]["turning_point_levels"],
                                "alpha_fine_launch_ms": params[0], "alpha_coarse_call_ms": params[1],
                                "beta_ms": params[2]},
                        "predicted_ms_per_cycle": {k: round(t, 4) for k, t in pred_cycle.items()},
                        "rho_cycles_40_80": {k: round(r, 5) for k, r in rho.items()},
                        "predicted_ms_to_tol": {k: round(t, 1) for k, t in table.items()},
                        "predicted_best_kappa": best_pred,
                        "measured_best_kappa": min(measured, key=measured.get) if measured else None}

    # ---------------------------------------------------------------- the paper's own protocol (Table 4 setting)
    paper_protocol = None
    if not args.no_sweep and world == 1:
        # 12 levels, phi = 45 deg, eps = 1e-4, damped Jacobi nu = 2+2, coarse operators rediscretized,
        # f = 0 and a random start, until the L2 error (the iterate) is reduced by 1e8 (Section 4)
        mp = kcycle.Multigrid(n, 1e-4, math.pi / 4, levels, 2, 2, omega=0.87)
        mp.set_option(kcycle.MG_OPT_COARSE_OP, 1)
        mp.set_option(kcycle.MG_OPT_STOP, 1)
        zero = torch.zeros_like(f)
        v0 = torch.tensor(np.random.default_rng(12345).uniform(-1.0, 1.0, (n, n)), device="cuda")
        paper_cycles = {"1": 6909, "2": 1403, "3": 651, "4": 495, "W": 470}
        paper_protocol = {"setting": "4095^2, 12 levels, phi=pi/4, eps=1e-4, omega=0.87, nu=2+2, rediscretized "
                                     "coarse operators, f=0, v0~U(-1,1) seed 12345, ||v_k||/||v_0|| <= 1e-8",
                          "paper_table4_cycles_gtx1060": paper_cycles}
        for k in (1, 2, 3, 4, KAPPA_W):
            vv = v0.clone()
            mp.solve(vv, zero, k, 1e-8, 1, history=False)
            vv = v0.clone()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            st_p, cyc_p, red_p, _ = mp.solve(vv, zero, k, 1e-8, 20000, history=False)
            b.record()
            torch.cuda.synchronize()
            paper_protocol[kname(k)] = {"cycles": cyc_p, "ms": round(a.elapsed_time(b), 1),
                                        "ms_per_cycle": round(a.elapsed_time(b) / max(cyc_p, 1), 3)}
        mp.close()

    # ---------------------------------------------------------------- zebra line relaxation (Tables 6-7 setting)
    zebra = semi = None
    if not args.no_sweep and world == 1:
        zebra = zebra_tables(n, levels, tol, np.random.default_rng(12345).uniform(-1.0, 1.0, (n, n)),
                             f, ((10, (2, 3, 4, KAPPA_W)), (45, (3, 4))))
        semi = zebra_tables(n, levels, tol, np.random.default_rng(12345).uniform(-1.0, 1.0, (n, n)),
                            f, ((10, (2, 3)), (45, (2, 3))), coarsening="y", mgcg_kappa=2)
    paper_scale = None
    if args.paper_scale and world == 1:
        # the paper's own size: 14 levels, 16383^2 (268M unknowns), 45 degrees
        n14 = 16383
        f14 = torch.tensor(rhs_normal(n14, 0), device="cuda")
        paper_scale = zebra_tables(n14, 14, tol, np.random.default_rng(12345).uniform(-1.0, 1.0, (n14, n14)),
                                   f14, ((45, (4,)),))
        del f14

    # ---------------------------------------------------------------- convection-diffusion (Section 5's proposal)
    convection = None
    if not args.no_sweep and world == 1:
        bc = (1000.0, 500.0)
        mc = kcycle.Multigrid(n, 1e-2, math.pi / 6, levels, convection=bc, coarse_op="rediscretized")
        vc_ = torch.zeros_like(f)
        convection = {"workload": f"{n}^2, {levels} levels, theta=pi/6, eps=1e-2, b=({bc[0]:g}, {bc[1]:g}) upwind, "
                                  "damped Jacobi, rediscretized upwind coarse operators, f~N(0,1), tol 1e-8"}
        for k in (1, 2, 3, 4, KAPPA_W):
            vc_.zero_()
            mc.solve(vc_, f, k, tol, 1, history=False)
            vc_.zero_()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            st_c, cyc_c, rel_c, _ = mc.solve(vc_, f, k, tol, 5000, history=False)
            b.record()
            torch.cuda.synchronize()
            convection[kname(k)] = {"cycles": cyc_c, "ms": round(a.elapsed_time(b), 1), "status": st_c}
        mc.close()

    # ---------------------------------------------------------------- MGCG 8191^2 (the preconditioner workload)
    mgcg = None
    if not args.no_sweep and world == 1:
        from paper_2010_00626_b300.inputs import PCG_LARGE, pcg_theta
        n8, lev8, eps8 = PCG_LARGE["n"], PCG_LARGE["levels"], 1e-5
        th8 = pcg_theta(0)
        m8 = kcycle.Multigrid(n8, eps8, th8, lev8)
        b8 = torch.tensor(rhs_normal(n8, 0), device="cuda")
        x8 = torch.zeros_like(b8)
        mgcg = {"workload": f"{n8}^2, {lev8} levels, theta={th8:.6f} (seed 0), eps={eps8:g}, b~N(0,1), x0=0, "
                            "tol 1e-10; kappa>1 cycles are not symmetric: flexible beta, or the symmetrised "
                            "preconditioner B+B^T-B^TAB with plain CG"}
        runs = [("fp64", 1, 0, False), ("fp64", 2, 0, True), ("fp64", 3, 0, True), ("fp64", 4, 0, True),
                ("fp64_symmetrised", 2, 1, False), ("fp64_symmetrised", 3, 1, False), ("mixed", 3, 0, True)]
        x8_star = torch.zeros_like(b8)
        st8s, it8s, rel8s, _ = m8.pcg(x8_star, b8, 3, REF_TOL, 2000, flexible=True, history=False)
        mgcg["reference_solution"] = {"what": "FP64 MGCG kappa=3, flexible beta", "tol": REF_TOL, "iterations": it8s,
                                      "relres": rel8s, "status": st8s}
        for name, k8, sym, flex in runs:
            m8.set_option(kcycle.MG_OPT_PRECOND, sym)
            mixed = name == "mixed"
            m8.pcg(x8, b8, k8, 1e-10, 1, flexible=flex, mixed=mixed, history=False)  # builds the graph
            x8.zero_()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            st8, it8, rel8, _ = m8.pcg(x8, b8, k8, 1e-10, 2000, flexible=flex, mixed=mixed, history=False)
            b.record()
            torch.cuda.synchronize()
            mgcg[f"{name}_k{k8}"] = {"ms": round(a.elapsed_time(b), 1), "iterations": it8, "relres": rel8,
                                     "status": st8, "flexible": flex}
            if mixed:
                mgcg[f"{name}_k{k8}"]["error_vs_fp64"] = error_vs_fp64(m8, x8, b8, x8_star)
        m8.close()
        del b8, x8, x8_star

    # ---------------------------------------------------------------- batched (256 ragged instances, one launch each)
    batched = None
    if not args.no_sweep and world == 1:
        from paper_2010_00626_b300.inputs import batched_instances, rhs_uniform
        inst = batched_instances(count=256, seed=0)
        ns = [d["n"] for d in inst]
        fs_b = [torch.tensor(rhs_uniform(d["n"], d["seed"]), device="cuda") for d in inst]
        xs_b = [torch.zeros_like(fb) for fb in fs_b]
        batched = {"workload": "256 instances, n uniform over {127,255,511,1023}, theta~U[0,pi), "
                               "log10 eps~U[-5,-1], f~U(-1,1), kappa=3, tol 1e-8, cap 3000 iterations",
                   "dof": int(sum(n * n for n in ns))}
        for mixed, smoother in ((True, "jacobi"), (False, "jacobi"), (True, "zebra"), (False, "zebra")):
            bt = kcycle.Batch(ns, [d["eps"] for d in inst], [d["theta"] for d in inst], smoother=smoother)
            chosen = bt.autotune(3, mixed=mixed)
            for xb in xs_b:
                xb.zero_()
            # builds the graph the timed solve runs (its key holds the tolerance and the cap, so
            # the warm-up is the same solve)
            bt.solve(xs_b, fs_b, 3, tol, 3000, mixed=mixed)
            for xb in xs_b:
                xb.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st_b, it_b, rel_b = bt.solve(xs_b, fs_b, 3, tol, 3000, mixed=mixed)
            ms_b = 1e3 * (time.perf_counter() - t0)
            conv = [i for i in range(len(ns)) if rel_b[i] <= tol]
            q = sorted(it_b)
            entry = {"ms_one_launch": round(ms_b, 1), "converged": len(conv), "of": len(ns),
                     "iterations_quartiles": [q[0], q[len(q) // 4], q[len(q) // 2], q[3 * len(q) // 4], q[-1]],
                     "autotuned_coarse_n": {str(k): v for k, v in chosen.items()},
                     "autotuned_shapes": {str(k): v for k, v in bt.shapes().items()}}
            if mixed:
                # the same problems solved one after another: each instance alone through its own
                # handle (the batch's, with the same tuned options), one graph launch per solve
                solo = [bt.instance(i) for i in range(len(ns))]
                ys = [torch.zeros_like(xb) for xb in xs_b]
                for i, m in enumerate(solo):  # builds its graph and a history for the cap; stops at once
                    m.solve_mixed(ys[i], fs_b[i], 3, 1.0, 3000, history=False)
                for y in ys:
                    y.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for i, m in enumerate(solo):
                    m.solve_mixed(ys[i], fs_b[i], 3, tol, 3000, history=False)
                torch.cuda.synchronize()
                seq_ms = 1e3 * (time.perf_counter() - t0)
                entry["sequential_ms"] = round(seq_ms, 1)
                entry["batch_speedup_vs_sequential"] = round(seq_ms / ms_b, 3)
                for m in solo:
                    m.close()
                del ys
            if mixed:
                # error against each sampled instance's FP64 solve to REF_TOL (a standalone handle)
                errs = []
                for i in range(0, len(ns), 16):
                    if not rel_b[i] <= tol:
                        continue  # a stalled instance (see the note) has no FP64 reference either
                    d = inst[i]
                    ms_ = kcycle.Multigrid(d["n"], d["eps"], d["theta"], int(round(math.log2(d["n"] + 1))),
                                           smoother=smoother)
                    xs_star = torch.zeros_like(fs_b[i])
                    st_s = ms_.solve(xs_star, fs_b[i], 3, REF_TOL, 3000, history=False)[0]
                    e = error_vs_fp64(ms_, xs_b[i], fs_b[i], xs_star)
                    errs.append({"instance": i, "n": d["n"], "reference_status": st_s, **e})
                    ms_.close()
                entry["error_vs_fp64_sample"] = errs
            batched[("mixed" if mixed else "fp64") + ("_zebra" if smoother == "zebra" else "")] = entry
            bt.close()
        batched["note"] = ("damped-Jacobi instances that miss tol are near-grid-aligned with small eps, where "
                           "point relaxation does not smooth; the *_zebra runs use alternating zebra line "
                           "relaxation (Section 4) on every instance")

    # ---------------------------------------------------------------- FP32 cycle of the mixed solve, per level
    per_level32 = roofline_fp32 = None
    if not args.no_sweep:
        for _ in range(3):
            prof32 = mg.profile_cycle(v, f, kappa, fp32=True, graph=True)
        per_level32 = per_level_report(mg, prof32, True, fp64_peak_ops, hbm_peak, False, sms, kappa, True)
        per_level32["cycle"] = f"FP32 kappa={kname(kappa)} cycle of the mixed solve (from zero)"
        # the bandwidth roofline of the FP32 fused passes at level 0 (tensor-copy kernels)
        roofline_fp32 = {}
        for e in per_level32["levels"]:
            if e["level"] == 0 and e["kind"] in ("pass_a", "pass_b"):
                roofline_fp32[e["kind"]] = {
                    "bound": "hbm", "achieved": e["gb_s"], "peak": hbm_peak, "unit": "GB/s", "frac": e["hbm_frac"],
                    "us_per_launch": e["us_per_launch"],
                    "traffic": measured_traffic(TMA_L0_TRAFFIC[e["kind"]]) if n == 4095 else None,
                    "note": "algorithmic bytes (pass A from zero: f read, v and coarse f written, 9 B per point; "
                            "pass B: v, f, coarse v read, v written, 13 B per point) over the launch's CUDA-event "
                            "time in the FP32 cycle, replayed from a graph as the solve runs it"}

    # ---------------------------------------------------------------- oracle on the host cores
    cpu = None
    if rank == 0 and not args.no_cpu:
        ms_cycle_cpu = time_oracle_cycles(kappa, 2)
        cyc_or = oracle_cycles_to_tol(kappa)
        cyc_used = cyc_or if cyc_or else cycles
        cpu = {"value": ms_cycle_cpu * cyc_used, "unit": "ms", "cores": cpu_cores_used(), "kind": "oracle",
               "sample": (f"2 kappa={kname(kappa)} oracle cycles on the 4095^2 problem from v0=0 "
                          f"({ms_cycle_cpu:.0f} ms/cycle) x {cyc_used} cycles to 1e-8 "
                          f"({'oracle count, tests/golden' if cyc_or else 'GPU count'})"), **host_cpu()}
        cpu["all_cores"] = oracle_all_cores(kappa, cyc_used)

    if rank == 0:
        line = {"metric": METRIC, "value": ms_step, "unit": "ms", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": bench_config(kappa, world), "cycles": cycles, "ms_per_cycle": ms_step / cycles,
                "roofline": roofline, "roofline_fp32_passes": roofline_fp32, "cycle_share": cycle_share,
                "per_level": per_level,
                "per_level_fp32": per_level32, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": gpu_launches, "clocks": clocks.summary(), "per_kappa": per_kappa,
                "per_kappa_mixed": per_kappa_mixed, "batched": batched, "model": model_report,
                "paper_protocol": paper_protocol, "zebra": zebra, "semi_coarsening": semi, "mgcg_8191": mgcg,
                "convection_diffusion": convection}
        if paper_scale is not None:
            line["zebra_16383"] = paper_scale
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
