"""Persistent deep calls (MG_OPT_DEEP_CALLS): a call at the largest level of side <= the option's
value runs, with every call below it, as one cooperative launch whose CTAs walk Algorithm 3's
recursion in lock step, separated by grid barriers. The tiles and the per-point arithmetic are
those of the separate launches and the condensed child calls sum each row in the same order, so
cycles, solves and MGCG must equal the launch-by-launch forms bit for bit (which the other GPU
tests hold to the oracle), and the graph must hold the launches mg_counters counts."""
import math

import numpy as np
import pytest

import oracle
from parity import rel
from paper_2010_00626_b300.inputs import KAPPA_W, rhs_normal, rhs_uniform

pytestmark = pytest.mark.gpu


def dev(a, dtype="float64"):
    import torch
    return torch.tensor(a, dtype=getattr(torch, dtype), device="cuda")


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()


@pytest.mark.parametrize("n,levels,kappa,deep", [(255, 8, 2, 255), (255, 8, KAPPA_W, 127), (1023, 10, 1, 511),
                                                 (1023, 10, 3, 255), (1023, 10, 4, 63), (4095, 12, 4, 255),
                                                 (4095, 12, 5, 511)])
def test_fp64_deep_cycles_equal_separate_launches(lib, n, levels, kappa, deep):
    import torch
    on = lib.Multigrid(n, 2e-4, 1.9, levels)
    off = lib.Multigrid(n, 2e-4, 1.9, levels)
    assert on.get_option(lib.MG_OPT_DEEP_CALLS) == 127  # the default
    on.set_option(lib.MG_OPT_DEEP_CALLS, deep)
    off.set_option(lib.MG_OPT_DEEP_CALLS, 0)
    assert on.get_option(lib.MG_OPT_DEEP_CALLS) == deep and off.get_option(lib.MG_OPT_DEEP_CALLS) == 0
    f = dev(rhs_uniform(n, 21))
    a, b = torch.zeros_like(f), torch.zeros_like(f)
    for _ in range(3):
        on.kcycle(a, f, kappa)
        off.kcycle(b, f, kappa)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
    calls, launches, _ = on.counters(kappa)
    assert on.get_option(lib.MG_OPT_LAUNCHES) == launches
    assert launches < off.counters(kappa)[1]  # the deep path was taken
    # the deep launches cover every level from the first of side <= deep down to the coarse kernel's
    top = max(1, next(l for l in range(levels) if (n + 1) // 2 ** l - 1 <= deep))  # never level 0
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    grid = on.level_grid(top)[1]
    assert grid in (sms, 2 * sms) and on.level_grid(top - 1)[1] != grid


def test_fp64_deep_cycle_matches_oracle(lib):
    n, levels, kappa = 511, 9, 3
    theta, eps = math.pi / 3, 1e-4
    h = oracle.Hierarchy(n, levels, theta, eps)
    f = rhs_normal(n, 4)
    mg = lib.Multigrid(n, eps, theta, levels)
    mg.set_option(lib.MG_OPT_DEEP_CALLS, 255)
    vd, fd = dev(np.zeros((n, n))), dev(f)
    v = np.zeros((n, n))
    for _ in range(3):
        mg.kcycle(vd, fd, kappa)
        v = oracle.cycle(h, v, f, kappa)
        assert rel(host(vd), v) <= 1e-12


def test_fp64_deep_solve_and_pcg_equal_separate_launches(lib):
    import torch
    n, levels = 1023, 10
    f = dev(rhs_normal(n, 0))
    outs = []
    for deep in (255, 0):
        mg = lib.Multigrid(n, 1e-4, math.pi / 3, levels)
        mg.set_option(lib.MG_OPT_DEEP_CALLS, deep)
        v = torch.zeros_like(f)
        st = mg.solve(v, f, 4, 1e-8, 2000)
        x = torch.zeros_like(f)
        pc = mg.pcg(x, f, 3, 1e-10, 500, flexible=True)
        torch.cuda.synchronize()
        outs.append((st, pc, v.clone(), x.clone()))
        mg.close()
    (s1, p1, v1, x1), (s2, p2, v2, x2) = outs
    assert s1[0] == 0 and s1 == s2 and p1 == p2
    assert torch.equal(v1, v2) and torch.equal(x1, x2)


def test_fp32_deep_cycles_and_mixed_solve(lib):
    """FP32 cycles: from 127^2 down the separate launches use the same tile passes, so the deep form
    is equal bit for bit; from 255^2 the deep launch replaces the tensor-copy passes of that level
    (another FP32 rounding order), so the mixed solve must still reach its tolerance in the same
    number of iterations."""
    import torch
    n, levels = 1023, 10
    f32 = dev(rhs_uniform(n, 5), "float32")
    outs = {}
    for deep in (127, 0):
        mg = lib.Multigrid(n, 1e-3, 0.7, levels)
        mg.set_option(lib.MG_OPT_DEEP_CALLS, deep)
        v = torch.zeros_like(f32)
        for _ in range(3):
            mg.kcycle_f32(v, f32, 3)
        torch.cuda.synchronize()
        outs[deep] = v.clone()
        mg.close()
    assert torch.equal(outs[127], outs[0])
    f = dev(rhs_normal(n, 6))
    res = {}
    for deep in (255, 0):
        mg = lib.Multigrid(n, 1e-4, math.pi / 3, levels)
        mg.set_option(lib.MG_OPT_DEEP_CALLS, deep)
        x = torch.zeros_like(f)
        res[deep] = mg.solve_mixed(x, f, 4, 1e-8, 500)
        mg.close()
    assert res[255][0] == 0 and res[255][2] <= 1e-8 and res[255][1] == res[0][1]


def test_deep_calls_fall_back_where_they_do_not_apply(lib):
    """Adjoint cycles, zebra smoothing and the general (convection) stencil run the separate
    launches with the option set (bit for bit the same results); bad values are refused."""
    import torch
    n, levels = 255, 8
    for kw in (dict(), dict(smoother="zebra"), dict(convection=(200.0, 50.0), coarse_op="rediscretized")):
        on = lib.Multigrid(n, 1e-2, 0.6, levels, **kw)
        off = lib.Multigrid(n, 1e-2, 0.6, levels, **kw)
        on.set_option(lib.MG_OPT_DEEP_CALLS, 255)
        off.set_option(lib.MG_OPT_DEEP_CALLS, 0)
        f = dev(rhs_uniform(n, 8))
        a, b = torch.zeros_like(f), torch.zeros_like(f)
        if not kw:
            on.kcycle_adjoint(a, f, 3)
            off.kcycle_adjoint(b, f, 3)
        else:
            on.kcycle(a, f, 3)
            off.kcycle(b, f, 3)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        if kw:
            assert on.counters(3)[1] == off.counters(3)[1]
    for bad in (1, 100, 1023, -1):
        with pytest.raises(lib.MultigridError):
            on.set_option(lib.MG_OPT_DEEP_CALLS, bad)


def test_grid_barrier_wait_runs_out_and_reports_timeout(lib):
    """Bounded grid-barrier waits: with the test hook one CTA of each deep launch leaves as it
    starts; the others' first barrier wait runs out (0.5 s), they record the timeout and leave, the
    solve reports MG_ERR_TIMEOUT (-4), and the same handle then solves as a fresh one does, bit for
    bit (the barrier words were cleared and the context stays usable)."""
    import time
    import torch
    n, levels = 1023, 10
    f = dev(rhs_normal(n, 0))
    mg = lib.Multigrid(n, 1e-4, math.pi / 3, levels)
    mg.set_option(lib.MG_OPT_TEST_STALL_BARRIER, 5)
    assert mg.get_option(lib.MG_OPT_TEST_STALL_BARRIER) == 5
    t0 = time.perf_counter()
    with pytest.raises(lib.MultigridError, match=r"\(-4\)"):
        mg.solve(torch.zeros_like(f), f, 1, 1e-8, 1)  # a V-cycle: one deep launch
    waited = time.perf_counter() - t0
    mg.set_option(lib.MG_OPT_TEST_STALL_BARRIER, -1)
    v = torch.zeros_like(f)
    st = mg.solve(v, f, 4, 1e-8, 500)
    fresh = lib.Multigrid(n, 1e-4, math.pi / 3, levels)
    w = torch.zeros_like(f)
    st2 = fresh.solve(w, f, 4, 1e-8, 500)
    print(f"timed-out solve took {waited:.2f} s")
    assert st[0] == 0 and st == st2 and torch.equal(v, w)
    with pytest.raises(lib.MultigridError):
        mg.set_option(lib.MG_OPT_TEST_STALL_BARRIER, -3)


@pytest.mark.parametrize("n,levels,coarse_n,deep,nu1,nu2,kappa", [
    (1023, 10, 7, 511, 2, 2, 3),    # six levels in one launch (511^2 down to 15^2), P at 7^2
    (1023, 10, 3, 511, 2, 2, 2),    # seven would be too many: the launches start at 255^2
    (511, 9, 15, 255, 1, 3, 4),     # other sweep counts
    (511, 9, 31, 127, 0, 2, KAPPA_W),  # no pre-smoothing
    (255, 8, 31, 63, 3, 1, 1),
])
def test_fp64_deep_shapes_equal_separate_launches(lib, n, levels, coarse_n, deep, nu1, nu2, kappa):
    """Depths, coarse thresholds and sweep counts: bit for bit the separate launches, and the
    launch count that mg_counters gives."""
    import torch
    on = lib.Multigrid(n, 1e-3, 0.4, levels, nu1=nu1, nu2=nu2, coarse_n=coarse_n)
    off = lib.Multigrid(n, 1e-3, 0.4, levels, nu1=nu1, nu2=nu2, coarse_n=coarse_n)
    on.set_option(lib.MG_OPT_DEEP_CALLS, deep)
    off.set_option(lib.MG_OPT_DEEP_CALLS, 0)
    f = dev(rhs_normal(n, 31))
    a, b = torch.zeros_like(f), torch.zeros_like(f)
    for _ in range(2):
        on.kcycle(a, f, kappa)
        off.kcycle(b, f, kappa)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    launches = on.counters(kappa)[1]
    assert on.get_option(lib.MG_OPT_LAUNCHES) == launches < off.counters(kappa)[1]


def test_fp32_deep_with_maps_too_large_to_stage(lib):
    """With the FP32 coarse kernel at 63^2 the condensed maps (3969 x 3969) have more rows per CTA
    than shared memory holds: the deep launch reads them from global memory (asked of L2 ahead),
    bit for bit the separate launches."""
    import torch
    n, levels = 1023, 10
    f32 = dev(rhs_uniform(n, 12), "float32")
    outs = {}
    for deep in (127, 0):
        mg = lib.Multigrid(n, 1e-3, 0.7, levels)
        mg.set_option(lib.MG_OPT_COARSE_N32, 63)
        mg.set_option(lib.MG_OPT_DEEP_CALLS, deep)
        v = torch.zeros_like(f32)
        for _ in range(2):
            mg.kcycle_f32(v, f32, 3)
        torch.cuda.synchronize()
        outs[deep] = v.clone()
        if deep:  # the 127^2 level (3) runs inside deep launches
            sms = torch.cuda.get_device_properties(0).multi_processor_count
            assert mg.level_grid(3, fp32=True)[1] in (sms, 2 * sms)
        mg.close()
    assert torch.equal(outs[127], outs[0])


@pytest.mark.parametrize("n,levels,deep,nu1,nu2,kappa", [
    (1023, 10, 511, 2, 2, 3),         # four levels of passes (511^2 down to 63^2) in one launch
    (1023, 10, 255, 2, 2, KAPPA_W),
    (511, 9, 255, 2, 3, 2),           # three post-sweeps: no merged phases
    (511, 9, 255, 1, 2, 4),           # one pre-sweep: the pass B phases merged, not B with A
    (255, 8, 127, 2, 2, 1),           # a V-cycle: no second child
])
def test_fp32_deep_merged_phases_equal_separate_launches(lib, n, levels, deep, nu1, nu2, kappa):
    """FP32 deep launches from 511^2, 255^2 and 127^2 with the tensor-copy passes off (the separate
    launches then use the tile passes at every level): the merged phases (a first child's pass B
    with the second child's pass A, the last child's pass B with its parent's) give the separate
    launches' cycles bit for bit."""
    import torch
    f32 = dev(rhs_normal(n, 17), "float32")
    outs = {}
    for d in (deep, 0):
        mg = lib.Multigrid(n, 1e-3, 0.9, levels, nu1=nu1, nu2=nu2)
        mg.set_option(lib.MG_OPT_TMA_PASSES, 0)
        mg.set_option(lib.MG_OPT_DEEP_CALLS, d)
        v = torch.zeros_like(f32)
        for _ in range(2):
            mg.kcycle_f32(v, f32, kappa)
        torch.cuda.synchronize()
        outs[d] = v.clone()
        mg.close()
    assert torch.equal(outs[deep], outs[0])
