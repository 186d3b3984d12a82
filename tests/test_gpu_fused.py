"""Fused calls (MG_OPT_FUSED_CALL): a call at the level just above the coarse kernel's runs as one
thread-block-cluster launch (pass A over that level's tiles, the coarse walk or the condensed
child calls, pass B) instead of three launches; with the default 2, a call two levels above runs
with its child calls as one launch too. Every point's arithmetic is that of the separate launches,
so iterates, histories and iteration counts must be equal bit for bit, and the graph must hold the
launches counted by saved_launches fewer. Oracle parity of the default (fused) path is in test_gpu_parity,
test_gpu_mixed and the others."""
import math

import numpy as np
import pytest

from paper_2010_00626_b300.inputs import KAPPA_W, rhs_normal, rhs_uniform

pytestmark = pytest.mark.gpu


def dev(a, dtype="float64"):
    import torch
    return torch.tensor(a, dtype=getattr(torch, dtype), device="cuda")


def pair(lib, *args, **kw):
    # FP64 fused calls run at 31^2, the level above a 15^2 coarse kernel (the default coarse kernel
    # at 31^2 leaves the FP64 cycle no level with at most 16 tiles above it)
    kw.setdefault("coarse_n", 15)
    on = lib.Multigrid(*args, **kw)
    off = lib.Multigrid(*args, **kw)
    for mg in (on, off):  # the fused calls, not the persistent deep launches that would contain them
        mg.set_option(lib.MG_OPT_DEEP_CALLS, 0)
    off.set_option(lib.MG_OPT_FUSED_CALL, 0)
    assert on.get_option(lib.MG_OPT_FUSED_CALL) == 1 and off.get_option(lib.MG_OPT_FUSED_CALL) == 0
    return on, off


def saved_launches(calls, lc, fused=1):
    """Launches a cycle saves with fused calls: each call one level above the coarse kernel's (not
    at level 0) is one launch in place of three; with fused = 2 a call two levels above (not at
    level 0) is one launch in place of its own two and the three of each child call."""
    if fused == 2 and lc - 2 >= 1:
        return calls[lc - 2] + 3 * calls[lc - 1]
    return 2 * calls[lc - 1] if lc - 1 >= 1 else 0


def first_coarse_level(n, levels, coarse_n):
    sides = [(n + 1) // 2 ** l - 1 for l in range(levels)]
    return next((l for l, s in enumerate(sides) if s <= coarse_n), levels - 1)


@pytest.mark.parametrize("n,levels,kappa", [(63, 6, 2), (127, 7, 1), (127, 7, KAPPA_W), (255, 8, 2),
                                            (255, 8, 3), (1023, 10, 4), (31, 5, 3)])
def test_fp64_cycles_equal_bitwise(lib, n, levels, kappa):
    import torch
    on, off = pair(lib, n, 1e-3, 0.7, levels)
    f = dev(rhs_uniform(n, 3))
    v_on, v_off = torch.zeros_like(f), torch.zeros_like(f)
    for _ in range(3):
        on.kcycle(v_on, f, kappa)
        off.kcycle(v_off, f, kappa)
        torch.cuda.synchronize()
        assert torch.equal(v_on, v_off)
    calls, launches, _ = on.counters(kappa)
    assert on.get_option(lib.MG_OPT_LAUNCHES) == launches
    assert off.get_option(lib.MG_OPT_LAUNCHES) == off.counters(kappa)[1]
    lc = first_coarse_level(n, levels, 15)
    assert off.counters(kappa)[1] - launches == saved_launches(calls, lc)


def test_fp64_solve_and_pcg_equal_bitwise(lib):
    import torch
    n, levels = 511, 9
    on, off = pair(lib, n, 1e-4, math.pi / 3, levels)
    f = dev(rhs_normal(n, 0))
    outs = []
    for mg in (on, off):
        v = torch.zeros_like(f)
        st = mg.solve(v, f, 4, 1e-8, 2000)
        x = torch.zeros_like(f)
        pc = mg.pcg(x, f, 3, 1e-10, 500, flexible=True)
        torch.cuda.synchronize()
        outs.append((st, pc, v.clone(), x.clone()))
    (s1, p1, v1, x1), (s2, p2, v2, x2) = outs
    assert s1 == s2 and p1 == p2
    assert torch.equal(v1, v2) and torch.equal(x1, x2)


def test_fp32_cycles_and_mixed_solve_equal_bitwise(lib):
    """FP32 cycles: the fused level is 63^2 (tiles of 16^2) above the FP32 coarse kernel at 31^2."""
    import torch
    n, levels = 255, 8
    on, off = pair(lib, n, 1e-3, 0.7, levels)
    f32 = dev(rhs_uniform(n, 5), "float32")
    a, b = torch.zeros_like(f32), torch.zeros_like(f32)
    for _ in range(3):
        on.kcycle_f32(a, f32, 3)
        off.kcycle_f32(b, f32, 3)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
    assert on.level_grid(2, fp32=True) == (63, 16) and off.level_grid(2, fp32=True) == (63, 64)
    f = dev(rhs_uniform(n, 6))
    res = []
    for mg in (on, off):
        x = torch.zeros_like(f)
        r = mg.solve_mixed(x, f, 3, 1e-8, 500)
        torch.cuda.synchronize()
        res.append((r, x.clone()))
    assert res[0][0] == res[1][0] and torch.equal(res[0][1], res[1][1])


def test_convection_cycles_equal_bitwise(lib):
    """The general-stencil (upwind convection) variant of the fused launch."""
    import torch
    n, levels = 255, 8
    kw = dict(convection=(300.0, -120.0), coarse_op="rediscretized")
    on, off = pair(lib, n, 1e-2, math.pi / 6, levels, **kw)
    f = dev(rhs_normal(n, 2))
    v_on, v_off = torch.zeros_like(f), torch.zeros_like(f)
    for _ in range(3):
        on.kcycle(v_on, f, 3)
        off.kcycle(v_off, f, 3)
        torch.cuda.synchronize()
        assert torch.equal(v_on, v_off)


def test_batch_equal_bitwise(lib):
    import torch
    ns, epss, thetas = [63, 127, 255], [1e-2, 1e-3, 1e-4], [0.3, 1.1, 2.4]
    runs = []
    for fused in (2, 1, 0):
        batch = lib.Batch(ns, epss, thetas)
        batch.set_option(lib.MG_OPT_FUSED_CALL, fused)
        fs = [dev(rhs_uniform(n, 40 + i)) for i, n in enumerate(ns)]
        xs = [torch.zeros_like(f) for f in fs]
        out = batch.solve(xs, fs, 3, 1e-8, 2000, mixed=True)
        torch.cuda.synchronize()
        runs.append((out, [x.clone() for x in xs]))
    for r in runs[1:]:
        assert runs[0][0] == r[0]
        assert all(torch.equal(a, b) for a, b in zip(runs[0][1], r[1]))


@pytest.mark.parametrize("nu1,nu2", [(0, 3), (3, 1), (1, 0)])
def test_fp64_cycles_equal_bitwise_other_sweeps(lib, nu1, nu2):
    """Pre- or post-smoothing counts other than 2 (including none) through the fused launch."""
    import torch
    n, levels = 255, 8
    on, off = pair(lib, n, 1e-2, 1.2, levels, nu1, nu2)
    f = dev(rhs_normal(n, 7))
    v_on, v_off = torch.zeros_like(f), torch.zeros_like(f)
    for _ in range(2):
        on.kcycle(v_on, f, 3)
        off.kcycle(v_off, f, 3)
        torch.cuda.synchronize()
        assert torch.equal(v_on, v_off)
    f32 = dev(rhs_uniform(n, 8), "float32")
    a, b = torch.zeros_like(f32), torch.zeros_like(f32)
    on.kcycle_f32(a, f32, 2)
    off.kcycle_f32(b, f32, 2)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("n,levels,kappa", [(255, 8, 3), (4095, 12, 4)])
def test_one_and_two_level_fusion_equal_bitwise(lib, n, levels, kappa):
    """MG_OPT_FUSED_CALL = 2 (calls two levels above the coarse kernel fused with their child calls)
    against 1 (only the level just above): same iterates in FP64 and FP32."""
    import torch
    two = lib.Multigrid(n, 3e-4, 2.2, levels, coarse_n=15)  # FP64: the fused levels above 15^2
    one = lib.Multigrid(n, 3e-4, 2.2, levels, coarse_n=15)
    for mg in (two, one):
        mg.set_option(lib.MG_OPT_DEEP_CALLS, 0)
    two.set_option(lib.MG_OPT_FUSED_CALL, 2)
    f = dev(rhs_uniform(n, 9))
    a, b = torch.zeros_like(f), torch.zeros_like(f)
    for _ in range(2):
        two.kcycle(a, f, kappa)
        one.kcycle(b, f, kappa)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    f32 = dev(rhs_uniform(n, 10), "float32")
    a, b = torch.zeros_like(f32), torch.zeros_like(f32)
    two.kcycle_f32(a, f32, kappa)
    one.kcycle_f32(b, f32, kappa)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    two.set_option(lib.MG_OPT_FUSED_CALL, 2)
    two.kcycle(torch.zeros_like(f), f, kappa)
    calls, launches, _ = two.counters(kappa)
    assert two.get_option(lib.MG_OPT_LAUNCHES) == launches
    lc = first_coarse_level(n, levels, 15)
    assert one.counters(kappa)[1] - launches == calls[lc - 2] + calls[lc - 1]
