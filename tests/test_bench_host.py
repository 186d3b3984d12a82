"""Host logic of the benchmark's per-level report (no GPU): bytes and FP64 operations per launch,
calls from zero, SM idle time, against hand counts for a three-level fake hierarchy."""
import math

import pytest

import bench


class FakeMG:
    """Three levels of sides 31, 15, 7; the 7^2 level is inside a one-CTA coarse kernel."""

    sides = [31, 15, 7]
    ctas = {0: 16, 1: 4, 2: 1}

    def counters(self, kappa):
        # calls per level of a kappa = 2 cycle on three levels: 1, 2, 3 (Proposition 2.2)
        return [1, 2, 3], None, None

    def level_grid(self, level, fp32=False):
        return self.sides[level], self.ctas[level]


def test_per_level_bytes_ops_and_idle():
    sms = 148
    # one cycle: pass A and B once at level 0, twice at level 1, and two coarse launches
    ms = [0.010, 0.020, 0.005, 0.005, 0.006, 0.006, 0.030, 0.030]
    kind = [0, 1, 0, 0, 1, 1, 2, 2]
    level = [0, 0, 1, 1, 1, 1, 2, 2]
    rep = bench.per_level_report(FakeMG(), (ms, kind, level), False, 1e12, 1000.0, True, sms, 2, False)
    rows = {(e["level"], e["kind"]): e for e in rep["levels"]}
    # level 0 pass A: v, f read, relaxed v written, coarse f (a quarter) written: 3.25 x 8 B per
    # point; 2 sweeps x 10 + residual 9 + full weighting 2.25 + the stopping test's square 1
    a0 = rows[(0, "pass_a")]
    assert a0["gb_s"] == pytest.approx(round(31 * 31 * 8 * 3.25 / 10e-6 / 1e9, 1))
    assert a0["fp64_frac"] == pytest.approx(round(31 * 31 * 32.25 / 10e-6 / 1e12, 4))
    # level 1 pass A: of its 2 calls, the first (below the level-0 call) starts from zero: no v read,
    # and its first sweep is one operation instead of ten
    a1 = rows[(1, "pass_a")]
    byt = 15 * 15 * 8 * (3.25 - 0.5)
    ops = 15 * 15 * (31.25 - 9 * 0.5)
    assert a1["gb_s"] == pytest.approx(round(byt / 5e-6 / 1e9, 1))
    assert a1["fp64_frac"] == pytest.approx(round(ops / 5e-6 / 1e12, 4))
    # pass B: interpolation + correction 3, 2 sweeps; no norm
    b1 = rows[(1, "pass_b")]
    assert b1["fp64_frac"] == pytest.approx(round(15 * 15 * 23 / 6e-6 / 1e12, 4))
    assert rows[(2, "coarse")]["us_per_launch"] == pytest.approx(30.0)
    assert "gb_s" not in rows[(2, "coarse")]
    # SM idle: every launch here has fewer CTAs than SMs
    idle = (0.030 * (sms - 16) + 0.022 * (sms - 4) + 0.060 * (sms - 1)) / sms
    assert rep["sm_idle"]["ms_per_cycle"] == pytest.approx(round(idle, 4))
    assert rep["sm_idle"]["launches_below_one_wave_ms"] == pytest.approx(round(sum(ms), 4))
    assert rep["sm_idle"]["frac_of_cycle"] == pytest.approx(round(idle / sum(ms), 4))


def test_per_level_fp32_from_zero():
    """FP32 cycle of the mixed solve: 4-byte fields, level 0 starts from zero, no FP64 fraction."""
    rep = bench.per_level_report(FakeMG(), ([0.004], [0], [0]), True, 1e12, 1000.0, False, 148, 2, True)
    e = rep["levels"][0]
    assert e["gb_s"] == pytest.approx(round(31 * 31 * 4 * 2.25 / 4e-6 / 1e9, 1))
    assert "fp64_frac" not in e


def test_profile_kinds_cover_the_abi():
    """Every launch kind mg_profile_cycle documents has a name."""
    assert set(bench.PROFILE_KINDS) == set(range(8))
    assert bench.PROFILE_KINDS[6] == "call" and bench.PROFILE_KINDS[7] == "deep"
    assert math.isclose(bench.dp_ops_per_point(0, 2, True)[0], 32.25)


def test_stored_traffic_is_dropped_when_the_kernel_source_changes(tmp_path, monkeypatch):
    src = tmp_path / "k.cuh"
    src.write_text("pass A body\n// Pass B: v <- v + P v_c\npass B body\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    entry = {"source": "k.cuh", "until": "// Pass B: v <- v + P v_c", "sha256": None, "bytes": 123}
    entry["sha256"] = bench.source_digest(entry)
    assert bench.measured_traffic(entry) == 123
    src.write_text("pass A body\n// Pass B: v <- v + P v_c\nchanged pass B body\n")
    assert bench.measured_traffic(entry) == 123  # outside the hashed section
    src.write_text("pass A body, changed\n// Pass B: v <- v + P v_c\npass B body\n")
    assert bench.measured_traffic(entry) is None


def test_stored_pass_a_traffic_matches_the_current_source():
    """The committed figure is used only while the pass A source it was captured on is unchanged."""
    got = bench.measured_traffic(bench.PASS_A_L0_TRAFFIC)
    assert got is None or got == bench.PASS_A_L0_TRAFFIC["bytes"]


def test_both_arms_print_the_same_config():
    cfg = bench.bench_config(4)
    for key in ("workload", "n", "levels", "theta", "eps", "kappa", "tol", "nu1", "nu2", "omega"):
        assert key in cfg
    assert "parallelism" not in cfg and bench.bench_config(4, 2)["parallelism"] == "replicas x2"
    assert set(bench.host_cpu()) == {"cpu_model", "nproc"}


def test_stored_fp32_pass_traffic_matches_the_current_source():
    """The FP32 tensor-copy passes' DRAM bytes are used only while tma_f32.cuh is the source the
    capture ran on; the stored figures are near the algorithmic bytes (4095^2: 151 MB for pass A from
    zero, 218 MB for pass B, writes partly still in L2 when the kernel ends)."""
    for kind, alg in (("pass_a", 9 * 4095 ** 2), ("pass_b", 13 * 4095 ** 2)):
        entry = bench.TMA_L0_TRAFFIC[kind]
        got = bench.measured_traffic(entry)
        assert got is None or got == entry["bytes"]
        assert 0.5 * alg < entry["bytes"] < 1.2 * alg
