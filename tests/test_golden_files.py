"""The stored full-size oracle runs (tests/golden/large_standalone_cycles_k*.json, written by
oracle/full_size_cycles.py) are self-consistent: the cycle count is the first cycle whose relative
residual is at or below the tolerance, the residual history decreases, and the counts do not grow
with kappa (a larger counter spends more coarse-grid work per cycle; Tables 4-6 of the paper show
the same ordering)."""
import glob
import json
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
FILES = sorted(glob.glob(os.path.join(HERE, "golden", "large_standalone_cycles_k*.json")))


def load(p):
    with open(p) as fh:
        return json.load(fh)


@pytest.mark.parametrize("path", FILES, ids=[os.path.basename(p) for p in FILES])
def test_golden_run_is_consistent(path):
    d = load(path)
    h, tol = d["history"], d["tol"]
    assert d["written_by"] == "oracle/full_size_cycles.py"
    assert (d["n"], d["levels"], tol) == (4095, 12, 1e-8)
    assert d["cycles"] == len(h)
    assert h[-1] <= tol < h[-2]
    assert all(b < a for a, b in zip(h, h[1:]))  # every cycle reduces the residual
    assert 0.1 < h[0] < 1.0


def test_first_cycles_run_is_consistent():
    """The oracle's first 200 V-cycles of the same solve (oracle/full_size_cycles.py --first 200):
    no tolerance applied, every cycle reduces the residual, and it has not reached 1e-8 (the full
    V-cycle solve needs about 4100 cycles)."""
    d = load(os.path.join(HERE, "golden", "large_standalone_first200_k1.json"))
    h = d["history"]
    assert d["written_by"] == "oracle/full_size_cycles.py" and d["tol"] is None and d["kappa"] == 1
    assert (d["n"], d["levels"], d["cycles"], len(h)) == (4095, 12, 200, 200)
    assert all(b < a for a, b in zip(h, h[1:]))
    assert 1e-8 < h[-1] < h[0] < 1.0


def test_counts_do_not_grow_with_kappa():
    counts = sorted((load(p)["kappa"], load(p)["cycles"]) for p in FILES)
    assert len(counts) >= 2
    assert all(c2 <= c1 for (_, c1), (_, c2) in zip(counts, counts[1:])), counts
