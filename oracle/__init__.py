"""FP64 CPU oracle for the kappa-cycle multigrid of Avnat & Yavneh (arXiv 2010.00626).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it. The CUDA
product path never imports, calls or links anything in this package, and this package
never imports the product (only the seeded input generators in
``paper_2010_00626_b300.inputs`` are shared, and they hold no method arithmetic).

Everything here is plain numpy in float64, written for a reader to check against the
paper by eye: no blocking, no fusion, no reordering beyond what the paper states.
Library primitives (numpy array arithmetic, a dense Cholesky factorisation) serve as
steps.

Parity status of each function is stated in its docstring. Every function is pinned by
a CPU test in ``tests/test_oracle_*.py`` except the ones marked "parity unpinned".
"""
from .mg import *  # noqa: F401,F403
