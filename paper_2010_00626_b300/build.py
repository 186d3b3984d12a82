"""Build libkcycle.so in-tree for sm_103a (B300) with nvcc.

    python -m paper_2010_00626_b300.build

The library is written next to this file so that it travels with the source tree.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libkcycle.so")
SOURCES = [os.path.join(HERE, "csrc", "kcycle.cu")]


def deps():
    """Every file the library is built from: all sources and headers under csrc/ and include/
    (a glob, so that a new header can never be left out of the staleness check)."""
    pats = [os.path.join(HERE, "csrc", "*.cu"), os.path.join(HERE, "csrc", "*.cuh"),
            os.path.join(HERE, "csrc", "*.h"), os.path.join(ROOT, "include", "*.h")]
    return sorted({p for pat in pats for p in glob.glob(pat)} | set(SOURCES))


def nvcc_command(out: str = LIB, extra=()):
    nvcc = os.environ.get("NVCC", "nvcc")
    return [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
            "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC", "-shared", "-I", os.path.join(ROOT, "include"),
            *extra, "-o", out, *SOURCES]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if force or not up_to_date():
        cmd = nvcc_command()
        if verbose:
            print(" ".join(cmd))
        subprocess.run(cmd, check=True)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
