"""Build the CPU oracle (test infrastructure) into oracle/libtco.so with gcc.

Plain C, -O2, no fused multiply-add contraction and no fast-math, so every
operation rounds as written in tco.c.  A second build, oracle/libtco_omp.so,
compiles the same source with -fopenmp: its only difference is that the
independent rows of tco_rows_grad run on all host threads (the multi-core CPU
baseline); every result is bit-identical to the plain build.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tco.c")
LIB = os.path.join(HERE, "libtco.so")


LIB_OMP = os.path.join(HERE, "libtco_omp.so")


def build(force: bool = False, openmp: bool = False) -> str:
    lib = LIB_OMP if openmp else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(SRC):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wextra"] + (["-fopenmp"] if openmp else []) + ["-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build(force="--force" in sys.argv, openmp=True))
