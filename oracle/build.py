"""Compile the FP64 oracle (plain C, gcc) into a shared library.

Test infrastructure only: building the checker is not using it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["oracle_core.c", "oracle_planes.c", "oracle_pipeline.c", "oracle_color.c"]
LIB = os.path.join(HERE, "_build", "liboracle.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SOURCES + ["oracle.h"]
    return any(os.path.getmtime(os.path.join(HERE, s)) > t for s in deps)


def build(force: bool = False, openmp: bool = True) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wno-unused-function",
           "-ffp-contract=off"]
    if openmp:
        cmd.append("-fopenmp")
    cmd += [os.path.join(HERE, s) for s in SOURCES] + ["-lm", "-o", LIB + ".tmp"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
