"""Compile the oracle's C direct-sum kernels (TEST INFRASTRUCTURE ONLY).

Builds oracle/_mdc_direct.so from oracle/mdc_direct.c with gcc, OpenMP and -O2 (no fast-math, so the
FP64 summation order is the one written in the source).  Portable C: the same source builds on x86_64
and aarch64.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mdc_direct.c")
LIB = os.path.join(HERE, "_mdc_direct.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
