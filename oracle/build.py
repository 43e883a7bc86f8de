"""Compile the FP64 CPU oracle (plain C) into oracle/_lib/libxrd_oracle.so.

The oracle is test infrastructure: the tests, the package smoke check and the
CPU-baseline leg of the benchmark load it; the CUDA library never does.
-ffp-contract=off keeps every product and sum rounded on its own, as written.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "_lib", "libxrd_oracle.so")
SRC = os.path.join(HERE, "xrd_oracle.c")


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "xrd_oracle.h"))):
        return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           SRC, "-o", LIB + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
