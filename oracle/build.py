"""Compile the oracle's C source into a shared library (test infrastructure only).

The oracle is the reference the CUDA library is compared with; building it is
not using it.  Only the tests, the smoke check and the benchmark's CPU-baseline
leg load the library this script writes.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dsmc_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Build ``oracle/_build/liboracle.so`` if missing or stale; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    # -ffp-contract=off: no fused multiply-add, so rounding follows the source
    # on every host (aarch64 gcc contracts by default).
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off",
           "-fno-fast-math", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
