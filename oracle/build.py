"""Compile the C oracle into ``oracle/_build/liboracle.so``.

Test infrastructure only: the oracle is built so that the test-suite, the smoke
check and the CPU-baseline leg of ``bench.py`` can load it.  Plain ``gcc``; no
x86- or Arm-specific flags, so the same source gives the same results on both.
``-ffp-contract=off`` keeps every binary32/binary64 operation individually
rounded (the acceptance threshold routine relies on that); ``fmaf`` is called
explicitly where a fused operation is meant.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rewl_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wno-unused-function", "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
