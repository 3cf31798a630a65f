"""Build the bit-vectorized CPU baseline (w = 64) as a shared library beside its source.

Plain gcc with OpenMP and portable flags, so the same source builds on x86_64 and aarch64.
Only the benchmark's CPU-baseline legs and the tests load it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sca_bitvec.c")
LIB = os.path.join(HERE, "libbitvec.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall", "-Wextra",
                           "-o", tmp, SRC, "-lm"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
