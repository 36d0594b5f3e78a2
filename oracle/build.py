"""Build step for the oracle's C library (test infrastructure only).

Compiles ``hpr_oracle.c`` into ``liborc_hpr.so`` beside it with gcc, FP64, OpenMP over
matrix rows (each row is summed in index order, so results do not depend on the
thread count).  ``-ffp-contract=off`` keeps a * b + c as two roundings, exactly as
written in the source.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hpr_oracle.c")
LIB = os.path.join(HERE, "liborc_hpr.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", LIB, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
