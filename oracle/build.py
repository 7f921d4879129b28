"""Compile the FP64 oracle (test infrastructure) into oracle/libd2oracle.so.

Plain gcc, no FMA contraction so that the rounding matches the stated
summation orders.  Used by tests/, __graft_entry__.build() and the CPU
baseline leg of bench.py only.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "d2_oracle.c")
LIB = os.path.join(HERE, "libd2oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
