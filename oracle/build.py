"""Compile the FP64 oracle (oracle/rbmd_oracle.c) into oracle/_rbmd_oracle.so.

Test infrastructure only: the oracle is the checker for the CUDA library and
is never linked into it.  Built with plain gcc, -O2, no fast-math and no
floating-point contraction, so that every operation rounds as written.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rbmd_oracle.c")
OUT = os.path.join(HERE, "_rbmd_oracle.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(OUT)
            and os.path.getmtime(OUT) >= os.path.getmtime(SRC)):
        return OUT
    tmp = OUT + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
