"""Build the CPU oracle (test infrastructure) into oracle/liboracle.so.

Only tests/, __graft_entry__ and bench.py's cpu_baseline / reference arm use
the oracle.  It is compiled without fused multiply-add contraction and without
fast-math so that every float operation is one IEEE 754 round-to-nearest step.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "szx_ref.c")
LIB = os.path.join(HERE, "liboracle.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
          "-fno-strict-aliasing", "-Wall", "-Wextra", "-shared", "-fPIC"]


def build(force=False):
    """Compile szx_ref.c when the library is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)
            and os.path.getmtime(LIB) >= os.path.getmtime(os.path.join(HERE, "szx_ref.h"))):
        return LIB
    cmd = ["gcc", *CFLAGS, SRC, "-o", LIB + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
