"""Compile the CPU oracle (test infrastructure only) into oracle/liblcq_oracle.so.

The flags are the paper's parity fix (Sec. 3.2): no FMA, no contraction, no
fast-math; -frounding-math keeps the directed-rounding helpers of the NOA
range at run time.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lcq_oracle.c")
LIB = os.path.join(HERE, "liblcq_oracle.so")

CFLAGS = [
    "-std=gnu11", "-O2", "-fPIC", "-shared",
    "-ffp-contract=off", "-mno-fma", "-fno-fast-math",
    "-frounding-math", "-fexcess-precision=standard",
    "-Wall", "-Wextra", "-Wno-unknown-pragmas",
]


def build(force: bool = False) -> str:
    """Compile the oracle if the library is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", *CFLAGS, "-o", tmp, SRC, "-lquadmath", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
