"""Build step for the CPU oracle (test infrastructure only).

Compiles oracle/gic_oracle.c into oracle/liboracle.so with gcc, FP64, no FMA
contraction (-ffp-contract=off), no architecture-specific flags, so it builds
and gives the same results on x86_64 and aarch64 hosts. OpenMP serves only
or_spmv_threads (the all-core CPU timing of the product; same results).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gic_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-Wall", "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
