"""Compile the C part of the FP64 oracle (test infrastructure only).

The oracle is built so that tests, the smoke check and the CPU-baseline leg of
the benchmark can run it; the product library never links it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "saq_oracle.c")
LIB = os.path.join(HERE, "_saq_oracle.so")


def build(force: bool = False) -> str:
    import platform
    marker = LIB + ".arch"
    same_arch = os.path.exists(marker) and open(marker).read() == platform.machine()
    if (not force and same_arch and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    # IEEE semantics on purpose: no -ffast-math, no -march=native (the same
    # source must give the same results on x86_64 and aarch64 hosts).
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
           "-ffp-contract=off", SRC, "-o", LIB + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    with open(marker, "w") as f:
        f.write(platform.machine())
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
