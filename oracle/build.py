"""Compile the FP64 CPU oracle (test infrastructure) into ``oracle/liboracle.so``.

Plain gcc, no vectorisation flags beyond -O2, so the same source gives the same
results on x86-64 and aarch64 hosts (``-ffp-contract=off`` keeps the compiler
from fusing multiply-adds, which would change rounding between the two).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hmc_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
           SRC, "-o", LIB + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
