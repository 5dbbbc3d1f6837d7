"""Build the oracle's C library (test infrastructure only).

Compiles ``oracle/wilson.c`` into ``oracle/liboracle_wilson.so`` with plain
gcc.  ``-ffp-contract=off`` keeps FP64 alias-table arithmetic free of fused
multiply-adds, so the tables are the same on every host.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "wilson.c")
LIB = os.path.join(HERE, "liboracle_wilson.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
           "-pthread", "-Wall", "-Wextra", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
