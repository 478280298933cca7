"""Compile the FP64 CPU oracle (oracle.c) into oracle/liboracle.so.

Test infrastructure: only tests, the smoke check and the benchmark's CPU
baseline load the result.  OpenMP is used when the compiler supports it (the
per-target loops are independent); otherwise the library is single-threaded.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra",
            "-fno-fast-math", "-ffp-contract=off", SRC, "-o", LIB + ".tmp", "-lm"]
    for extra in (["-fopenmp"], []):
        cmd = base[:1] + extra + base[1:]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(LIB + ".tmp", LIB)
            if verbose:
                print(" ".join(cmd))
            return LIB
    sys.stderr.write(r.stderr)
    raise RuntimeError("oracle build failed")


if __name__ == "__main__":
    print(build(force=True, verbose=True))
