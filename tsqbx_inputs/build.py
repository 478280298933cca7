"""Compile the octree/list builder (octree.cpp) into tsqbx_inputs/liboctree.so."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "octree.cpp")
LIB = os.path.join(HERE, "liboctree.so")


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(__file__)):
        return LIB
    # no FMA contraction: the geometric tests round every product and sum
    # separately on every host (aarch64 g++ would otherwise fuse d2 += t * t),
    # which is also how the GPU builder evaluates them
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-Wall", "-Wextra", "-ffp-contract=off", SRC,
           "-o", LIB + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stderr)
        raise RuntimeError("octree builder compilation failed")
    os.replace(LIB + ".tmp", LIB)
    if verbose:
        print(" ".join(cmd))
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
