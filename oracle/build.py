"""Builds the FP64 CPU oracle (oracle.c) into oracle/_build/liboracle.so with gcc.

Test infrastructure: the product path never loads this library.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-Wall", "-Wno-unused-function",
            SRC, "-o", tmp, "-lm"]
    # OpenMP over pixels when the compiler has it; the result does not depend on it
    for extra in (["-fopenmp"], []):
        cmd = base[:-3] + extra + base[-3:]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, LIB)
            if verbose:
                print(" ".join(cmd))
            return LIB
    sys.stderr.write(r.stderr)
    raise RuntimeError("oracle build failed")


if __name__ == "__main__":
    print(build(force=True, verbose=True))
