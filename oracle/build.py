"""Compile the CPU oracle (test infrastructure) into oracle/_build/liblap5oracle.so.

Plain C11, -ffp-contract=off so that every multiply-add in the oracle is two
roundings exactly as written.  Only tests, the smoke check and the benchmark's
CPU-baseline leg load the result.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lap5_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblap5oracle.so")


LIB_OMP = os.path.join(OUT_DIR, "liblap5oracle_omp.so")


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle if the shared library is missing or older than its source.

    openmp=True builds the timing variant (-fopenmp -DORA_OMP): the same source
    with its binary64 row loops on all threads and per-thread partial dot
    products.  It serves the benchmark's CPU-baseline timing only; parity uses
    the sequential build."""
    lib = LIB_OMP if openmp else LIB
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= os.path.getmtime(SRC)):
        return lib
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-Wall", "-o", tmp, SRC, "-lm"]
    if openmp:
        cmd[1:1] = ["-fopenmp", "-DORA_OMP"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    if "--openmp" in sys.argv:
        print(build(force="--force" in sys.argv, openmp=True))
