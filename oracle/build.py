"""Compile the C oracle into oracle/liboracle.so (test infrastructure only).

Flags: -O2 with FMA contraction off and no fast-math, so every float
operation in the oracle is one correctly rounded IEEE-754 operation in the
order the source writes it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mmr_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
          "-fexcess-precision=standard", "-Wall", "-Wextra"]


OMP_SRC = os.path.join(HERE, "mmr_cpu_omp.c")
OMP_LIB = os.path.join(HERE, "libcpu_omp.so")


def _compile(srcs, lib, extra, force):
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= max(os.path.getmtime(s) for s in srcs)):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, *extra, *srcs, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """The single-threaded oracle."""
    return _compile([SRC], LIB, [], force)


def build_omp(force: bool = False) -> str:
    """The OpenMP CPU baseline (mmr_cpu_omp.c over the oracle's routines),
    with the oracle's floating-point flags, so its frames equal the
    oracle's."""
    return _compile([OMP_SRC, SRC], OMP_LIB, ["-fopenmp"], force)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build_omp(force="--force" in sys.argv))
