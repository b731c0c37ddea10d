"""Build the FP64 CPU oracle (test infrastructure) into oracle/_build/.

Plain gcc, no fast-math and no FP contraction, so that every arithmetic
operation is an IEEE double operation on both x86-64 and aarch64.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "eslbm_oracle.c")
HDR = os.path.join(HERE, "eslbm_oracle.h")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
LIB_OMP = os.path.join(OUT_DIR, "liboracle_omp.so")  # the same source with OpenMP over cells and planes


def up_to_date(lib=LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return t >= os.path.getmtime(SRC) and t >= os.path.getmtime(HDR)


def _compile(lib, extra):
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-Wall", "-Wextra", "-Wno-unknown-pragmas", *extra, "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """The single-threaded oracle (what the tests load)."""
    if not force and up_to_date(LIB):
        return LIB
    return _compile(LIB, [])


def build_openmp(force: bool = False):
    """The OpenMP build (cells and planes split over the host cores; the same arithmetic per cell),
    or None where the compiler has no OpenMP."""
    if not force and up_to_date(LIB_OMP):
        return LIB_OMP
    try:
        return _compile(LIB_OMP, ["-fopenmp"])
    except (subprocess.CalledProcessError, OSError):
        return None


if __name__ == "__main__":
    print(build(force=True))
    print(build_openmp(force=True))
