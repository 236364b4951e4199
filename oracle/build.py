"""Build the CPU oracle shared library (test infrastructure only).

Plain C, FP64, compiled with FMA contraction off so that x86_64 and aarch64
hosts round identically.  Two builds of the same source: the serial library
the tests use, and an OpenMP one whose substep loop shares the sites of a
(direction, parity) class among all host cores, for the all-cores CPU
baseline of the benchmark (same links, same counts).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "su2_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle_su2.so")
LIB_OMP = os.path.join(OUT_DIR, "liboracle_su2_omp.so")


def _compile(out, extra, force):
    deps = [SRC, os.path.join(HERE, "su2_oracle.h"), os.path.abspath(__file__)]
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= max(os.path.getmtime(d) for d in deps)):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wno-unknown-pragmas"] + extra + ["-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False, omp: bool = False) -> str:
    """Compile su2_oracle.c into oracle/_build/liboracle_su2.so (omp=True:
    liboracle_su2_omp.so, with OpenMP); return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if omp:
        return _compile(LIB_OMP, ["-fopenmp"], force)
    return _compile(LIB, [], force)


def build_all(force: bool = False):
    return build(force), build(force, omp=True)


if __name__ == "__main__":
    print(build_all(force=True))
