"""Build libsu2.so, the CUDA library behind include/su2.h, in-tree.

nvcc compiles each translation unit for sm_103a only (in parallel), and links
them into paper_1010_4834_gb300/_build/libsu2.so with the CUDA runtime linked
statically.  Rebuilds only when a source is newer than the library.
"""
import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libsu2.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path():
    p = shutil.which("nvcc")
    if p:
        return p
    for c in ("/usr/local/cuda/bin/nvcc",):
        if os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsu2")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale():
    if not os.path.exists(LIB):
        return True
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
    deps += glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]
    return os.path.getmtime(LIB) < max(os.path.getmtime(d) for d in deps)


def build(force=False, verbose=False, extra_flags=(), out=None):
    """Compile libsu2.so if needed; return its path.  `out` and `extra_flags`
    build a separately named variant (used for tuning sweeps)."""
    lib = out or LIB
    if not force and out is None and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tag = "" if out is None else "." + os.path.basename(out).replace(".so", "")
    nvcc = nvcc_path()
    # -ftz=true: FP32 denormals flush to zero (link components and sums are
    # O(1); it removes the denormal fix-ups around the SFU approximations).
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-ftz=true", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                     "-I", CSRC] + list(extra_flags)

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.basename(src) + tag + ".o")
        cmd = [nvcc] + common + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0 or verbose:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s" % src)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("linking libsu2.so failed")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv,
                extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else ()))
