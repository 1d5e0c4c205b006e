"""In-tree build of libsoma.so for sm_103a (nvcc; no JIT cache, no torch types)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsoma.so")
# checked build (-DSOMA_DEBUG): bounds checks in the move kernel that set the
# device error word, the stand-in for a memory checker on this platform
OBJ_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libsoma_debug.so")
SOURCES = ["soma_move.cu", "soma_kernels.cu", "soma_f64.cu", "soma_sort.cu", "soma_scan.cu", "soma_api.cu",
           "soma_noalloc.cu"]
HEADERS = ["soma_internal.cuh", "soma_launch.h", "soma_device.cuh"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
                "--expt-relaxed-constexpr", "-I", os.path.join(HERE, "..", "include")]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, extra_flags=(), debug=False):
    """Compile every CUDA source of the package and link libsoma.so (or, with
    debug=True, the checked libsoma_debug.so); returns its path."""
    OBJ, LIB = (OBJ_DEBUG, LIB_DEBUG) if debug else (globals()["OBJ"], globals()["LIB"])
    if debug:
        extra_flags = list(extra_flags) + ["-DSOMA_DEBUG"]
    os.makedirs(OBJ, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(HERE, "..", "include", "soma.h")]
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OBJ, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            cmd = [NVCC] + FLAGS + list(extra_flags) + ["-c", s, "-o", o]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            subprocess.check_call(cmd)
    if force or _stale(LIB, objs):
        cmd = [NVCC] + ARCH + ["-shared", "-cudart", "shared", "-o", LIB] + objs
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [], debug="--debug" in sys.argv)
