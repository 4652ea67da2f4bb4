"""Build the CUDA library libgeotrace.so in-tree for sm_103a (nvcc, no cmake).

Every translation unit under csrc/ is compiled in parallel with
``-gencode arch=compute_103a,code=sm_103a``; the objects are linked into
``paper_2310_15183_gb300/libgeotrace.so`` against the shared CUDA runtime.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgeotrace.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
         "-I" + INCLUDE]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgeotrace")
    return path


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + \
        sorted(glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _deps())


def _compile(src: str) -> tuple:
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
    extra = os.environ.get("GT_NVCC_EXTRA", "").split()  # e.g. -DGT_FIELD_NOINLINE
    cmd = [nvcc()] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, p.stdout, p.stderr))
    return obj, p.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/*.cu for sm_103a and link libgeotrace.so (skipped when up to date)."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, len(_sources()))) as ex:
        results = list(ex.map(_compile, _sources()))
    with open(os.path.join(BUILD, "ptxas.log"), "w") as f:
        for obj, log in results:
            f.write("== %s\n%s\n" % (os.path.basename(obj), log))
    if verbose:
        for obj, log in results:
            print(log)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + [o for o, _ in results]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (p.stdout, p.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))


OPCOUNT_SRC = os.path.join(HERE, "opcount.cpp")
OPCOUNT_BIN = os.path.join(BUILD, "opcount")


def op_counts() -> dict:
    """Build (host C++, no GPU) and run the op counter: algorithmic flops per RK4 step
    counted from the kernels' own spacetime templates."""
    import json
    os.makedirs(BUILD, exist_ok=True)
    deps = [OPCOUNT_SRC, os.path.join(CSRC, "spacetime.cuh")]
    if (not os.path.exists(OPCOUNT_BIN)
            or any(os.path.getmtime(p) > os.path.getmtime(OPCOUNT_BIN) for p in deps)):
        cuda_inc = os.path.join(os.path.dirname(os.path.dirname(nvcc())), "include")
        subprocess.run(["g++", "-std=c++17", "-O0", "-x", "c++", "-I" + cuda_inc, OPCOUNT_SRC,
                        "-o", OPCOUNT_BIN], check=True)
    return json.loads(subprocess.run([OPCOUNT_BIN], check=True, capture_output=True,
                                     text=True).stdout)
