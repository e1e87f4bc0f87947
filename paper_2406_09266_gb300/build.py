"""Builds libsymgpu.so in-tree for sm_103a (GB300) with nvcc.

Each .cu/.cpp under csrc/ is compiled to an object in parallel, then linked
into one shared library.  Objects are rebuilt only when a source or header is
newer.  No CMake; one -gencode.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsymgpu.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (CUDA toolkit required to build libsymgpu)")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


# The bounds-checked library (every gather / scatter index of the hot-path kernels checked, violations counted):
# the sources it needs, compiled with -DSYM_BOUNDS_CHECK into a build folder of its own.
LIB_BC = os.path.join(PKG, "libsymgpu_bc.so")
BUILD_BC = os.path.join(PKG, "_build_bc")
BC_SOURCES = ("common.cu", "sort.cu", "tensor.cu", "mttkrp.cu", "mttkrp_n2.cu", "mttkrp_n3.cu", "mttkrp_n4.cu",
              "mttkrp_n5.cu", "spmv.cu", "spmv_cluster.cu", "spmv_band.cu", "spmv_batch.cu", "cpals.cu")


def _compile(src: str, extra, build_dir: str = BUILD) -> str:
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    newest_dep = max([os.path.getmtime(src)] + [os.path.getmtime(h) for h in _headers()])
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest_dep:
        return obj
    cmd = [nvcc()] + ARCH + NVCC_FLAGS + list(extra) + ["-c", src, "-o", obj + ".tmp"]
    if src.endswith(".cpp"):
        cmd = [nvcc()] + ARCH + NVCC_FLAGS + list(extra) + ["-x", "cu", "-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    if r.stderr.strip():
        sys.stderr.write(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, jobs: int | None = None, extra=(), bounds_check: bool = False) -> str:
    build_dir, lib = (BUILD_BC, LIB_BC) if bounds_check else (BUILD, LIB)
    os.makedirs(build_dir, exist_ok=True)
    srcs = _sources()
    if bounds_check:
        srcs = [s for s in srcs if os.path.basename(s) in BC_SOURCES]
        extra = tuple(extra) + ("-DSYM_BOUNDS_CHECK",)
    if force:
        for f in glob.glob(os.path.join(build_dir, "*.o")):
            os.remove(f)
    jobs = jobs or min(len(srcs), max(2, os.cpu_count() or 2))
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, build_dir), srcs))
    newest = max(os.path.getmtime(o) for o in objs)
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < newest:
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, bounds_check="--bounds-check" in sys.argv))
