"""Build libmg.so (CUDA kernels + C ABI) in-tree for sm_103a, and beside it
libmg_cpu.so (the SIMD CPU build of the same program, host compiler).

One nvcc invocation per translation unit, run in parallel, then a shared-
library link.  Rebuilds only when a source or header is newer than the
library.  ``MG_PTXAS_VERBOSE=1`` adds ``-Xptxas -v`` (registers, spills);
``MG_NVCC_DEFINES`` adds preprocessor definitions (tuning knobs such as
``-DMG_HS_NT=256``).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", CSRC, "-I", INCLUDE]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _deps():
    files = glob.glob(os.path.join(CSRC, "**", "*.cu"), recursive=True)
    files += glob.glob(os.path.join(CSRC, "**", "*.cuh"), recursive=True)
    files += glob.glob(os.path.join(CSRC, "**", "*.h"), recursive=True)
    files += glob.glob(os.path.join(INCLUDE, "*.h"))
    return files


CPU_SRC = os.path.join(HERE, "cpu", "mg_cpu.cpp")
CPU_LIB = os.path.join(BUILD, "libmg_cpu.so")


def cuda_include() -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc()))), "include")


def build_cpu(force: bool = False) -> str:
    """The SIMD CPU build (cpu/mg_cpu.cpp) with the host C++ compiler: no
    target-specific flags, FMA contraction where the target has it."""
    deps = _deps() + [CPU_SRC]
    if not force and os.path.exists(CPU_LIB) and all(os.path.getmtime(f) <= os.path.getmtime(CPU_LIB) for f in deps):
        return CPU_LIB
    os.makedirs(BUILD, exist_ok=True)
    cxx = os.environ.get("CXX") or shutil.which("g++") or "c++"
    tmp = CPU_LIB + ".%d.tmp" % os.getpid()
    cmd = [cxx, "-std=c++17", "-O3", "-ffp-contract=fast", "-Wno-psabi", "-fPIC", "-shared", "-pthread", "-I", CSRC, "-I",
           INCLUDE, "-I", cuda_include(), CPU_SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("host compiler failed for %s:\n%s" % (CPU_SRC, r.stderr))
    os.replace(tmp, CPU_LIB)
    return CPU_LIB


def is_stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not is_stale():
        build_cpu()
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    # the largest translation units (the many-leg processes) first, so the
    # parallel compile ends with the small ones
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")),
                  key=lambda f: (-max([int(c) for c in os.path.basename(f) if c.isdigit()] or [0]), f))
    extra = ["-Xptxas", "-v"] if os.environ.get("MG_PTXAS_VERBOSE") else []
    extra += os.environ.get("MG_NVCC_DEFINES", "").split()  # e.g. -DMG_HS_NT=256 (tuning)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stderr))
        return obj, r.stderr

    jobs = min(len(srcs) + 1, os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        cpu = ex.submit(build_cpu, True)  # the host build alongside the CUDA translation units
        results = list(ex.map(compile_one, srcs))
        cpu.result()
    if verbose or extra:
        for obj, err in results:
            if err.strip():
                print("==", os.path.basename(obj))
                print(err)
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
