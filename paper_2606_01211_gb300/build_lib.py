"""Build liblwe.so (the C-ABI library of include/lwe.h) for sm_103a, in-tree.

Each CUDA translation unit is compiled in parallel with nvcc
(-gencode arch=compute_103a,code=sm_103a) and linked into
paper_2606_01211_gb300/liblwe.so against the shared CUDA runtime; the
bounds-checked debug variant (-DLWE_CHECK_BOUNDS) goes to liblwe_check.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "liblwe.so")
LIB_CHECK = os.path.join(PKG, "liblwe_check.so")
UNITS = ["kem_kernels.cu", "gemm_tc.cu", "lwe_api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblwe.so")


def _inputs():
    files = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))
             if f.endswith((".cu", ".cuh", ".h"))]
    inc = os.path.join(ROOT, "include")
    files += [os.path.join(inc, f) for f in sorted(os.listdir(inc)) if f.endswith(".h")]
    files.append(os.path.abspath(__file__))
    return files


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, check_bounds: bool = False) -> str:
    """liblwe.so, or with check_bounds the debug library liblwe_check.so
    whose kernels skip and count out-of-bounds accesses (LWE_CHECK_BOUNDS)."""
    lib = LIB_CHECK if check_bounds else LIB
    if not force and up_to_date(lib):
        return lib
    bdir = os.path.join(BUILD, "check") if check_bounds else BUILD
    os.makedirs(bdir, exist_ok=True)
    nv = nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-I", os.path.join(ROOT, "include")]
    if check_bounds:
        flags.append("-DLWE_CHECK_BOUNDS")

    def compile_unit(unit):
        src = os.path.join(CSRC, unit)
        obj = os.path.join(bdir, unit.replace(".cu", ".o"))
        cmd = [nv] + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (unit, r.stdout, r.stderr))
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = [nv] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
