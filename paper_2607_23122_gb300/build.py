"""Builds liboccreuse.so (the C-ABI library of include/*.h) in-tree with nvcc.

One -gencode for sm_103a, translation units compiled in parallel, static cudart.
Rebuilds only when a source or header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "liboccreuse.so")
# Library variants: "" is the product library; "counters" is the instrumented build whose
# traversal counts node visits, triangle tests and the distinct nodes and triangles it
# touched (occ_debug_bvh_counters), used to measure the bytes a trace launch must read.
VARIANTS = {"": [], "counters": ["-DOCC_COUNTERS=1"]}

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden,-O3",
         "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) \
        + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]


def lib_path(variant: str = "") -> str:
    if variant not in VARIANTS:
        raise ValueError(f"unknown library variant {variant!r} (known: {sorted(VARIANTS)})")
    return LIB if not variant else os.path.join(OUT_DIR, f"liboccreuse_{variant}.so")


def up_to_date(variant: str = "") -> bool:
    lib = lib_path(variant)
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra=None, variant: str = "") -> str:
    """Compiles the library (or one of VARIANTS).  OCC_NVCC_EXTRA (environment) appends nvcc
    flags, e.g. a tuning define such as -DOCC_TRACE_MIN_BLOCKS=10; set it with force=True."""
    lib = lib_path(variant)
    if not force and up_to_date(variant):
        return lib
    obj_dir = OUT_DIR if not variant else os.path.join(OUT_DIR, variant)
    os.makedirs(obj_dir, exist_ok=True)
    cc = nvcc()
    extra = list(extra or []) + VARIANTS[variant] + os.environ.get("OCC_NVCC_EXTRA", "").split()

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        if src.endswith(".cpp"):
            cmd = [cc, *FLAGS, *extra, "-x", "c++", "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"], capture_output=True,
                       text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    var = next((a.split("=", 1)[1] for a in sys.argv if a.startswith("--variant=")), "")
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None, variant=var))
