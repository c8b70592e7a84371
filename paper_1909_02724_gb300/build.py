"""Builds the ifdk C-ABI library (``lib/libifdk.so``) and the input generator
(``lib/libifdk_phantom.so``) in-tree with nvcc for sm_103a.

Translation units compile in parallel; the CUDA runtime is linked statically
into each shared object, so the libraries depend only on the driver.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "lib")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(LIBDIR, "libifdk.so")
CHECK_LIB = os.path.join(LIBDIR, "libifdk_check.so")   # the checked build (IFDK_CHECK)
PHANTOM_LIB = os.path.join(LIBDIR, "libifdk_phantom.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
           "--expt-relaxed-constexpr", f"-I{INCLUDE}", f"-I{CSRC}"]
LIB_SOURCES = ["ifdk_plan.cu", "ifdk_bp.cu", "ifdk_bp_packed.cu", "ifdk_filter.cu", "ifdk_filter_tc.cu", "ifdk_filter_static.cu",
               "ifdk_rates.cu", "ifdk_iter.cu",
               "ifdk_project.cu", "ifdk_stream.cu", "ifdk_volume.cu"]
PHANTOM_SOURCES = [os.path.join(PKG, "phantom", "phantom.cu")]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the ifdk CUDA library cannot be built")
    return exe


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _headers() -> list[str]:
    hs = [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    hs += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return hs


def _compile(src: str, obj: str, extra: list[str]) -> None:
    cmd = [nvcc(), *ARCH, *NVFLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stderr}")


def _link(objs: list[str], out: str) -> None:
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed for {os.path.basename(out)}:\n{r.stderr}")
    os.replace(tmp, out)


def build_checked(force: bool = False) -> str:
    """The library compiled with -DIFDK_CHECK (window-bounds checks on every tap read
    of the packed back-projector; a miss sets the plan's status to IFDK_ERR_BOUNDS),
    for tests.  Its objects sit beside the normal ones with a _check suffix."""
    os.makedirs(LIBDIR, exist_ok=True)
    headers = _headers()
    objs, jobs = [], []
    for s in LIB_SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(LIBDIR, s.replace(".cu", "_check.o"))
        objs.append(obj)
        if force or _stale(obj, [src, *headers]):
            jobs.append((src, obj))
    if jobs:
        with ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
            for f in [ex.submit(_compile, s, o, ["-DIFDK_CHECK"]) for s, o in jobs]:
                f.result()
    if force or _stale(CHECK_LIB, objs):
        _link(objs, CHECK_LIB)
    return CHECK_LIB


def build(force: bool = False, verbose_ptxas: bool = False) -> list[str]:
    """Compiles whatever is stale; returns the library paths."""
    os.makedirs(LIBDIR, exist_ok=True)
    headers = _headers()
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    jobs = []
    lib_objs = []
    for s in LIB_SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(LIBDIR, s.replace(".cu", ".o"))
        lib_objs.append(obj)
        if force or _stale(obj, [src, *headers]):
            jobs.append((src, obj))
    ph_objs = []
    for src in PHANTOM_SOURCES:
        obj = os.path.join(LIBDIR, "phantom.o")
        ph_objs.append(obj)
        if force or _stale(obj, [src, *headers]):
            jobs.append((src, obj))
    if jobs:
        with ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
            for f in [ex.submit(_compile, s, o, extra) for s, o in jobs]:
                f.result()
    if force or _stale(LIB, lib_objs):
        _link(lib_objs, LIB)
    if force or _stale(PHANTOM_LIB, ph_objs):
        _link(ph_objs, PHANTOM_LIB)
    return [LIB, PHANTOM_LIB]


if __name__ == "__main__":
    import sys
    for p in build(force="--force" in sys.argv, verbose_ptxas="--ptxas" in sys.argv):
        print(p)
