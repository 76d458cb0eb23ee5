"""Build ``libqcmet.so`` in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel into ``_build/``; the objects are
linked into ``paper_2004_09084_gb300/libqcmet.so`` with the CUDA runtime linked
statically, so the library depends only on the driver at run time.
"""
from __future__ import annotations

import concurrent.futures as cf
import fcntl
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libqcmet.so")
# the debug build: the same sources with every gathered / scattered index checked
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libqcmet_debug.so")
DEBUG_FLAGS = ["-DQCMET_DEBUG_CHECKS=1"]
INCLUDE = os.path.join(ROOT, "include")

SOURCES = ["layout.cpp", "api.cpp", "batch.cpp", "decode.cu", "decode_group.cu", "learned.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
          f"-I{INCLUDE}"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libqcmet.so")
    return exe


def _deps():
    paths = [os.path.join(CSRC, s) for s in SOURCES]
    paths += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    paths.append(os.path.join(INCLUDE, "qcmet.h"))
    return paths


def up_to_date(debug: bool = False) -> bool:
    lib = LIB_DEBUG if debug else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def _compile(src: str, extra, build_dir: str) -> str:
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    cmd = [nvcc(), *ARCH, *COMMON, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose_ptxas: bool = False, debug: bool = False) -> str:
    """Compile and link the library; returns its path.

    ``debug`` builds ``libqcmet_debug.so`` instead: the same sources with
    QCMET_DEBUG_CHECKS=1, whose kernels check every index they gather or
    scatter (``qcmet_debug_checks``).  Holds an exclusive lock on the build
    folder so that processes that start together (one per GPU) build once.
    """
    lib, folder = (LIB_DEBUG, BUILD_DEBUG) if debug else (LIB, BUILD)
    if not force and up_to_date(debug):
        return lib
    os.makedirs(folder, exist_ok=True)
    with open(os.path.join(folder, ".lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        if not force and up_to_date(debug):
            return lib
        return _build_locked(verbose_ptxas, debug)


def _build_locked(verbose_ptxas: bool, debug: bool = False) -> str:
    lib, folder = (LIB_DEBUG, BUILD_DEBUG) if debug else (LIB, BUILD)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    flags = DEBUG_FLAGS if debug else []
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(
            lambda s: _compile(s, flags + (extra if s.endswith(".cu") else []), folder), SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv,
                debug="--debug" in sys.argv))
