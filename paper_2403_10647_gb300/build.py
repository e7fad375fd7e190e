"""Compiles the CUDA grid library (``_build/libgrid.so``) for sm_103a.

Two translation units (kernels, host runtime) are compiled in parallel with
nvcc and linked into one shared library exporting the C ABI of
``include/grid.h``.  Floating-point contraction is off in both device and
host code so the world-to-grid mapping rounds each operation separately.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
REPO_DIR = os.path.dirname(PKG_DIR)
CSRC = os.path.join(PKG_DIR, "csrc")
INCLUDE = os.path.join(REPO_DIR, "include")
BUILD_DIR = os.path.join(PKG_DIR, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libgrid.so")

SOURCES = ["kernels.cu", "runtime.cu", "noalloc.cu", "serve.cu", "sorted_grid.cu"]
HEADERS = ["device.cuh", "kernels.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the grid library")


def _flags(verbose_ptxas: bool) -> list[str]:
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC",
                "-Xcompiler", "-ffp-contract=off", "-I", INCLUDE, "-I", CSRC]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _inputs() -> list[str]:
    return ([os.path.join(CSRC, s) for s in SOURCES] + [os.path.join(CSRC, h) for h in HEADERS]
            + [os.path.join(INCLUDE, "grid.h"), os.path.abspath(__file__)])


def up_to_date() -> bool:
    if not os.path.exists(LIB_PATH):
        return False
    t = os.path.getmtime(LIB_PATH)
    return all(os.path.getmtime(p) <= t for p in _inputs())


def build_library(force: bool = False, verbose_ptxas: bool = False, out: str | None = None,
                  defines: tuple = ()) -> str:
    """Builds the library (into ``out`` if given, with extra -D ``defines``)."""
    if out is None and not defines and not force and up_to_date():
        return LIB_PATH
    target = out or LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    cc = nvcc()
    pid = os.getpid()

    def compile_one(src: str) -> tuple[str, str]:
        tag = abs(hash((target, defines))) % 10**8
        obj = os.path.join(BUILD_DIR, f"{os.path.splitext(src)[0]}.{pid}.{tag}.o")
        cmd = [cc] + _flags(verbose_ptxas) + [f"-D{d}" for d in defines] + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    tag = abs(hash((target, defines))) % 10**8
    objs = [os.path.join(BUILD_DIR, f"{os.path.splitext(src)[0]}.{pid}.{tag}.o") for src in SOURCES]
    try:
        with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
            results = list(ex.map(compile_one, SOURCES))
        if verbose_ptxas:
            for _, log in results:
                print(log)
        tmp = target + f".tmp{pid}"
        cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, target)
    finally:
        for o in objs:   # the objects of a failed build too
            try:
                os.remove(o)
            except OSError:
                pass
    return target


if __name__ == "__main__":
    import sys
    print(build_library(force=True, verbose_ptxas="-v" in sys.argv))
