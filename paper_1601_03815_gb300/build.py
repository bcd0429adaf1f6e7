"""Build libkin.so in-tree for sm_103a (GB300) with nvcc.

Each .cu file under csrc/ is compiled in parallel, then linked with cuFFT into
paper_1601_03815_gb300/libkin.so, and a second time with -DKIN_DEBUG into
libkin_debug.so (the stencil kernels check their indices and record the first
failure instead of trapping; see csrc/kin_debug.cuh).  Rebuilds only what is
older than its sources.  Usage: ``python -m paper_1601_03815_gb300.build [--force]``.
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
OBJDIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libkin.so")
DEBUG_OBJDIR = os.path.join(PKG, "_build_debug")
DEBUG_LIB = os.path.join(PKG, "libkin_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
              "-I", INCLUDE, "-I", CSRC] + ARCH


def nvcc() -> str:
    path = shutil.which("nvcc")
    if path:
        return path
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libkin")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)])


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def _compile(src: str, objdir: str, extra: list[str]) -> str:
    obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc(), "-c", src, "-o", obj] + NVCC_FLAGS + extra
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    return obj


def _link(objs: list[str], lib: str) -> None:
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-lcufft", "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None, debug: bool = True) -> str:
    """Compile every csrc/*.cu for sm_103a and link libkin.so (and, with
    debug, libkin_debug.so), the translation units of both in one parallel
    pool; returns the path of libkin.so."""
    extra = list(extra or [])
    targets = [(LIB, OBJDIR, extra)]
    if debug:
        targets.append((DEBUG_LIB, DEBUG_OBJDIR, extra + ["-DKIN_DEBUG"]))
    targets = [t for t in targets if force or not up_to_date(t[0])]
    if not targets:
        return LIB
    srcs = _sources()
    jobs = []
    for lib, objdir, flags in targets:
        os.makedirs(objdir, exist_ok=True)
        jobs += [(lib, src, objdir, flags) for src in srcs]
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda j: (j[0], _compile(j[1], j[2], j[3])), jobs))
    for lib, _, _ in targets:
        _link([o for l, o in objs if l == lib], lib)
        if verbose:
            print("built", lib)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else None)
