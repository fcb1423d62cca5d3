"""In-tree build of libkmedoids.so for sm_103a (nvcc, no cmake).

Each CUDA translation unit is compiled in parallel to an object file under
``_build/`` and the objects are linked into ``libkmedoids.so`` next to this
file.  Objects are rebuilt only when a source or header is newer.

``build(bounds_check=True)`` (or ``python -m paper_2008_05171_gb300.build
--bounds-check``) makes the bounds-checking variant ``libkmedoids_bounds.so``
from ``_build_bounds/`` with ``-DKM_BOUNDS_CHECK``: its kernels check every
index they load from memory and report KM_E_BOUNDS instead of reading or
writing out of range.  The Python binding loads it when the environment sets
``KMEDOIDS_BOUNDS_CHECK=1``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libkmedoids.so")
BUILD_BOUNDS = os.path.join(HERE, "_build_bounds")
LIB_BOUNDS = os.path.join(HERE, "libkmedoids_bounds.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-O2", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for p in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if p and (os.path.sep not in p or os.path.exists(p)):
            return p
    return "nvcc"


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers() -> list[str]:
    return (glob.glob(os.path.join(CSRC, "*.h")) +
            glob.glob(os.path.join(CSRC, "*.cuh")) +
            glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, extra: list[str], outdir: str = BUILD) -> str:
    obj = os.path.join(outdir, os.path.basename(src)[:-3] + ".o")
    if _stale(obj, [src] + _headers()):
        cmd = [_nvcc()] + ARCH + NVCC_FLAGS + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" %
                               (src, " ".join(cmd), r.stderr[-6000:]))
    return obj


def build(force: bool = False, verbose: bool = False,
          extra: list[str] | None = None, bounds_check: bool = False) -> str:
    """Compile every kernel translation unit and link libkmedoids.so (the
    bounds-checking variant libkmedoids_bounds.so with bounds_check)."""
    outdir, lib = (BUILD_BOUNDS, LIB_BOUNDS) if bounds_check else (BUILD, LIB)
    os.makedirs(outdir, exist_ok=True)
    extra = list(extra or []) + (["-DKM_BOUNDS_CHECK"] if bounds_check else [])
    if force:
        for f in glob.glob(os.path.join(outdir, "*.o")):
            os.remove(f)
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs),
                                                      os.cpu_count() or 1))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, outdir), srcs))
    if _stale(lib, objs):
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s" % r.stderr[-4000:])
        os.replace(tmp, lib)
    if verbose:
        print("built", lib)
    return lib


if __name__ == "__main__":
    import sys
    build(verbose=True, bounds_check="--bounds-check" in sys.argv[1:])
