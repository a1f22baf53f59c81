"""Build libreallife.so in-tree with nvcc for sm_103a (GB300).

Each CUDA translation unit is compiled in parallel to ``_build/<machine>/`` and linked
into ``paper_2307_03017_gb300/libreallife.so`` (static CUDA runtime).  Rebuilds only
when a source or header is newer than the library, and then recompiles only the
translation units whose object is older than the unit or any header.

``build(debug=True)`` makes the bounds-checked variant ``libreallife_debug.so``
(``-DRL_DEBUG``, objects in ``_build/<machine>-debug/``), loaded instead of the release
library when the environment sets ``REALLIFE_DEBUG=1``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import platform
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libreallife.so")
LIB_DEBUG = os.path.join(HERE, "libreallife_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libreallife")


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers() -> list[str]:
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]


def _deps() -> list[str]:
    return sources() + _headers()


def up_to_date(debug: bool = False) -> bool:
    lib = LIB_DEBUG if debug else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None,
          debug: bool = False) -> str:
    """Compile and link the library (the debug variant with ``debug``) if needed; returns its path."""
    lib = LIB_DEBUG if debug else LIB
    if not force and up_to_date(debug):
        return lib
    exe = nvcc()
    objdir = os.path.join(HERE, "_build", platform.machine() + ("-debug" if debug else ""))
    os.makedirs(objdir, exist_ok=True)
    flags = NVCC_FLAGS + (["-DRL_DEBUG"] if debug else []) + (extra_flags or [])
    newest_header = max(os.path.getmtime(p) for p in _headers())

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        if not force and not extra_flags and os.path.exists(obj) and \
                os.path.getmtime(obj) >= max(os.path.getmtime(src), newest_header):
            return obj
        cmd = [exe] + ARCH + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [exe] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
