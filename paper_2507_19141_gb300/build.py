"""Builds libdash.so in-tree from csrc/*.cu for sm_103a (GB300).

Each translation unit is compiled by its own nvcc process, in parallel, then
linked into paper_2507_19141_gb300/_build/libdash.so.  No cmake, no torch
extension machinery: the library has a plain C ABI (include/dash.h).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC_DIR = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libdash.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdash")


def _sources():
    return sorted(glob.glob(os.path.join(SRC_DIR, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(SRC_DIR, "*.cuh")) + [os.path.join(ROOT, "include", "dash.h")]


DEBUG_DIR = os.path.join(HERE, "_build_debug")
DEBUG_LIB = os.path.join(DEBUG_DIR, "libdash_debug.so")


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def _build_variant(out_dir: str, lib: str, extra: list, verbose: bool, ex) -> list:
    """Compiles every source into out_dir (through the shared executor) and
    returns a callable that links them into lib."""
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                     "-I" + os.path.join(ROOT, "include"), "-I" + SRC_DIR] + extra
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [cc] + common + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    return [ex.submit(compile_one, src) for src in _sources()]


def _link(lib: str, futures) -> None:
    objs = [f.result() for f in futures]
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False, debug: bool = True) -> str:
    """Builds libdash.so and, with `debug`, the bounds-checked variant
    libdash_debug.so (-DDASH_DEBUG: every point-row index is checked before
    it is used), compiling both sets of translation units in parallel."""
    todo = []
    if force or not up_to_date(LIB):
        todo.append((OUT_DIR, LIB, []))
    if debug and (force or not up_to_date(DEBUG_LIB)):
        todo.append((DEBUG_DIR, DEBUG_LIB, ["-DDASH_DEBUG"]))
    if not todo:
        return LIB
    workers = max(1, min(len(_sources()) * len(todo), os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        jobs = [(lib, _build_variant(d, lib, extra, verbose, ex)) for d, lib, extra in todo]
        for lib, futures in jobs:
            _link(lib, futures)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
