"""Compile librsi.so (the CUDA library behind include/rsi.h) in-tree.

nvcc compiles each translation unit of csrc/ for sm_103a in parallel and links
them into paper_2209_02878_gb300/librsi.so (static CUDA runtime).  Objects go
to paper_2209_02878_gb300/_build/.  Nothing here runs on the GPU.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "librsi.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librsi")


def _sources(src_dir=None):
    return sorted(glob.glob(os.path.join(src_dir or CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh")) +
            glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h")) +
            [os.path.abspath(__file__)])


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra=(), out: str | None = None,
          objdir: str | None = None, src_dir: str | None = None) -> str:
    """Build librsi.so if any source is newer; return its path.  `extra`
    adds nvcc flags; `out` / `objdir` / `src_dir` build a variant elsewhere."""
    lib = out or LIB
    objs_dir = objdir or BUILD
    if not force and out is None and up_to_date():
        return LIB
    os.makedirs(objs_dir, exist_ok=True)
    cc = nvcc()
    srcs = _sources(src_dir)

    def compile_one(src):
        obj = os.path.join(objs_dir, os.path.basename(src)[:-3] + ".o")
        inc = ["-I" + src_dir] if src_dir else []
        cmd = [cc, "-c", src, "-o", obj] + ARCH + inc + FLAGS + list(extra)
        if verbose:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose:
        for _, log in results:
            print(log)
    tmp = lib + ".tmp"
    cmd = [cc, "-shared", "-o", tmp] + ARCH + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
