"""Builds libbfly.so (the C-ABI library) in-tree with nvcc for sm_103a.

    python -m paper_1502_01379_gb300.build          # build if stale
    python -m paper_1502_01379_gb300.build --force  # rebuild
    python -m paper_1502_01379_gb300.build --checked  # the bounds-checked variant
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libbfly.so")
CHECKED_DIR = os.path.join(OUT_DIR, "checked")
CHECKED_LIB = os.path.join(CHECKED_DIR, "libbfly_checked.so")
SOURCES = [os.path.join(CSRC, n) for n in ("bf_capi.cu", "bf_diff.cu", "bf_quad.cu", "bf_sketch.cu", "bf_file.cu")]
DEPS = SOURCES + [os.path.join(CSRC, n) for n in sorted(os.listdir(CSRC)) if n.endswith(".cuh")] + [
    os.path.join(INCLUDE, "bfly.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (set NVCC or put the CUDA toolkit on PATH)")


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in DEPS)


def _run(cmd: list, verbose: bool) -> None:
    if verbose:
        print(" ".join(cmd), flush=True)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + res.stdout + res.stderr)
    if verbose:
        print(res.stdout + res.stderr)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile the library if it is missing or older than its sources; return
    its path.  The translation units compile in parallel, then link.
    ``checked``: the BF_CHECKED variant (bounds-checked kernels, see
    include/bfly.h: bf_plan_check), built into its own directory."""
    lib, out_dir = (CHECKED_LIB, CHECKED_DIR) if checked else (LIB, OUT_DIR)
    if not force and not stale(lib):
        return lib
    from concurrent.futures import ThreadPoolExecutor
    os.makedirs(out_dir, exist_ok=True)
    flags = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    if checked:
        flags.append("-DBF_CHECKED=1")
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    objs = [os.path.join(out_dir, os.path.basename(src)[:-3] + ".o") for src in SOURCES]
    with ThreadPoolExecutor(len(SOURCES)) as ex:
        list(ex.map(lambda so: _run([nvcc(), *flags, "-c", so[0], "-o", so[1]], verbose), zip(SOURCES, objs)))
    tmp = lib + ".tmp"
    _run([nvcc(), "-shared", *ARCH, *objs, "-o", tmp], verbose)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
