"""Build libpilot.so (every CUDA source under csrc/) in-tree for sm_103a.

Each source compiles to its own object under _build/ (in parallel), then one
link makes the shared library."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpilot.so")
CHECKED_LIB = os.path.join(HERE, "libpilot_checked.so")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
OBJ_DIR = os.path.join(HERE, "_build")

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-lineinfo",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "--expt-relaxed-constexpr"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Build libpilot.so, or with ``checked`` libpilot_checked.so: every graph
    index is range-tested before it addresses a row and an out-of-range one
    is counted (status word 6) and skipped instead of being dereferenced.
    Select it for the binding with PILOT_LIBRARY=<path>."""
    lib = CHECKED_LIB if checked else LIB
    if not force and not _stale(lib):
        return lib
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    tag = f"{'checked' if checked else 'plain'}.{os.getpid()}"
    os.makedirs(OBJ_DIR, exist_ok=True)
    extra = ["-DPILOT_CHECKED"] if checked else []
    jobs, objs = [], []
    for src in sources():
        obj = os.path.join(OBJ_DIR, os.path.basename(src)[:-3] + f".{tag}.o")
        cmd = [nvcc, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-c", "-o", obj, src]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        jobs.append((src, subprocess.Popen(cmd)))
        objs.append(obj)
    failed = [src for src, p in jobs if p.wait() != 0]
    try:
        if failed:
            raise RuntimeError(f"nvcc failed on {', '.join(os.path.basename(f) for f in failed)}")
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp, *objs],
                       check=True)
        os.replace(tmp, lib)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
