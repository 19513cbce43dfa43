"""Builds the sm_103a shared library ``libgaussianpile.so`` in-tree with nvcc.

Every ``csrc/*.cu`` / ``csrc/*.cpp`` file is compiled to an object under
``_build/`` (in parallel, only when its sources changed) and linked into
``paper_2603_20611_b300/libgaussianpile.so``.  nvcc cross-compiles for
``sm_103a`` without a GPU.  Run ``python -m paper_2603_20611_b300.build``.

``build(check=True)`` builds the bounds-checked debug variant
``libgaussianpile_check.so`` (objects under ``_build_check/``, ``-DGP_CHECK``):
the kernels check their shared- and global-memory indices, skip an
out-of-range access and record it, and every render / backward / batch call
waits for its stream and returns GP_ERR_STATE naming the failed check.  The
binding loads it when the environment sets ``GP_LIBRARY=check``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libgaussianpile.so")
BUILD_CHECK = os.path.join(ROOT, "_build_check")
LIB_CHECK = os.path.join(PKG, "libgaussianpile_check.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
           "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) +
                  glob.glob(os.path.join(INCLUDE, "*.h")))


def _digest(src, extra):
    h = hashlib.sha256()
    for p in [src] + _headers():
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(extra).encode())
    return h.hexdigest()[:16]


def _compile(src, extra, build_dir=BUILD):
    base = os.path.splitext(os.path.basename(src))[0]
    obj = os.path.join(build_dir, f"{base}.o")
    stamp = obj + ".hash"
    dig = _digest(src, extra)
    if os.path.exists(obj) and os.path.exists(stamp) and open(stamp).read() == dig:
        return obj
    cmd = [NVCC] + ARCH + CUFLAGS + extra + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
    with open(stamp, "w") as f:
        f.write(dig)
    return obj


def build(verbose: bool = False, extra=(), check: bool = False) -> str:
    build_dir, lib = (BUILD_CHECK, LIB_CHECK) if check else (BUILD, LIB)
    os.makedirs(build_dir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    extra = list(extra) + (["-DGP_CHECK"] if check else [])
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, build_dir), srcs))
    newest = max(os.path.getmtime(o) for o in objs)
    if not os.path.exists(lib) or os.path.getmtime(lib) < newest:
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    if verbose:
        print(lib)
    return lib


if __name__ == "__main__":
    args = [a for a in sys.argv[1:] if a != "--check"]
    build(verbose=True, extra=args, check="--check" in sys.argv[1:])
