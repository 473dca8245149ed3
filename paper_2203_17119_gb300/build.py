"""Build the CUDA library ``libdwf.so`` in-tree for sm_103a.

Each ``csrc/*.cu`` translation unit is compiled in parallel with nvcc into
``_build/`` and linked into ``_build/libdwf.so`` (static CUDA runtime).  A
unit is rebuilt only when it or one of the headers is newer than its object.

    python -m paper_2203_17119_gb300.build [-v] [--ptxas]
"""

from __future__ import annotations

import argparse
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
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libdwf.so")
# the debug build (-DDWF_DEBUG): host-side bounds checks of every caller buffer
# and of the handle's tables in the entry points (csrc/debug.cu)
OUT_DEBUG = os.path.join(PKG, "_build_debug")
LIB_DEBUG = os.path.join(OUT_DEBUG, "libdwf_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (CUDA toolkit required to build libdwf.so)")


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(src: str, obj: str, newest_header: float) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return os.path.getmtime(src) > t or newest_header > t


def build(verbose: bool = False, ptxas: bool = False, jobs: int | None = None, debug: bool = False) -> str:
    """Compile every translation unit and link the library; returns its path.
    ``debug``: the DWF_DEBUG variant (``_build_debug/libdwf_debug.so``)."""
    out_dir, lib = (OUT_DEBUG, LIB_DEBUG) if debug else (OUT, LIB)
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    newest = max((os.path.getmtime(f) for f in _headers()), default=0.0)
    extra = (["-Xptxas", "-v"] if ptxas else []) + (["-DDWF_DEBUG"] if debug else [])

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        if not ptxas and not _stale(src, obj, newest):
            return obj, ""
        cmd = [cc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stdout + r.stderr

    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(compile_one, srcs))
    objs = [o for o, _ in results]
    if verbose or ptxas:
        for _, log in results:
            if log:
                print(log, file=sys.stderr)
    need_link = not os.path.exists(lib) or any(
        os.path.getmtime(o) > os.path.getmtime(lib) for o in objs)
    if need_link:
        cmd = [cc, *ARCH, "-shared", "-o", lib, *objs, "-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return lib


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("-v", action="store_true")
    ap.add_argument("--ptxas", action="store_true", help="print -Xptxas -v register/smem usage")
    ap.add_argument("--debug", action="store_true", help="the DWF_DEBUG library (bounds checks)")
    a = ap.parse_args()
    print(build(verbose=a.v, ptxas=a.ptxas, debug=a.debug))
