"""Build ``libfdbb.so`` (the CUDA kernels and the C ABI) in-tree for sm_103a.

Each ``csrc/*.cu`` translation unit is compiled by ``nvcc`` in parallel into
``_build/``, then linked into ``paper_1809_09851_gb300/libfdbb.so`` with the
CUDA runtime linked statically and every symbol except the ``fdbb_*`` C ABI
hidden.  The build is skipped when the library is newer than every source.
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
BUILD = os.path.join(PKG, "_build")
LIBRARY = os.path.join(PKG, "libfdbb.so")
# The debug build (-DFDBB_DEBUG): every kernel checks its indices before each
# access and records violations (fdbb_debug_index_faults); slower, for testing.
BUILD_DEBUG = os.path.join(PKG, "_build_debug")
LIBRARY_DEBUG = os.path.join(PKG, "libfdbb_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden",
                     "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfdbb.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)])


def up_to_date(debug: bool = False) -> bool:
    lib = LIBRARY_DEBUG if debug else LIBRARY
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, debug: bool = False) -> str:
    """Compile and link libfdbb.so (debug=True: libfdbb_debug.so, with the
    kernels' index checks); returns its path."""
    if not force and up_to_date(debug):
        return LIBRARY_DEBUG if debug else LIBRARY
    nvcc = _nvcc()
    bdir = BUILD_DEBUG if debug else BUILD
    target = LIBRARY_DEBUG if debug else LIBRARY
    os.makedirs(bdir, exist_ok=True)
    srcs = _sources()
    extra = (["-Xptxas", "-v"] if ptxas_info else []) + (["-DFDBB_DEBUG=1"] if debug else [])

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    workers = max(1, min(len(srcs), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose or ptxas_info:
        for obj, log in results:
            if log:
                print(log, file=sys.stderr)
    objs = [o for o, _ in results]
    tmp = target + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-Xlinker", "--exclude-libs,ALL", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, target)
    return target


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                debug="--debug" in sys.argv))
