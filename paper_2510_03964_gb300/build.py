"""Builds libwrs.so in-tree with nvcc for sm_103a (GB300).

Each .cu file under csrc/ is compiled in parallel and linked into one shared
library with the CUDA runtime linked statically, so the library has no
dependency beyond the driver. Host code is built without floating-point
contraction; device code marks its exact steps with round-to-nearest
intrinsics. The same sources are also built with WRS_CHECKED into
libwrs_checked.so, whose kernels test every index and copy range against its
buffer (a debug library for tests; the package loads it when the environment
sets WRS_CHECKED=1).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libwrs.so")
LIB_CHECKED = os.path.join(OUT_DIR, "libwrs_checked.so")
VARIANTS = {LIB: ("", []), LIB_CHECKED: ("checked", ["-DWRS_CHECKED"])}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math", "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libwrs")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + sorted(
        glob.glob(os.path.join(CSRC, "*.h"))) + [os.path.join(INCLUDE, "wrs.h"), __file__]


def is_stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False,
          libs=(LIB, LIB_CHECKED)) -> str:
    """Builds the given libraries (default: both) from the sources; every
    translation unit of every library compiles in one parallel pool."""
    todo = [lib for lib in libs if force or is_stale(lib)]
    if not todo:
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_one(job):
        lib, src = job
        sub, defines = VARIANTS[lib]
        out = os.path.join(OUT_DIR, sub)
        os.makedirs(out, exist_ok=True)
        obj = os.path.join(out, os.path.basename(src).replace(".cu", ".o"))
        cmd = [cc, *ARCH, *NVCC_FLAGS, *defines, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}{' (' + sub + ')' if sub else ''}:\n{r.stderr}")
        return lib, obj, r.stderr

    jobs = [(lib, src) for lib in todo for src in _sources()]
    with cf.ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        results = list(ex.map(compile_one, jobs))
    if verbose or ptxas_info:
        for _, _, log in results:
            if log:
                print(log)
    for lib in todo:
        tmp = lib + f".{os.getpid()}.tmp"
        cmd = [cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp,
               *[o for l, o, _ in results if l == lib]]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose=True, ptxas_info="-v" in sys.argv))
