"""Build libslos.so (the CUDA library behind include/slos.h) in-tree.

Every translation unit under csrc/ is compiled for sm_103a in parallel and
linked into paper_2602_11092_gb300/libslos.so.  Rebuilds only when a source
is newer than the library.

build_debug() links libslos_debug.so: the same library with the device-side
bounds checks of SLOS_DEBUG compiled into the translation units that have
them (the others reuse the release objects).
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libslos.so")
DEBUG_LIB = os.path.join(HERE, "libslos_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xcompiler", "-Wno-unused-function"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def headers():
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in sources() + headers() + [__file__])


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    srcs = sources()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    workers = max(1, min(len(srcs), os.cpu_count() or 1))
    with ThreadPoolExecutor(workers) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-ldl", "-lrt", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def debug_sources():
    """Sources whose kernels carry SLOS_DEBUG bounds checks."""
    return [f for f in sources() if "SLOS_IDX(" in open(f).read()]


def build_debug(force: bool = False) -> str:
    build()
    t = os.path.getmtime(LIB)
    if not force and os.path.exists(DEBUG_LIB) and os.path.getmtime(DEBUG_LIB) >= t:
        return DEBUG_LIB
    cc = nvcc()
    dbg_dir = os.path.join(BUILD, "debug")
    os.makedirs(dbg_dir, exist_ok=True)
    dsrc = debug_sources()

    def compile_one(src):
        obj = os.path.join(dbg_dir, os.path.basename(src) + ".o")
        cmd = [cc, *ARCH, *FLAGS, "-DSLOS_DEBUG", "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj

    with ThreadPoolExecutor(max(1, len(dsrc))) as ex:
        dobjs = list(ex.map(compile_one, dsrc))
    names = {os.path.basename(f) for f in dsrc}
    objs = dobjs + [os.path.join(BUILD, os.path.basename(f) + ".o") for f in sources()
                    if os.path.basename(f) not in names]
    tmp = DEBUG_LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-ldl", "-lrt", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, DEBUG_LIB)
    return DEBUG_LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
