"""Build the engine's shared library (libara_b300.so) in-tree with nvcc for sm_103a.

Usage: ``python paper_1412_4556_b300/build.py [--force] [-v]``.  This file is
run (or loaded by path) without importing the package, whose import needs the
built library.  The library exports the C ABI declared in ``include/ara.h``.
"""
from __future__ import annotations

import concurrent.futures
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libara_b300.so")
SOURCES = ["ara_api.cu", "fold.cu", "ylt.cu", "select.cu", "validate.cu", "noalloc.cu", "service.cu", "yelt.cu", "plan.cu", "ingest.cu", "compact.cu", "tail.cu", "probe.cu"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-fvisibility=hidden", "-I", INCLUDE, "-I", CSRC]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "ara.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every CUDA source and link libara_b300.so (skipped when up to date)."""
    if not force and not _stale():
        return LIB
    objdir = os.path.join(PKG, "_build")
    os.makedirs(objdir, exist_ok=True)
    objs = [os.path.join(objdir, src.replace(".cu", ".o")) for src in SOURCES]

    def compile_one(src_obj):
        src, obj = src_obj
        subprocess.check_call([NVCC, *ARCH, *FLAGS, "-Xptxas", "-v" if verbose else "-O3", "-c",
                               os.path.join(CSRC, src), "-o", obj])

    # the translation units are independent: compile them side by side
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 1)) as ex:
        list(ex.map(compile_one, zip(SOURCES, objs)))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt",
                           "-lpthread", "-ldl"])
    os.replace(tmp, LIB)
    return LIB



if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
