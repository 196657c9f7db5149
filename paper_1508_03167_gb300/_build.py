"""Builds libmergeshuffle.so (the CUDA kernels and the C ABI) in-tree for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked into one shared library under
``paper_1508_03167_gb300/_build/``. The CUDA runtime is linked statically, so the library only
needs the driver at run time.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_NAME = "libmergeshuffle.so"
LIB_PATH = os.path.join(BUILD_DIR, LIB_NAME)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["ms_api.cu", "ms_leaf.cu", "ms_level.cu", "ms_static.cu", "ms_batch.cu", "ms_wlevel.cu",
           "ms_tune.cu", "ms_span.cu", "ms_tile.cu", "ms_bits.cu", "ms_rs.cu", "ms_narrow.cu"]

_lock = threading.Lock()


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmergeshuffle")


def _inputs() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)
             if f.endswith((".cu", ".cuh", ".h"))]
    files.append(os.path.join(INCLUDE, "mergeshuffle.h"))
    return files


def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None) -> str:
    """Compile every CUDA source and link the shared library; returns its path."""
    with _lock:
        if not force and not _stale():
            return LIB_PATH
        os.makedirs(BUILD_DIR, exist_ok=True)
        nvcc = nvcc_path()
        common = ["-O3", "-lineinfo", "-std=c++17", *ARCH, "-Xcompiler", "-fPIC",
                  "-I", INCLUDE, "-I", CSRC, *(extra_flags or [])]
        objs = []

        def compile_one(src: str) -> str:
            obj = os.path.join(BUILD_DIR, os.path.splitext(src)[0] + ".o")
            cmd = [nvcc, *common, "-c", os.path.join(CSRC, src), "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
            if verbose and (r.stdout or r.stderr):
                print(r.stdout, r.stderr)
            return obj

        with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
            objs = list(ex.map(compile_one, SOURCES))
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB_PATH)
        return LIB_PATH


if __name__ == "__main__":
    print(build(force=True, verbose=True))
