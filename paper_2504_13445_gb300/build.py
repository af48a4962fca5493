"""Build librkm.so in-tree: nvcc for sm_103a, one object per source, compiled in parallel.

build(debug=True) builds librkm_debug.so instead: the same sources with RKM_DEBUG defined,
which turns on the device index checks (a failed check sets the status word and the call
returns RKM_EINTERNAL).  Select it with the environment variable RKM_LIBRARY."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "lib")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "librkm.so")
LIB_DEBUG = os.path.join(OUT_DIR, "librkm_debug.so")
BUILD_DIR_DEBUG = os.path.join(HERE, "_build_debug")
SOURCES = ["api.cu", "prep.cu", "simt.cu", "exact.cu", "topn.cu", "tc.cu", "noalloc.cu", "serve.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
              "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(obj: str, deps: list[str]) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, extra_flags: list[str] | None = None, debug: bool = False) -> str:
    build_dir = BUILD_DIR_DEBUG if debug else BUILD_DIR
    lib = LIB_DEBUG if debug else LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(build_dir, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "rkm.h"))
    flags = NVCC_FLAGS + (["-DRKM_DEBUG"] if debug else []) + (extra_flags or [])
    cc = nvcc()

    def compile_one(src: str) -> str:
        path = os.path.join(CSRC, src)
        obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
        if _stale(obj, [path] + headers):
            cmd = [cc, *ARCH, *flags, "-c", path, "-o", obj]
            if verbose:
                print(" ".join(cmd), flush=True)
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
            if verbose and r.stderr.strip():
                print(r.stderr, flush=True)
        return obj

    with ThreadPoolExecutor(max(1, min(len(SOURCES), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    if _stale(lib, objs):
        cmd = [cc, *ARCH, "-shared", "-o", lib, *objs, "-ldl", "-lpthread", "-lrt"]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
