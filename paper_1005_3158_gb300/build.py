"""Build libfem.so in-tree for sm_103a (nvcc for the kernels, g++ for the host
side, compiled in parallel, linked by nvcc)."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libfem.so")
# the checked build: the same library with device-side bounds checks on every
# indexed shared/global access (FEM_CHECKED), for tests
LIB_CHECKED = os.path.join(PKG, "libfem_checked.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

SOURCES = {
    "fem_kernels.cu": "nvcc",
    "fem_io.cu": "nvcc",
    "fem_noalloc.cu": "nvcc",
    "fem_surrogate.cu": "nvcc",
    "fem_api.cpp": "g++",
    "fem_plan.cpp": "g++",
}


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "fem.h"))
    files.append(os.path.abspath(__file__))
    return files


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _deps())


def _compile(src: str, tool: str, verbose: bool, checked: bool = False) -> str:
    obj = os.path.join(BUILD, src + (".checked.o" if checked else ".o"))
    path = os.path.join(CSRC, src)
    inc = ["-I", INCLUDE, "-I", CSRC] + (["-DFEM_CHECKED"] if checked else [])
    if tool == "nvcc":
        cmd = [NVCC, "-std=c++17", "-O3", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
               "-Xptxas", "-v" if verbose else "-O3", *inc, "-c", path, "-o", obj]
    else:
        # -ffp-contract=off: host geometry rounds the same on every machine
        cmd = ["g++", "-std=c++17", "-O3", "-ffp-contract=off", "-fPIC", "-Wall", "-Wextra",
               "-I", os.path.join(CUDA_HOME, "include"), *inc, "-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compiling {src} failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile and link paper_1005_3158_gb300/libfem.so (libfem_checked.so
    with checked=True: kernels with device-side bounds checks) if any source
    is newer."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    os.makedirs(BUILD, exist_ok=True)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda kv: _compile(kv[0], kv[1], verbose,
                                               checked and kv[0] == "fem_kernels.cu"),
                           SOURCES.items()))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-shared", "-Xcompiler", "-fPIC", *objs, "-o", tmp, "-lcudart_static",
           "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"linking libfem.so failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def clean() -> None:
    shutil.rmtree(BUILD, ignore_errors=True)
    for lib in (LIB, LIB_CHECKED):
        if os.path.exists(lib):
            os.remove(lib)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                checked="--checked" in sys.argv))
