"""Build the rimo CUDA library in-tree with nvcc for sm_103a (GB300).

Each translation unit compiles in parallel to an object file under _build/, then
the objects link into librimo.so next to this file.  No CMake, no torch extension
machinery: the library is a plain C-ABI shared object.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librimo.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
SOURCES = ["planner.cu", "plan.cu", "fft.cu", "grid.cu", "gbuild.cu", "apply.cu", "noalloc.cu", "mlp.cu", "batch.cu", "hmat.cu", "weights.cu", "fb.cu", "planfile.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librimo")


def _flags(verbose_ptxas: bool = False) -> list[str]:
    f = ["-O3", "-std=c++17", ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
         "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


# Host-side AddressSanitizer + UBSan build of the same sources (device code unchanged), for
# checking the host code (planner, plan files, weights, argument checks); it is loaded with
# RIMO_LIBRARY=<its path> and the two sanitizer runtimes preloaded.
SAN_BUILD = os.path.join(BUILD, "san")
SAN_LIB = os.path.join(HERE, "librimo_san.so")
SAN_FLAGS = ["-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined",
             "-Xcompiler", "-fno-omit-frame-pointer", "-Xcompiler", "-g"]


def _compile(src: str, verbose_ptxas: bool, sanitize: bool = False) -> tuple[str, str]:
    obj = os.path.join(SAN_BUILD if sanitize else BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + _flags(verbose_ptxas) + (SAN_FLAGS if sanitize else [])
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "rimo.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose_ptxas: bool = False, quiet: bool = True, sanitize: bool = False) -> str:
    """Compile all sources and link librimo.so (librimo_san.so with sanitize); returns its path."""
    lib = SAN_LIB if sanitize else LIB
    if not sanitize and not force and not _stale():
        return LIB
    os.makedirs(SAN_BUILD if sanitize else BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose_ptxas, sanitize), SOURCES))
    if verbose_ptxas or not quiet:
        for _, log in results:
            sys.stderr.write(log)
    objs = [o for o, _ in results]
    tmp = lib + ".tmp"
    cmd = [nvcc(), "-shared", ARCH, "-o", tmp] + objs + ["-lpthread"] + (SAN_FLAGS if sanitize else [])
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv, quiet=False,
                sanitize="--sanitize" in sys.argv))
