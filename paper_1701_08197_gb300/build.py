"""Build step of the CUDA flagger library (liblof.so, sm_103a only).

Compiles the translation units of csrc/ in parallel with nvcc (the kernel
file once per input type) and links them into
paper_1701_08197_gb300/_build/liblof.so (in-tree, git-ignored).  Rebuilds
only when a source or header is newer than the library.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import threading
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblof.so")
# (source, object, extra nvcc flags)
UNITS = [
    ("lof_kernels.cu", "lof_kernels_ci16.o", ["-DLOF_KERNEL_DT=2"]),
    ("lof_kernels.cu", "lof_kernels_ci8.o", ["-DLOF_KERNEL_DT=1"]),
    ("lof_f32.cu", "lof_f32.o", []),
    ("lof_sir.cu", "lof_sir.o", []),
    ("lof_integ.cu", "lof_integ.o", []),
    ("lof_api.cu", "lof_api.o", []),
    ("lof_noalloc.cu", "lof_noalloc.o", []),
]
SOURCES = sorted({u[0] for u in UNITS})
HEADERS = [os.path.join(CSRC, "lof_internal.h"), os.path.join(INCLUDE, "lof.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
_lock = threading.Lock()


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA flagger library cannot be built")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + HEADERS
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile liblof.so for sm_103a; returns its path."""
    with _lock:
        if not force and not _stale():
            return LIB
        os.makedirs(BUILD, exist_ok=True)
        cc = nvcc()
        common = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE] + ARCH

        def compile_one(unit):
            src, oname, extra = unit
            obj = os.path.join(BUILD, oname)
            cmd = [cc] + common + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
            return obj

        with ThreadPoolExecutor(len(UNITS)) as ex:
            objs = list(ex.map(compile_one, UNITS))
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
