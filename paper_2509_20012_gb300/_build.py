"""In-tree build of libfredopt.so for sm_103a (nvcc; no cmake).

The translation units (kernels, C ABI, server, no-allocation product, volume
statistics) compile in parallel, then link into
paper_2509_20012_gb300/libfredopt.so with the CUDA runtime linked statically.
`defines` builds variants elsewhere, e.g. the bounds-checked FO_CHECKED=1
library that tests/test_gpu_checked.py loads.
Rebuilds only when a source or header is newer than the library.
"""
from __future__ import annotations

import os
import subprocess
import sys
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libfredopt.so")
SOURCES = ["fredopt_kernels.cu", "fredopt_api.cu", "fredopt_server.cu", "fredopt_noalloc.cu", "fredopt_volume.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]

_lock = threading.Lock()


def nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "fredopt.h"))
    return files


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose: bool = False, lib: str = LIB, defines=()) -> str:
    """Compile the library to `lib`; `defines` are extra -D macros."""
    with _lock:
        if not force and lib == LIB and not needs_build():
            return LIB
        bdir = BUILD if lib == LIB else lib + ".objs"
        os.makedirs(bdir, exist_ok=True)
        objs, procs = [], []
        for src in SOURCES:
            obj = os.path.join(bdir, src.replace(".cu", ".o"))
            objs.append(obj)
            cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *[f"-D{d}" for d in defines], "-c",
                   os.path.join(CSRC, src), "-o", obj]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        for cmd, p in procs:
            out, _ = p.communicate()
            if p.returncode != 0:
                raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{out.decode(errors='replace')}")
        tmp = lib + f".{os.getpid()}.tmp"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout.decode(errors='replace')}")
        os.replace(tmp, lib)
        return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
