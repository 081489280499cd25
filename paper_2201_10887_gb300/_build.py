"""Compile the CUDA library ``libhf.so`` in-tree for sm_103a with nvcc.

The translation units are compiled in parallel and linked into one shared
library next to this file.  Re-running is a no-op when nothing changed.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "libhf.so")
OBJDIR = os.path.join(HERE, "_build")

SOURCES = ["hf_host.cpp", "hf_fit.cpp", "hf_kernels.cu", "hf_noalloc.cu", "hf_rates.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2,-pthread,-ffp-contract=off",
          "-I" + CSRC, "-I" + INCLUDE]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhf.so")
    return cand


def _deps() -> list:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "hf.h"))
    files.append(os.path.abspath(__file__))
    return files


def _compile(src: str, extra: list) -> str:
    obj = os.path.join(OBJDIR, os.path.basename(src) + ".o")
    cmd = [nvcc()] + ARCH + COMMON + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
    subprocess.run(cmd, check=True)
    return obj


def build(force: bool = False, extra_flags: list | None = None, verbose: bool = False) -> str:
    extra = list(extra_flags or [])
    newest = max(os.path.getmtime(p) for p in _deps())
    if not force and not extra and os.path.exists(OUT) and os.path.getmtime(OUT) >= newest:
        return OUT
    os.makedirs(OBJDIR, exist_ok=True)
    if verbose:
        extra = extra + ["-Xptxas", "-v"]
    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    tmp = OUT + f".tmp{os.getpid()}"
    subprocess.run([nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
                   + ["-Xcompiler", "-pthread"], check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
