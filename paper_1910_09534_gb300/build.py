"""Build the sycsim CUDA library in-tree: paper_1910_09534_gb300/_build/libsycsim.so.

Each translation unit is compiled by nvcc for sm_103a only (one -gencode, so the build
stays quick on the GPU host), in parallel, then linked into one shared library with the
CUDA runtime linked statically.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libsycsim.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["sim_core.cu", "apply.cu", "permute.cu", "reduce.cu", "store.cu", "apply_tc.cu", "apply_tcgen05.cu", "serve.cu", "gates.cpp", "plan.cpp", "split.cpp", "contract.cu",
           "shard.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3",
                 "--expt-relaxed-constexpr", "-I" + INCLUDE]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return "nvcc"


def _headers_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")]
    paths.append(os.path.join(INCLUDE, "sycsim.h"))
    return max(os.path.getmtime(p) for p in paths)


def _compile(src: str, extra: list) -> str:
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    s = os.path.join(CSRC, src)
    if (os.path.exists(obj) and os.path.getmtime(obj) > os.path.getmtime(s)
            and os.path.getmtime(obj) > _headers_mtime()):
        return obj
    cmd = [nvcc()] + CFLAGS + extra + ["-c", s, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj


def build(verbose: bool = False, extra: list | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    extra = extra or []
    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    if not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcuda"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    if verbose:
        print(LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
