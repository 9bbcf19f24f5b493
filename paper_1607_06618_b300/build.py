"""Builds ``libgerbil.so`` in-tree with nvcc for sm_103a (B300)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
SOURCES = ["partition.cu", "count.cu", "runtime.cu", "membench.cu", "server.cu", "encode.cu",
           "sort.cu", "insert_w1_2.cu", "insert_w3.cu", "insert_w4.cu", "insert_w5_7.cu",
           "insert_w8_11.cu", "insert_w12_15.cu"]
HEADERS = ["common.cuh", "kernels.h", "insert.cuh"]
LIB = os.path.join(HERE, "libgerbil.so")
ROOT = os.path.dirname(HERE)

NVCC_FLAGS = [
    "-O3", "-std=c++17", "-lineinfo",
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-Xcompiler", "-fPIC,-O2", "-shared",
    "-I" + os.path.join(ROOT, "include"),
]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps.append(os.path.join(ROOT, "include", "gerbil.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compiles every source to an object in parallel, then links the shared library."""
    if not (force or _stale()):
        return LIB
    from concurrent.futures import ThreadPoolExecutor
    nvcc = os.environ.get("NVCC", "nvcc")
    tag = "tmp%d" % os.getpid()
    flags = [f for f in NVCC_FLAGS if f != "-shared"] + (["-Xptxas", "-v"] if ptxas_info else [])
    flags += os.environ.get("GERBIL_NVCC_FLAGS", "").split()  # e.g. -DGERBIL_MINB_SMALL=4
    objs = [os.path.join(HERE, "_obj_%s_%s.o" % (os.path.splitext(f)[0], tag)) for f in SOURCES]
    cmds = [[nvcc] + flags + ["-c", os.path.join(CSRC, f), "-o", o] for f, o in zip(SOURCES, objs)]
    tmp = LIB + "." + tag
    try:
        with ThreadPoolExecutor(max_workers=min(len(cmds), os.cpu_count() or 1)) as ex:
            for cmd, rc in zip(cmds, ex.map(subprocess.call, cmds)):
                if verbose:
                    print(" ".join(cmd), file=sys.stderr)
                if rc != 0:
                    raise subprocess.CalledProcessError(rc, cmd)
        link = [nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a"] + objs + ["-o", tmp]
        if verbose:
            print(" ".join(link), file=sys.stderr)
        subprocess.check_call(link)
        os.replace(tmp, LIB)
    finally:
        for o in objs + [tmp]:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
