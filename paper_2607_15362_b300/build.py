"""Build libgoc.so (the C-ABI library) in-tree with nvcc for sm_103a."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libgoc.so")
# translation units, compiled in parallel: the host side of the C ABI (with the
# metric, initial-state and reduction kernels) and the step kernels of each
# storage type
SOURCES = ["goc_api.cu", "goc_kernels_f32.cu", "goc_kernels_f16.cu", "goc_kernels_bf16.cu"]
DEPS = SOURCES + ["goc_step.cuh", "goc_aux.cuh", "goc_device.cuh", "goc_vec.cuh", "goc_std.cuh",
                  "goc_internal.h", "goc_launch.cuh", "goc_lean.cuh", "goc_aa.cuh"]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    srcs = [os.path.join(CSRC, f) for f in DEPS]
    srcs.append(os.path.join(HERE, "..", "include", "goc.h"))
    return any(os.path.getmtime(s) > t for s in srcs)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    tag = f"{os.getpid()}"
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(CSRC, src.replace(".cu", f".{tag}.o"))
        cmd = [nvcc, *NVCC_FLAGS, "-c", "-o", obj, os.path.join(CSRC, src)]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
            print(" ".join(cmd), file=sys.stderr)
        objs.append(obj)
        procs.append(subprocess.Popen(cmd))
    failed = [src for src, pr in zip(SOURCES, procs) if pr.wait() != 0]
    try:
        if failed:
            raise subprocess.CalledProcessError(1, f"nvcc {' '.join(failed)}")
        tmp = LIB + f".{tag}.tmp"
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp, *objs], check=True)
        os.replace(tmp, LIB)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
