"""Builds the library libhyena.so in-tree for sm_103a.

Three translation units compiled in parallel (host.cpp with the host C++
compiler; device.cu, the encrypted-convolution kernels, and mlp.cu, the cost
model's network, with nvcc), linked by nvcc with the static CUDA runtime.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libhyena.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhyena")


def _sources():
    return [os.path.join(CSRC, f) for f in ("host.cpp", "device.cu", "mlp.cu", "internal.h")] + [
        os.path.join(os.path.dirname(HERE), "include", h) for h in ("hyena.h", "hyena_costmodel.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(os.path.dirname(HERE), "include")]
    host_o = os.path.join(OUT_DIR, "host.o")
    dev_o = os.path.join(OUT_DIR, "device.o")
    mlp_o = os.path.join(OUT_DIR, "mlp.o")
    cmds = [
        ["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", "-Wall", "-c", os.path.join(CSRC, "host.cpp"), "-o", host_o] + inc,
        [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v" if verbose else "-O3",
         "-c", os.path.join(CSRC, "device.cu"), "-o", dev_o] + inc,
        [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v" if verbose else "-O3",
         "-c", os.path.join(CSRC, "mlp.cu"), "-o", mlp_o] + inc,
    ]
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for c in cmds]
    for c, pr in zip(cmds, procs):
        out, _ = pr.communicate()
        if verbose and out:
            print(out)
        if pr.returncode != 0:
            raise RuntimeError(f"build failed: {' '.join(c)}\n{out}")
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.run([nvcc, *ARCH, "-shared", "-Xcompiler", "-pthread", "-o", tmp, host_o, dev_o, mlp_o], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force=True, verbose="-v" in sys.argv))
