"""Build libkcs.so (the C-ABI library) in-tree with nvcc for sm_103a."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libkcs.so")
SOURCES = ["projector.cu", "kinetics.cu", "icm.cu", "fma_peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_cmd(verbose_ptxas=False):
    cmd = ["nvcc", "-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-shared",
           "-o", LIB] + [os.path.join(SRC, s) for s in SOURCES]
    if verbose_ptxas:
        cmd[1:1] = ["-Xptxas", "-v"]
    return cmd


def build(force=False, verbose_ptxas=False):
    deps = [os.path.join(SRC, s) for s in os.listdir(SRC)] + [
        os.path.join(HERE, "..", "include", "kcs.h")]
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(map(os.path.getmtime, deps)):
        return LIB
    subprocess.run(nvcc_cmd(verbose_ptxas), check=True)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose_ptxas="-v" in sys.argv)
    print(LIB)
