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


def nvcc_cmd(verbose_ptxas=False, defines=()):
    cmd = ["nvcc", "-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-shared",
           *defines, "-o", LIB] + [os.path.join(SRC, s) for s in SOURCES]
    if verbose_ptxas:
        cmd[1:1] = ["-Xptxas", "-v"]
    return cmd


def build(force=False, verbose_ptxas=False, defines=()):
    deps = [os.path.join(SRC, s) for s in os.listdir(SRC)] + [
        os.path.join(HERE, "..", "include", "kcs.h")]
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(map(os.path.getmtime, deps)):
        return LIB
    subprocess.run(nvcc_cmd(verbose_ptxas, defines), check=True)
    return LIB


if __name__ == "__main__":
    # -DNAME[=VALUE] arguments select build-time alternatives (for example
    # -DKCS_FWD_STAGED=1, the shared-memory-staged forward projector); run the
    # script again without them to restore the default library
    build(force=True, verbose_ptxas="-v" in sys.argv,
          defines=[a for a in sys.argv[1:] if a.startswith("-D")])
    print(LIB)
