"""The forward projector with the image staged in shared memory (GPU).

`k_forward_staged` is built into the library only with -DKCS_FWD_STAGED=1
(it is slower than `k_forward`, so the default library leaves it out).  This
test compiles that form of the projector into a library of its own and checks
through the C ABI that its projections and ratio sinograms equal the default
library's bit for bit: each ray sums the same samples in the same order.  The
geometries cover bins equal to, finer and coarser than the voxels, odd grid
sizes and 2, 3, 4 and 6 frame quads per bin (20 to 64 rays per block).
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1803_10045_b300")


def _declare(lib):
    vp, fp = C.c_void_p, C.c_float
    lib.kcs_create_geometry.argtypes = [C.POINTER(vp), C.c_int, C.c_int, C.c_int, fp, C.c_int,
                                        C.c_int, fp, C.c_int]
    lib.kcs_destroy_geometry.argtypes = [vp]
    lib.kcs_forward_project.argtypes = [vp, C.c_int, C.c_int, vp, vp, vp]
    lib.kcs_osl_ratio.argtypes = [vp, C.c_int, C.c_int, vp, fp, vp, vp, C.c_int, vp, vp, vp, vp]
    lib.kcs_last_error.restype = C.c_char_p
    return lib


def _check(lib, rc):
    assert rc == 0, lib.kcs_last_error().decode()


@pytest.fixture(scope="module")
def libs(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = tmp_path_factory.mktemp("staged") / "libkcs_staged.so"
    subprocess.run([nvcc, "-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-Xcompiler", "-fPIC", "-shared", "-DKCS_FWD_STAGED=1", "-o", str(out),
                    os.path.join(PKG, "csrc", "projector.cu")], check=True)
    return _declare(C.CDLL(os.path.join(PKG, "libkcs.so"))), _declare(C.CDLL(str(out)))


CASES = [  # nx, ny, nz, bins, angles, bin_mm, subsets, frames
    (37, 31, 3, 47, 36, 2.0, 4, 24),
    (64, 64, 2, 96, 90, 2.0, 4, 8),
    (50, 44, 2, 61, 40, 1.7, 5, 12),
    (40, 40, 2, 48, 36, 2.6, 3, 16),
]


@pytest.mark.parametrize("case", CASES)
def test_staged_forward_equals_default(cuda_ok, libs, case):
    nx, ny, nz, B, A, bin_mm, S, M = case
    gen = torch.Generator(device="cuda").manual_seed(nx + M)
    x = torch.rand((nz, ny, nx, M), device="cuda", generator=gen)
    dt = torch.linspace(0.5, 3.0, M, device="cuda")
    counts = torch.randint(0, 20, (nz, A, B, M), device="cuda", generator=gen).float()
    ptr = lambda t: C.c_void_p(t.data_ptr())
    geoms = []
    for lib in libs:
        g = C.c_void_p()
        _check(lib, lib.kcs_create_geometry(C.byref(g), nx, ny, nz, 2.0, B, A, bin_mm, S))
        geoms.append(g)
    try:
        for k in [-1] + list(range(S)):
            n_ang = A if k < 0 else len(range(k, A, S))
            ys = []
            for lib, g in zip(libs, geoms):
                y = torch.full((nz, n_ang, B, M), float("nan"), device="cuda")
                _check(lib, lib.kcs_forward_project(g, k, M, ptr(x), ptr(y), None))
                ys.append(y)
            if k >= 0:
                for lib, g in zip(libs, geoms):
                    rho = torch.full((nz, n_ang, B, M), float("nan"), device="cuda")
                    _check(lib, lib.kcs_osl_ratio(g, k, M, ptr(dt), 0.7, ptr(counts), None, 0, None,
                                                  ptr(x), ptr(rho), None))
                    ys.append(rho)
            torch.cuda.synchronize()
            assert torch.isfinite(ys[0]).all()
            for a_, b_ in zip(ys[0::2], ys[1::2]):
                assert torch.equal(a_, b_), (case, k)
    finally:
        for lib, g in zip(libs, geoms):
            lib.kcs_destroy_geometry(g)
