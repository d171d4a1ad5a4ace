"""CUDA Joseph projector vs the FP64 oracle (GPU).

Tolerance derivation: the kernels place samples with float32 fused
multiply-adds, so a fractional position has an absolute error of a few ulp of
the largest coordinate (< 1e-4 of a voxel at these sizes); a sample's value
error is that times the neighbour difference, and float32 accumulation adds
~1e-7 per term.  For positive images with bounded contrast that bounds each
ray's relative error well below 1e-4, and the relative L2 error of a whole
projection below 2e-5.
"""
import numpy as np
import pytest
import torch

import kcs_synth as S
from oracle import projector as OP
from cases import rel_l2

pytestmark = pytest.mark.gpu

CASES = [  # nx, ny, nz, B, A, S, M, bin_mm
    (37, 29, 3, 45, 30, 4, 8, 1.7),
    (64, 64, 2, 96, 90, 4, 12, 2.0),
    (20, 20, 1, 29, 17, 3, 4, 2.0),
    (33, 33, 1, 40, 64, 5, 32, 2.3),
]


def _pair(case):
    import paper_1803_10045_b300 as K
    nx, ny, nz, B, A, Sb, M, db = case
    return (K.Geometry(nx, ny, nz, 2.0, B, A, db, Sb), OP.Geometry(nx, ny, 2.0, B, A, db, Sb))


@pytest.mark.parametrize("case", CASES)
def test_subset_angles_bit_exact(cuda_ok, case):
    kg, og = _pair(case)
    for k in range(og.n_subsets):
        np.testing.assert_array_equal(kg.subset_angles(k), og.subsets[k])
    np.testing.assert_array_equal(kg.subset_angles(-1), np.arange(og.n_angles))


@pytest.mark.parametrize("case", CASES)
def test_forward_matches_oracle(cuda_ok, case):
    import paper_1803_10045_b300 as K
    kg, og = _pair(case)
    nx, ny, nz, B, A, Sb, M, _ = case
    x = S.random_images((nz, ny, nx, M), seed=11)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    for k in [-1, 0, Sb - 1]:
        y = K.forward_project(kg, xt, k).double().cpu().numpy()
        ref = og.forward(x, None if k < 0 else k)
        assert rel_l2(y, ref) < 2e-5
        big = np.abs(ref) > 1e-3 * np.abs(ref).max()
        assert np.max(np.abs(y - ref)[big] / np.abs(ref)[big]) < 1e-4
        assert np.max(np.abs(y - ref)[~big], initial=0) < 1e-4 * np.abs(ref).max()


@pytest.mark.parametrize("case", CASES)
def test_back_matches_oracle(cuda_ok, case):
    import paper_1803_10045_b300 as K
    kg, og = _pair(case)
    nx, ny, nz, B, A, Sb, M, _ = case
    for k in [-1, 1]:
        nA = A if k < 0 else len(og.subsets[k])
        y = S.random_images((nz, nA, B, M), seed=12)
        yt = torch.tensor(y, dtype=torch.float32, device="cuda")
        x = K.back_project(kg, yt, k).double().cpu().numpy()
        ref = og.back(y, None if k < 0 else k)
        assert rel_l2(x, ref) < 2e-5
        big = np.abs(ref) > 1e-3 * np.abs(ref).max()
        assert np.max(np.abs(x - ref)[big] / np.abs(ref)[big]) < 1e-4


@pytest.mark.parametrize("case", CASES[:3])
def test_adjoint_identity(cuda_ok, case):
    import paper_1803_10045_b300 as K
    kg, _ = _pair(case)
    nx, ny, nz, B, A, Sb, M, _ = case
    x = torch.tensor(S.random_images((nz, ny, nx, M), seed=1), dtype=torch.float32, device="cuda")
    for k in [-1, 2]:
        nA = A if k < 0 else kg.n_sub(k)
        y = torch.tensor(S.random_images((nz, nA, B, M), seed=2), dtype=torch.float32, device="cuda")
        lhs = (K.forward_project(kg, x, k).double() * y.double()).sum().item()
        rhs = (x.double() * K.back_project(kg, y, k).double()).sum().item()
        assert abs(lhs / rhs - 1.0) < 1e-6


def test_back_projection_is_the_exact_transpose(cuda_ok):
    # The matrix of the forward (unit images, one per plane) and that of the
    # back-projection (unit sinograms, one per plane) must be bitwise transposes:
    # both kernels generate the same (voxel, bin, weight) triples.
    import paper_1803_10045_b300 as K
    nx = ny = 9
    B, A, M = 13, 10, 4
    V, D = nx * ny, A * B
    gf = K.Geometry(nx, ny, V, 2.0, B, A, 1.9, 1)
    gb = K.Geometry(nx, ny, D, 2.0, B, A, 1.9, 1)
    x = torch.zeros((V, ny, nx, M), device="cuda")
    x.view(V, V, M)[torch.arange(V), torch.arange(V)] = 1.0
    Pf = K.forward_project(gf, x).reshape(V, D, M)[:, :, 0].cpu().numpy()      # [v][d]
    y = torch.zeros((D, A, B, M), device="cuda")
    y.view(D, D, M)[torch.arange(D), torch.arange(D)] = 1.0
    Pb = K.back_project(gb, y).reshape(D, V, M)[:, :, 0].cpu().numpy()        # [d][v]
    np.testing.assert_array_equal(Pf.T, Pb)
    ref = OP.system_matrix(nx, ny, 2.0, B, A, 1.9).toarray()
    np.testing.assert_allclose(Pb, ref, atol=2e-5 * ref.max())


def test_full_size_sampled_rays(cuda_ok):
    # PR2 geometry (344^2 x 127, 344 x 252, 24 frames, subset 7 of 21): sampled
    # rays against the oracle's rows for those angles.
    import paper_1803_10045_b300 as K
    W = S.WORKLOADS["pr2"]
    kg = K.Geometry(W.nx, W.ny, W.nz, W.vox_mm, W.n_bins, W.n_angles, W.bin_mm, W.n_subsets)
    M = W.n_frames
    rng = np.random.default_rng(5)
    gen = torch.Generator(device="cuda").manual_seed(5)
    x = torch.rand((W.nz, W.ny, W.nx, M), device="cuda", generator=gen)
    k = 7
    y = K.forward_project(kg, x, k)
    angles = kg.subset_angles(k)
    for _ in range(6):
        z = int(rng.integers(W.nz))
        ia = int(rng.integers(len(angles)))
        P = OP.system_matrix(W.nx, W.ny, W.vox_mm, W.n_bins, W.n_angles, W.bin_mm, [angles[ia]])
        ref = P @ x[z].reshape(-1, M).double().cpu().numpy()
        got = y[z, ia].double().cpu().numpy()
        assert rel_l2(got, ref) < 2e-5


KINDS = {"bf16": torch.bfloat16, "f16": torch.float16}


@pytest.mark.parametrize("kind", ["bf16", "f16"])
@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[3]])
def test_stored_forward_and_back_match_oracle(cuda_ok, case, kind):
    """Precision form of the standalone projector: an image stored as
    bfloat16 / float16 with a per-frame scale is projected (float32
    accumulation) to the oracle's projection of the same stored values times
    the scale; a stored sinogram is back-projected likewise.  The oracle sees
    exactly the stored values (oracle.osl.quantize of the same numbers)."""
    import paper_1803_10045_b300 as K
    from oracle import osl as OO
    kg, og = _pair(case)
    nx, ny, nz, B, A, Sb, M, _ = case
    rng = np.random.default_rng(5)
    scale = rng.uniform(0.5, 4.0, M)
    x = S.random_images((nz, ny, nx, M), seed=12)
    xs = OO.quantize(x / scale, kind)                    # stored image values
    xt = torch.tensor(xs, dtype=torch.float64).to(KINDS[kind]).cuda()
    assert np.array_equal(xt.double().cpu().numpy(), xs)
    sc = torch.tensor(scale, dtype=torch.float32, device="cuda")
    sc64 = sc.double().cpu().numpy()
    for k in [-1, 1]:
        y = K.forward_project(kg, xt, k, x_scale=sc).double().cpu().numpy()
        ref = og.forward(xs * sc64, None if k < 0 else k)
        assert rel_l2(y, ref) < 2e-5, k
        ys = OO.quantize(og.forward(x, None if k < 0 else k) / scale, kind)   # stored sinogram
        yt = torch.tensor(ys, dtype=torch.float64).to(KINDS[kind]).cuda()
        xb = K.back_project(kg, yt, k, y_scale=sc).double().cpu().numpy()
        refb = og.back(ys * sc64, None if k < 0 else k)
        assert rel_l2(xb, refb) < 2e-5, k


def test_stored_calls_with_float32_equal_plain_calls(cuda_ok):
    import paper_1803_10045_b300 as K
    from paper_1803_10045_b300._lib import lib
    import ctypes as C
    kg, _ = _pair(CASES[1])
    nx, ny, nz, B, A, Sb, M, _ = CASES[1]
    x = torch.tensor(S.random_images((nz, ny, nx, M), seed=13), dtype=torch.float32,
                     device="cuda")
    y0 = K.forward_project(kg, x, 2)
    y1 = torch.empty_like(y0)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.kcs_forward_project_ex(kg.handle, 2, M, C.c_void_p(x.data_ptr()), 0, None,
                                      C.c_void_p(y1.data_ptr()), st) == 0
    b0 = K.back_project(kg, y0, 2)
    b1 = torch.empty_like(b0)
    assert lib.kcs_back_project_ex(kg.handle, 2, M, C.c_void_p(y0.data_ptr()), 0, None,
                                   C.c_void_p(b1.data_ptr()), st) == 0
    torch.cuda.synchronize()
    assert torch.equal(y0, y1) and torch.equal(b0, b1)


def test_geometry_created_on_a_stream_equals_synchronous_one(cuda_ok):
    """kcs_create_geometry_ex uploads the angle table on a stream; work issued
    after it on that stream projects exactly as with the synchronous call."""
    import ctypes as C
    import paper_1803_10045_b300 as K
    from paper_1803_10045_b300._lib import check, lib
    nx, ny, nz, B, A, Sb, M, db = CASES[0]
    kg = K.Geometry(nx, ny, nz, 2.0, B, A, db, Sb)
    x = torch.tensor(S.random_images((nz, ny, nx, M), seed=14), dtype=torch.float32,
                     device="cuda")
    ref = K.forward_project(kg, x, -1)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        h = C.c_void_p()
        check(lib.kcs_create_geometry_ex(C.byref(h), nx, ny, nz, 2.0, B, A, db, Sb,
                                         C.c_void_p(s.cuda_stream)))
        y = torch.empty_like(ref)
        check(lib.kcs_forward_project(h, -1, M, C.c_void_p(x.data_ptr()),
                                      C.c_void_p(y.data_ptr()), C.c_void_p(s.cuda_stream)))
    s.synchronize()
    assert torch.equal(y, ref)
    assert lib.kcs_destroy_geometry(h) == 0


def test_forward_of_an_image_aligned_to_16_bytes_only(cuda_ok):
    """The ABI promises 16-byte alignment only: an image placed 16 bytes off a
    32-byte boundary projects to the same bits as an aligned copy, plain and
    fused with the ratio."""
    import paper_1803_10045_b300 as K
    nx, ny, nz, B, A, Sb, M, db = (33, 29, 2, 40, 36, 4, 24, 2.0)
    kg = K.Geometry(nx, ny, nz, 2.0, B, A, db, Sb)
    x = torch.tensor(S.random_images((nz, ny, nx, M), seed=15), dtype=torch.float32,
                     device="cuda")
    buf = torch.empty(x.numel() + 8, dtype=torch.float32, device="cuda")
    off = 4 if buf.data_ptr() % 32 == 0 else 0      # floats: 16 bytes off a 32-byte boundary
    xs = buf[off:off + x.numel()].view(x.shape)
    xs.copy_(x)
    assert xs.data_ptr() % 16 == 0 and xs.data_ptr() % 32 != 0
    assert x.data_ptr() % 32 == 0
    for k in (-1, 1):
        assert torch.equal(K.forward_project(kg, x, k), K.forward_project(kg, xs, k))
    dt = torch.linspace(0.5, 3.0, M, device="cuda")
    counts = torch.poisson(K.forward_project(kg, x, -1) * dt * 3.0)
    r1 = K.osl_ratio(kg, 2, x, dt, 3.0, counts)
    r2 = K.osl_ratio(kg, 2, xs, dt, 3.0, counts)
    assert torch.equal(r1[..., :M], r2[..., :M])     # the row pitch pads frames M.. unwritten
    # the OSL update reads and writes the image by 256-bit accesses only when
    # it and the model TACs are 32-byte aligned; the 16-byte path gives the same bits
    F = x * 0.9
    xa, xb = x.clone(), xs
    K.osl_update(kg, 2, xa, dt, 3.0, counts, F=F, beta=0.5)
    K.osl_update(kg, 2, xb, dt, 3.0, counts, F=F, beta=0.5)
    assert torch.equal(xa, xb)
