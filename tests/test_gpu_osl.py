"""CUDA OS-MAP-OSL-KP update vs the FP64 oracle, teacher-forced (GPU).

Both sides start every update from the same image; the GPU result must be
within 1e-4 relative L2 of the oracle's (the image tolerance of the method).
"""
import numpy as np
import pytest
import torch

from oracle import osl as OO
from oracle import projector as OP
from cases import pr1_problem, rel_l2

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _f32(a):
    return None if a is None else np.asarray(a, np.float32).astype(np.float64)


def _small(seed=0, randoms="full", nf=True, bin_mm=2.0):
    nx, ny, nz, B, A, Sb, M = 37, 31, 2, 47, 36, 4, 8
    og = OP.Geometry(nx, ny, 2.0, B, A, bin_mm, Sb)
    rng = np.random.default_rng(seed)
    x_true = rng.uniform(0.5, 3.0, (nz, ny, nx, M))
    dt = np.linspace(0.25, 3.0, M)
    kappa = 3.0
    n = rng.uniform(0.7, 1.3, (nz, A, B)) if nf else None
    ybar = og.forward(x_true) * kappa * dt * (n[..., None] if nf else 1.0)
    r = None
    if randoms == "full":
        r = rng.uniform(0.1, 0.5, ybar.shape) * ybar.mean()
    elif randoms == "frame":
        r = np.full(M, 0.2 * ybar.mean())
    counts = rng.poisson(ybar + (0 if r is None else r)).astype(float)
    x0 = rng.uniform(0.5, 3.0, x_true.shape)
    F = x_true * rng.uniform(0.8, 1.2, x_true.shape)
    # both sides consume float32-representable inputs
    return og, (nx, ny, nz, B, A, Sb, M), _f32(x0), _f32(dt), kappa, counts, _f32(r), _f32(n), _f32(F)


@pytest.mark.parametrize("randoms", ["none", "frame", "full"])
@pytest.mark.parametrize("prior", [0.0, 2.0])
def test_osl_update_matches_oracle(cuda_ok, randoms, prior):
    import paper_1803_10045_b300 as K
    og, (nx, ny, nz, B, A, Sb, M), x0, dt, kappa, counts, r, n, F = _small(randoms=randoms)
    kg = K.Geometry(nx, ny, nz, 2.0, B, A, 2.0, Sb)
    rfull = None if r is None else (np.broadcast_to(r, counts.shape) if r.ndim == 1 else r)
    for k in range(Sb):
        xg = _t(x0)
        K.osl_update(kg, k, xg, _t(dt), kappa, _t(counts), None if r is None else _t(r), _t(n),
                     _t(F) if prior else None, prior, 1.0)
        ref = OO.osl_update(og, x0, k, counts[:, og.subsets[k]], kappa, dt, n[:, og.subsets[k]],
                            None if rfull is None else rfull[:, og.subsets[k]],
                            F if prior else None, prior, 1.0)
        assert rel_l2(xg.cpu().numpy(), ref) < 1e-4


@pytest.mark.parametrize("prior", [0.0, 2.0])
def test_osl_update_float_storage_with_scale(cuda_ok, prior):
    """Float32 storage with a per-frame scale (x held as x / scale[m]; the ABI
    takes a scale for every storage type): the stored update times the scale
    equals the oracle's update of the activity, on 32-byte-aligned arrays of
    an even frame-quad count (where the unscaled update uses 256-bit
    accesses)."""
    import paper_1803_10045_b300 as K
    og, (nx, ny, nz, B, A, Sb, M), x0, dt, kappa, counts, r, n, F = _small()
    kg = K.Geometry(nx, ny, nz, 2.0, B, A, 2.0, Sb)
    assert (M // 4) % 2 == 0
    scale = _f32(np.linspace(0.5, 4.0, M))
    stored = _f32(x0 / scale)
    for k in range(Sb):
        xs = _t(stored)
        assert xs.data_ptr() % 32 == 0
        K.osl_update(kg, k, xs, _t(dt), kappa, _t(counts), _t(r), _t(n),
                     _t(F) if prior else None, prior, 1.0, x_scale=_t(scale))
        ref = OO.osl_update(og, stored * scale, k, counts[:, og.subsets[k]], kappa, dt,
                            n[:, og.subsets[k]], r[:, og.subsets[k]], F if prior else None,
                            prior, 1.0)
        assert rel_l2(xs.double().cpu().numpy() * scale, ref) < 1e-4


@pytest.mark.parametrize("bin_mm", [1.7, 2.6])
def test_osl_update_other_bin_pitch(cuda_ok, bin_mm):
    """Bins finer than the voxels (|beta| < 1 at some angles: up to three rays
    reach a voxel per angle, the back-projection's general candidate loop) and
    coarser ones (the two-candidate instance)."""
    import paper_1803_10045_b300 as K
    og, (nx, ny, nz, B, A, Sb, M), x0, dt, kappa, counts, r, n, F = _small(bin_mm=bin_mm)
    kg = K.Geometry(nx, ny, nz, 2.0, B, A, bin_mm, Sb)
    for k in range(Sb):
        xg = _t(x0)
        K.osl_update(kg, k, xg, _t(dt), kappa, _t(counts), _t(r), _t(n), _t(F), 2.0, 1.0)
        ref = OO.osl_update(og, x0, k, counts[:, og.subsets[k]], kappa, dt, n[:, og.subsets[k]],
                            r[:, og.subsets[k]], F, 2.0, 1.0)
        assert rel_l2(xg.cpu().numpy(), ref) < 1e-4


def test_sensitivity_matches_oracle(cuda_ok):
    import paper_1803_10045_b300 as K
    og, (nx, ny, nz, B, A, Sb, M), x0, dt, kappa, counts, r, n, F = _small()
    kg = K.Geometry(nx, ny, nz, 2.0, B, A, 2.0, Sb)
    s = K.sensitivity(kg, 2, _t(n)).cpu().numpy()
    ref = og.back(n[:, og.subsets[2], :, None], 2)[..., 0]
    assert rel_l2(s, ref) < 1e-5


def test_init_image_matches_oracle(cuda_ok):
    import paper_1803_10045_b300 as K
    og, (nx, ny, nz, B, A, Sb, M), x0, dt, kappa, counts, r, n, F = _small(randoms="full")
    kg = K.Geometry(nx, ny, nz, 2.0, B, A, 2.0, Sb)
    x = K.init_image(kg, _t(dt), kappa, _t(counts), _t(r), _t(n)).cpu().numpy()
    ref = OO.initial_image(og, counts, kappa, dt, nz, n, r)
    np.testing.assert_allclose(x, ref, rtol=1e-5)


def test_pr1_osem_pass_matches_oracle(cuda_ok):
    # Config PR1 data, one full pass over the 4 subsets from the uniform start image.
    import paper_1803_10045_b300 as K
    P = pr1_problem()
    W = P["W"]
    kg = K.Geometry(W.nx, W.ny, W.nz, W.vox_mm, W.n_bins, W.n_angles, W.bin_mm, W.n_subsets)
    x0 = _f32(OO.initial_image(P["g"], P["counts"], P["kappa"], P["dt"], 1))
    dt = _f32(P["dt"])
    xg = _t(x0)
    ct, dtt = _t(P["counts"]), _t(dt)
    x = x0.copy()
    for k in range(W.n_subsets):
        K.osl_update(kg, k, xg, dtt, P["kappa"], ct)
        x = OO.osl_update(P["g"], x, k, P["counts"][:, P["g"].subsets[k]], P["kappa"], dt)
    assert rel_l2(xg.cpu().numpy(), x) < 1e-4


@pytest.mark.parametrize("randoms", [False, True])
def test_loglik_matches_oracle(cuda_ok, randoms):
    """Poisson log-likelihood of an image (full forward projection, float64
    accumulation) against the oracle's."""
    import paper_1803_10045_b300 as K
    from cases import pr1_problem
    from oracle import osl as OO
    P = pr1_problem()
    W = P["W"]
    kg = K.Geometry(W.nx, W.ny, W.nz, W.vox_mm, W.n_bins, W.n_angles, W.bin_mm, W.n_subsets)
    dt = np.asarray(P["dt"], np.float32).astype(np.float64)
    kappa = float(np.float32(P["kappa"]))
    x = np.asarray(OO.osl_pass(P["g"], OO.initial_image(P["g"], P["counts"], kappa, dt, 1),
                               P["counts"], kappa, dt), np.float32).astype(np.float64)
    r = None
    if randoms:
        r_m = np.asarray(0.2 * P["counts"].mean(axis=(0, 1, 2)), np.float32).astype(np.float64)
        r = np.broadcast_to(r_m, P["counts"].shape)
    ref = OO.loglik(P["g"], x, P["counts"], kappa, dt, randoms=r)
    tt = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    got = K.loglik(kg, tt(x), tt(dt), kappa, tt(P["counts"]),
                   randoms=None if r is None else tt(r_m)).item()
    print(f"loglik gpu {got:.9e} oracle {ref:.9e} rel {abs(got / ref - 1):.2e}")
    assert abs(got / ref - 1) < 1e-5


@pytest.mark.parametrize("M", [8, 12, 24])
def test_split_ratio_pitch_equals_fused_update(cuda_ok, M):
    """The two halves of the update at any ratio row pitch (dense, the padded
    pitch the fused update keeps internally, a wider one) give the fused
    update's image bit for bit, and the ratio frames agree bit for bit."""
    import paper_1803_10045_b300 as K
    nx, ny, nz, B, A, Sb = 37, 31, 2, 47, 36, 4
    og = OP.Geometry(nx, ny, 2.0, B, A, 2.0, Sb)
    rng = np.random.default_rng(M)
    x_true = rng.uniform(0.5, 3.0, (nz, ny, nx, M))
    dt = _f32(np.linspace(0.25, 3.0, M))
    counts = rng.poisson(og.forward(x_true) * 3.0 * dt + 0.5).astype(float)
    x0, F = _f32(rng.uniform(0.5, 3.0, x_true.shape)), _f32(x_true)
    kg = K.Geometry(nx, ny, nz, 2.0, B, A, 2.0, Sb)
    k = 1
    fused = _t(x0)
    K.osl_update(kg, k, fused, _t(dt), 3.0, _t(counts), F=_t(F), beta=2.0)
    pitches = sorted({M, K.rho_frames(M), M + 8})
    assert K.rho_frames(M) == (M + 4 if (M // 4) % 2 == 0 else M)
    rhos = []
    for P in pitches:
        rho = torch.full(kg.sino_shape(P, k), float("nan"), device="cuda")
        K.osl_ratio(kg, k, _t(x0), _t(dt), 3.0, _t(counts), out=rho)
        xs = _t(x0)
        K.osl_backproject(kg, k, xs, _t(dt), 3.0, rho, F=_t(F), beta=2.0)
        assert torch.equal(xs, fused), P
        rhos.append(rho[..., :M])
    for r in rhos[1:]:
        assert torch.equal(r, rhos[0])
    assert torch.isnan(rho[..., M:]).all()     # padding frames are never written
