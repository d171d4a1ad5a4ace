"""Pins of the oracle OS-MAP-OSL-KP update (CPU only)."""
import numpy as np

from oracle import osl
from oracle import projector as P


def _setup(S=1, randoms=True, seed=0):
    g = P.Geometry(24, 24, 2.0, 36, 30, 2.0, S)
    rng = np.random.default_rng(seed)
    xt = rng.uniform(0.5, 3.0, (2, 24, 24, 3))
    dt = np.array([0.5, 1.0, 3.0])
    kappa = 2.0
    ybar = g.forward(xt) * kappa * dt
    r = np.full(ybar.shape, 0.3 * ybar.mean()) if randoms else None
    if r is not None:
        ybar = ybar + r
    counts = rng.poisson(ybar).astype(float)
    return g, xt, dt, kappa, r, counts, ybar


def test_mlem_loglik_monotone():
    g, xt, dt, kappa, r, counts, _ = _setup(S=1, randoms=True)
    x = osl.initial_image(g, counts, kappa, dt, 2, randoms=r)
    prev = osl.loglik(g, x, counts, kappa, dt, randoms=r)
    for _ in range(15):
        x = osl.osl_pass(g, x, counts, kappa, dt, randoms=r)
        cur = osl.loglik(g, x, counts, kappa, dt, randoms=r)
        assert cur >= prev - 1e-9 * abs(prev)
        prev = cur


def test_noise_free_truth_is_fixed_point():
    # s = ybar(x): the MLEM ratio is 1 everywhere, so x is unchanged.
    g, xt, dt, kappa, r, _, ybar = _setup(S=3, randoms=True)
    for k in range(3):
        xn = osl.osl_update(g, xt, k, ybar[:, g.subsets[k]], kappa, dt,
                            randoms_k=r[:, g.subsets[k]])
        np.testing.assert_allclose(xn, xt, rtol=1e-12)


def test_prior_vanishes_at_model_and_pulls_towards_it():
    g, xt, dt, kappa, r, counts, _ = _setup(S=2)
    x = osl.initial_image(g, counts, kappa, dt, 2, randoms=r)
    ck, rk = counts[:, g.subsets[0]], r[:, g.subsets[0]]
    plain = osl.osl_update(g, x, 0, ck, kappa, dt, randoms_k=rk)
    at_f = osl.osl_update(g, x, 0, ck, kappa, dt, randoms_k=rk, F=x.copy(), beta=5.0)
    np.testing.assert_allclose(at_f, plain, rtol=1e-14)
    hi = osl.osl_update(g, x, 0, ck, kappa, dt, randoms_k=rk, F=x + 10.0, beta=5.0)
    lo = osl.osl_update(g, x, 0, ck, kappa, dt, randoms_k=rk, F=0.1 * x, beta=5.0)
    inside = plain > 0
    assert np.all(hi[inside] >= plain[inside]) and np.all(lo[inside] <= plain[inside])


def test_positivity_and_support():
    g, xt, dt, kappa, r, counts, _ = _setup(S=3)
    x = osl.initial_image(g, counts, kappa, dt, 2, randoms=r)
    for _ in range(3):
        x = osl.osl_pass(g, x, counts, kappa, dt, randoms=r, F=0.5 * x, beta=2.0)
    assert np.all(x >= 0)


def test_mlem_single_voxel_closed_form():
    # One voxel seen by one bin with weight w: MLEM gives x s / (x_scale ybar) in one step.
    g = P.Geometry(1, 1, 2.0, 1, 2, 2.0, 1)
    x = np.full((1, 1, 1, 1), 2.0)
    s = np.array([[[[7.0]], [[5.0]]]])
    w = g.P().toarray()[:, 0]                     # both angles, single bin
    out = osl.osl_update(g, x, 0, s, 1.0, [1.0])
    ref = 2.0 * (w[0] * 7.0 / (w[0] * 2.0) + w[1] * 5.0 / (w[1] * 2.0)) / (w[0] + w[1])
    np.testing.assert_allclose(out[0, 0, 0, 0], ref, rtol=1e-14)


def test_quantize_f16_is_ieee_binary16():
    rng = np.random.default_rng(7)
    v = np.concatenate([rng.uniform(0, 2, 5000), 10.0 ** rng.uniform(-9, 5, 5000)])
    want = np.minimum(v.astype(np.float32), 65504).astype(np.float16).astype(np.float64)
    got = osl.quantize(v, "f16")
    # float64 -> binary16 directly and via float32 agree except at double-rounding ties
    assert np.mean(got == want) > 0.999
    assert np.all(np.abs(got - want) <= np.spacing(np.float16(np.clip(want, 6.1e-5, 32768))).astype(float))
    assert osl.quantize(np.array([1e6]), "f16")[0] == 65504.0


def test_quantize_bf16_grid_ties_and_bound():
    # exactly representable values (8 significant bits) are unchanged
    k = np.arange(128, 256, dtype=np.float64)
    for e in (-20, -3, 0, 7, 30):
        v = np.ldexp(k, e)
        assert np.array_equal(osl.quantize(v, "bf16"), v)
    # ties go to the even neighbour: 1 + 2^-8 -> 1, 1 + 3 2^-8 -> 1 + 2^-6
    t = osl.quantize(np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -8 + 2.0 ** -30]), "bf16")
    assert np.array_equal(t, [1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7])
    # relative error at most half a unit in the last place (2^-8 relative)
    rng = np.random.default_rng(8)
    v = 10.0 ** rng.uniform(-30, 30, 20000)
    q = osl.quantize(v, "bf16")
    assert np.all(np.abs(q - v) <= 2.0 ** -8 * v * (1 + 1e-12))
    # agrees with torch's float32 -> bfloat16 conversion on float32 inputs
    import torch
    v32 = v.astype(np.float32)
    ref = torch.from_numpy(v32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(osl.quantize(v32.astype(np.float64), "bf16"), ref)


def test_stored_update_reduces_to_float64_update_at_fine_grid():
    g, xt, dt, kappa, r, counts, _ = _setup(S=3, randoms=True)
    x = osl.initial_image(g, counts, kappa, dt, 2, randoms=r)
    k = 1
    ref = osl.osl_update(g, x, k, osl.subset_slice(counts, g, k), kappa, dt, None,
                         osl.subset_slice(r, g, k))
    scale = x[0, 0, 0, :]
    for kind, tol in (("f32", 1e-6), ("f16", 2e-3), ("bf16", 1.6e-2)):
        got = osl.osl_update_stored(g, osl.quantize(x / scale, kind), k,
                                    osl.subset_slice(counts, g, k), kappa, dt, scale, kind,
                                    randoms_k=osl.subset_slice(r, g, k)) * scale
        err = np.abs(got - ref) / ref
        assert err.max() < tol, (kind, err.max())


def test_icm_methods_compose_as_defined():
    """INDIRECT = OSEM passes then one fit; DIRECT = KCS with beta_h = 0."""
    import kcs_synth as S
    from oracle import icm, lm
    g, xt, dt, kappa, r, counts, _ = _setup(S=3, randoms=False)
    counts = counts[:, :, :, :]
    ts = np.concatenate([[0.0], np.cumsum(dt)[:-1]])
    te = np.cumsum(dt)
    x0 = osl.initial_image(g, counts, kappa, dt, 2)
    xi0 = np.broadcast_to(np.array(S.XI0)[:, None, None, None], (4, 2, 24, 24)).copy()
    xa, xia, _, _ = icm.icm(g, counts, kappa, ts, te, S.FENG, 2, 2, 0.1, 0.1, 0.01,
                            method="indirect")
    xr = osl.osl_pass(g, osl.osl_pass(g, x0, counts, kappa, dt), counts, kappa, dt)
    assert np.array_equal(xa, xr)
    xir, _ = lm.lm_fit(xr, xi0, 2, ts, te, S.FENG, 0.0, 0.01)
    assert np.array_equal(xia, xir)
    xd, xid, _, _ = icm.icm(g, counts, kappa, ts, te, S.FENG, 2, 2, 0.1, 0.1, 0.01, method="direct")
    xk, xik, _, _ = icm.icm(g, counts, kappa, ts, te, S.FENG, 2, 2, 0.1, 0.0, 0.01, method="kcs")
    assert np.array_equal(xd, xk) and np.array_equal(xid, xik)


def test_icm_noise_free_fixed_point():
    """Noise-free data of a phantom with uniform kinetic maps is a fixed point
    of the whole ICM (Sec. II-D): started from those maps and their model
    TACs, every ratio s / ybar is 1, so each OSL update returns the image (the
    back-projected ones equal the sensitivity, and the prior term vanishes
    where x = F); the LM residual and the Huber gradient of uniform maps are
    zero, so the fit keeps the maps.  A wrong sensitivity, kappa or frame
    duration anywhere in the update would move the image off the point."""
    import kcs_synth as S
    from oracle import icm, kinetics
    g = P.Geometry(16, 16, 2.0, 26, 12, 2.0, 3)
    ts, te = S.schedule([(2, 30), (2, 120), (2, 300)])
    dt = te - ts
    xi = np.broadcast_to(np.array(S.CLASS_XI["gm"], float)[:, None, None, None],
                         (4, 1, 16, 16)).copy()
    F = kinetics.model_maps(xi, ts, te, S.FENG)
    kappa = 0.7
    counts = g.forward(F) * kappa * dt
    x, xi_out, _, _ = icm.icm(g, counts, kappa, ts, te, S.FENG, 3, 4, 0.5, 0.5, 0.01,
                              x0=F.copy(), xi0=xi.copy())
    assert np.max(np.abs(x - F) / F) < 1e-9
    assert np.max(np.abs(xi_out - xi) / xi) < 1e-9
    # the same data with the image perturbed is not a fixed point
    x2, _, _, _ = icm.icm(g, counts, kappa, ts, te, S.FENG, 1, 4, 0.5, 0.5, 0.01,
                          x0=F * 1.01, xi0=xi.copy())
    assert np.max(np.abs(x2 - F * 1.01) / F) > 1e-4


def test_osl_prior_linear_response():
    """The kinetics prior in one OSL update (Eq. 2-3), to first order: at
    x = F (1 + eps) in one voxel v, the update with weight beta shrinks the
    deviation by r = (beta / S) F / (sigma2 kappa dt sens_k[v]) more than the
    update without the prior -- the factor that decides the stability of the
    one-step-late update (|1 - r| < 1).  Fixes the sign of the prior term,
    its 1 / S per subset and its sigma2."""
    import kcs_synth as S
    from oracle import kinetics
    g = P.Geometry(16, 16, 2.0, 26, 12, 2.0, 3)
    ts, te = S.schedule([(2, 30), (2, 120)])
    dt = te - ts
    xi = np.broadcast_to(np.array(S.CLASS_XI["gm"], float)[:, None, None, None],
                         (4, 1, 16, 16)).copy()
    F = kinetics.model_maps(xi, ts, te, S.FENG)
    kappa, eps, k, v = 0.7, 1e-6, 1, (0, 8, 7)
    counts_k = osl.subset_slice(g.forward(F) * kappa * dt, g, k)
    x = F.copy()
    x[v] *= 1 + eps
    sens = g.back(np.ones(counts_k.shape[:-1] + (1,)), k)[..., 0]   # P_k^T 1
    x0 = osl.osl_update(g, x, k, counts_k, kappa, dt)
    for beta, sigma2 in ((0.3, 1.0), (0.3, 2.0), (1.2, 1.0)):
        xb = osl.osl_update(g, x, k, counts_k, kappa, dt, None, None, F, beta, sigma2)
        shrink = ((x0[v] - F[v]) - (xb[v] - F[v])) / (F[v] * eps)
        r = (beta / g.n_subsets) * F[v] / (sigma2 * kappa * dt * sens[v])
        assert np.allclose(shrink, r, rtol=1e-4), (beta, sigma2, shrink, r)
