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
