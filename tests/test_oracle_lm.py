"""Pins of the oracle Huber prior and MAP-LM step (CPU only)."""
import numpy as np
import pytest

import kcs_synth as S
from oracle import kinetics as K
from oracle import lm


def test_huber_is_continuous_and_psi_is_its_derivative():
    d = 0.3
    t = np.linspace(-2, 2, 4001)
    h = lm.huber(t, d)
    assert np.max(np.abs(np.diff(h))) < 1e-3
    fd = (lm.huber(t + 1e-7, d) - lm.huber(t - 1e-7, d)) / 2e-7
    np.testing.assert_allclose(fd, lm.psi(t, d), atol=1e-6)


def test_huber_large_delta_is_quadratic_laplacian():
    rng = np.random.default_rng(0)
    maps = rng.random((4, 2, 7, 9))
    g = lm.huber_grad(maps, 1e30)
    # interior: 8 xi_v - sum of the 8 neighbours
    m = maps
    nb = sum(np.roll(np.roll(m, -dy, axis=2), -dx, axis=3) for dy, dx in lm.NEIGHBOURS)
    np.testing.assert_allclose(g[:, :, 1:-1, 1:-1], (8 * m - nb)[:, :, 1:-1, 1:-1], rtol=1e-12)
    # corner (0,0): 3 neighbours
    ref = 3 * m[:, :, 0, 0] - m[:, :, 0, 1] - m[:, :, 1, 0] - m[:, :, 1, 1]
    np.testing.assert_allclose(g[:, :, 0, 0], ref, rtol=1e-12)


def test_huber_grad_constant_maps_is_zero():
    assert np.all(lm.huber_grad(np.full((4, 1, 5, 5), 0.7), 0.01) == 0.0)


def test_huber_grad_is_gradient_of_energy():
    rng = np.random.default_rng(1)
    maps = rng.random((4, 1, 6, 6)) * 0.05
    d = 0.01

    def energy(m):
        return 0.5 * lm.huber_local(m, m, d).sum()

    g = lm.huber_grad(maps, d)
    for idx in [(0, 0, 2, 3), (2, 0, 0, 0), (3, 0, 5, 1)]:
        e = np.zeros_like(maps)
        e[idx] = 1e-7
        fd = (energy(maps + e) - energy(maps - e)) / 2e-7
        assert abs(fd - g[idx]) < 1e-6


def _tacs(xi, sched="pr1"):
    ts, te = S.schedule(S.SCHEDULES[sched])
    return ts, te, K.model(xi, ts, te, S.FENG, jacobian=False)


def test_noise_free_recovery():
    xi = np.array([[0.10, 0.13, 0.06, 0.04], [0.05, 0.10, 0.04, 0.03], [0.03, 0.08, 0.02, 0.02]])
    ts, te, F = _tacs(xi)
    x = F.reshape(1, 1, 3, -1)
    start = np.broadcast_to(np.array(S.XI0)[:, None, None, None], (4, 1, 1, 3)).copy()
    maps, _ = lm.lm_fit(x, start, 40, ts, te, S.FENG, beta=0.0, delta=0.01)
    np.testing.assert_allclose(maps.reshape(4, 3).T, xi, rtol=1e-8)


def test_objective_never_increases():
    rng = np.random.default_rng(2)
    xi = S.jittered_params(6, seed=5)
    ts, te, F = _tacs(xi)
    x = (F * (1 + 0.05 * rng.standard_normal(F.shape))).reshape(1, 2, 3, -1)
    maps = np.broadcast_to(np.array(S.XI0)[:, None, None, None], (4, 1, 2, 3)).copy()
    lam = np.full((1, 2, 3), lm.LAMBDA0)
    _, _, _, phi_prev = lm.lm_step(x, maps, lam, ts, te, S.FENG, 0.0, 0.01)
    for _ in range(8):
        maps, lam, acc, phi = lm.lm_step(x, maps, lam, ts, te, S.FENG, 0.0, 0.01)
        assert np.all(phi <= phi_prev * (1 + 1e-10))   # same point re-evaluated: rounding only
        phi_prev = phi


def test_lm_beats_brute_force_grid():
    # single voxel, noisy TAC: after LM the objective is no worse than the best
    # point of a 13^4 grid over a box around the truth.
    xi_t = np.array([0.10, 0.13, 0.06, 0.04])
    ts, te, F = _tacs(xi_t[None])
    rng = np.random.default_rng(3)
    x = F[0] * (1 + 0.02 * rng.standard_normal(F.shape[1]))
    axes = [np.linspace(0.5 * v, 1.5 * v, 13) for v in xi_t]
    G = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 4)
    Fg = K.model(G, ts, te, S.FENG, jacobian=False)
    phig = 0.5 * np.sum((x[None] - Fg) ** 2, axis=1)
    best = G[np.argmin(phig)]
    start = best.reshape(4, 1, 1, 1).copy()
    maps, _ = lm.lm_fit(x.reshape(1, 1, 1, -1), start, 30, ts, te, S.FENG, 0.0, 0.01)
    phi = 0.5 * np.sum((x - K.model(maps.reshape(1, 4), ts, te, S.FENG, jacobian=False)[0]) ** 2)
    assert phi <= phig.min() + 1e-12
    cell = np.array([(a[1] - a[0]) for a in axes])
    assert np.all(np.abs(maps.ravel()[[0, 3]] - best[[0, 3]]) <= 2 * cell[[0, 3]])


@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_step_solves_damped_normal_equations(beta):
    # the accepted trial is xi + solve(J^T J + lam I, J^T r - beta g) (inside the box)
    xi = S.jittered_params(4, seed=6)
    ts, te, F = _tacs(xi)
    x = (F * 1.01).reshape(1, 2, 2, -1)
    maps = (xi.T * 0.97).reshape(4, 1, 2, 2)
    lam = np.full((1, 2, 2), 0.3)
    new, _, acc, _ = lm.lm_step(x, maps, lam, ts, te, S.FENG, beta, 0.01)
    F0, J0 = K.model(maps.reshape(4, -1).T, ts, te, S.FENG)
    g = lm.huber_grad(maps, 0.01).reshape(4, -1).T
    for v in range(4):
        A = J0[v].T @ J0[v] + 0.3 * np.eye(4)
        step = np.linalg.solve(A, J0[v].T @ (x.reshape(4, -1)[v] - F0[v]) - beta * g[v])
        if acc.ravel()[v]:
            np.testing.assert_allclose(new.reshape(4, -1)[:, v],
                                       np.clip(maps.reshape(4, -1)[:, v] + step, 0, [2, 2, 1, 1]),
                                       rtol=1e-10)


def test_huber_3d_large_delta_is_26_neighbour_laplacian():
    rng = np.random.default_rng(5)
    m = rng.random((4, 5, 6, 7))
    g = lm.huber_grad(m, 1e30, nbhd="3d")
    nb = sum(np.roll(m, (-dz, -dy, -dx), axis=(1, 2, 3)) for dz, dy, dx in lm.NEIGHBOURS_3D)
    np.testing.assert_allclose(g[:, 1:-1, 1:-1, 1:-1], (26 * m - nb)[:, 1:-1, 1:-1, 1:-1],
                               rtol=1e-12)
    # corner voxel (0,0,0): 7 neighbours
    ref = 7 * m[:, 0, 0, 0] - sum(m[:, dz, dy, dx] for dz in (0, 1) for dy in (0, 1)
                                  for dx in (0, 1) if (dz, dy, dx) != (0, 0, 0))
    np.testing.assert_allclose(g[:, 0, 0, 0], ref, rtol=1e-12)


def test_huber_3d_single_plane_equals_2d_and_constant_is_zero():
    rng = np.random.default_rng(6)
    m = rng.random((4, 1, 8, 9)) * 0.05
    np.testing.assert_array_equal(lm.huber_grad(m, 0.01, nbhd="3d"), lm.huber_grad(m, 0.01))
    np.testing.assert_array_equal(lm.huber_local(m, m, 0.01, nbhd="3d"), lm.huber_local(m, m, 0.01))
    assert np.all(lm.huber_grad(np.full((4, 3, 4, 4), 0.2), 0.01, nbhd="3d") == 0.0)


def test_huber_3d_grad_is_gradient_of_energy():
    rng = np.random.default_rng(7)
    maps = rng.random((4, 3, 5, 5)) * 0.05
    d = 0.01

    def energy(m):
        return 0.5 * lm.huber_local(m, m, d, nbhd="3d").sum()

    g = lm.huber_grad(maps, d, nbhd="3d")
    for idx in [(0, 1, 2, 3), (2, 0, 0, 0), (3, 2, 4, 1)]:
        e = np.zeros_like(maps)
        e[idx] = 1e-7
        fd = (energy(maps + e) - energy(maps - e)) / 2e-7
        assert abs(fd - g[idx]) < 1e-6
