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


TAUS = [0.0, lm.TAU]


@pytest.mark.parametrize("tau", TAUS)
def test_noise_free_recovery(tau):
    xi = np.array([[0.10, 0.13, 0.06, 0.04], [0.05, 0.10, 0.04, 0.03], [0.03, 0.08, 0.02, 0.02]])
    ts, te, F = _tacs(xi)
    x = F.reshape(1, 1, 3, -1)
    start = np.broadcast_to(np.array(S.XI0)[:, None, None, None], (4, 1, 1, 3)).copy()
    maps, _ = lm.lm_fit(x, start, 40, ts, te, S.FENG, beta=0.0, delta=0.01, tau=tau)
    np.testing.assert_allclose(maps.reshape(4, 3).T, xi, rtol=1e-8)


@pytest.mark.parametrize("tau", TAUS)
def test_objective_never_increases(tau):
    rng = np.random.default_rng(2)
    xi = S.jittered_params(6, seed=5)
    ts, te, F = _tacs(xi)
    x = (F * (1 + 0.05 * rng.standard_normal(F.shape))).reshape(1, 2, 3, -1)
    maps = np.broadcast_to(np.array(S.XI0)[:, None, None, None], (4, 1, 2, 3)).copy()
    lam = np.full((1, 2, 3), lm.LAMBDA0)
    maps, lam, _, phi_prev = lm.lm_step(x, maps, lam, ts, te, S.FENG, 0.0, 0.01, tau=tau)
    for _ in range(8):
        maps, lam, acc, phi = lm.lm_step(x, maps, lam, ts, te, S.FENG, 0.0, 0.01, tau=tau)
        assert np.all(phi <= phi_prev * (1 + 1e-10))   # same point re-evaluated: rounding only
        # an accepted step lowers Phi by more than tau of its value (phi_prev
        # was evaluated without the Jacobian states: equal up to rounding)
        assert np.all(phi[acc] < phi_prev[acc] * (1 - tau + 1e-12))
        phi_prev = phi


def test_tau_one_rejects_every_trial():
    # Phi >= 0, so no trial can lower it by its whole value: every step is a
    # reject, the maps stay and lambda grows tenfold
    xi = S.jittered_params(6, seed=5)
    ts, te, F = _tacs(xi)
    x = (F * 1.03).reshape(1, 2, 3, -1)
    maps = np.broadcast_to(np.array(S.XI0)[:, None, None, None], (4, 1, 2, 3)).copy()
    lam = np.full((1, 2, 3), 0.1)
    new, lam2, acc, _ = lm.lm_step(x, maps, lam, ts, te, S.FENG, 0.5, 0.01, tau=1.0)
    assert not acc.any()
    np.testing.assert_array_equal(new, maps)
    np.testing.assert_allclose(lam2, 1.0)
    # the same step at tau = 0 does accept (the start point is far from the fit)
    assert lm.lm_step(x, maps, lam, ts, te, S.FENG, 0.5, 0.01, tau=0.0)[2].all()


def test_accepted_set_shrinks_as_tau_grows():
    rng = np.random.default_rng(4)
    xi = S.jittered_params(64, seed=7)
    ts, te, F = _tacs(xi)
    x = (F * (1 + 0.02 * rng.standard_normal(F.shape))).reshape(1, 8, 8, -1)
    maps = (xi.T * rng.uniform(0.97, 1.03, xi.T.shape)).reshape(4, 1, 8, 8)
    lam = 10.0 ** rng.uniform(-4, 1, (1, 8, 8))
    prev = None
    counts = []
    for tau in (0.0, 1e-7, 1e-5, 1e-3, 1e-1):
        acc = lm.lm_step(x, maps, lam, ts, te, S.FENG, 0.1, 0.01, tau=tau)[2]
        if prev is not None:
            assert np.all(prev | ~acc)           # acc(tau) is a subset of acc(smaller tau)
        prev = acc
        counts.append(int(acc.sum()))
    assert counts[0] > counts[-1]                # the threshold does decide some voxels


@pytest.mark.parametrize("tau", TAUS)
def test_lm_beats_brute_force_grid(tau):
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
    maps, _ = lm.lm_fit(x.reshape(1, 1, 1, -1), start, 30, ts, te, S.FENG, 0.0, 0.01, tau=tau)
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


def _perturbed_step(x, maps, lam, ts, te, beta, delta, eps_F, eps_J, rng, tau):
    """The step and decision margin of lm_step recomputed (float64) from a model
    whose values and Jacobian entries are moved by +-eps of their per-voxel
    maxima (random signs): what a float32 evaluation within that budget may do."""
    M = x.shape[-1]
    xi = maps.reshape(4, -1).T
    xv = x.reshape(-1, M)

    def pert_model(p, jac):
        out = K.model(p, ts, te, S.FENG, jacobian=jac)
        F = out[0] if jac else out
        Fp = F + eps_F * np.abs(F).max(axis=1, keepdims=True) * rng.choice([-1, 1], F.shape)
        if not jac:
            return Fp
        J = out[1]
        Jp = J + (np.asarray(eps_J)[None, None, :] * np.abs(J).max(axis=1, keepdims=True)
                  * rng.choice([-1, 1], J.shape))
        return Fp, Jp

    F, J = pert_model(xi, True)
    r = xv - F
    H = lm.huber_local(maps, maps, delta).ravel()
    phi = 0.5 * np.sum(r * r, axis=1) + beta * H
    g = lm.huber_grad(maps, delta).reshape(4, -1).T
    A = np.einsum("vmi,vmj->vij", J, J) + lam.ravel()[:, None, None] * np.eye(4)
    step = np.linalg.solve(A, (np.einsum("vmi,vm->vi", J, r) - beta * g)[..., None])[..., 0]
    trial = np.clip(xi + step, 0, [2, 2, 1, 1])
    rt = xv - pert_model(trial, False)
    Ht = lm.huber_local(trial.T.reshape(maps.shape), maps, delta).ravel()
    phi_t = 0.5 * np.sum(rt * rt, axis=1) + beta * Ht
    return step, phi_t - phi + tau * phi


@pytest.mark.parametrize("beta", [0.0, 50.0])
def test_step_error_bound_holds_for_perturbed_models(beta):
    """step_error_bound is a bound: on every voxel where it is small (the
    first-order regime it is used in), the step and the decision margin
    recomputed from randomly perturbed models within the budget move by less."""
    rng = np.random.default_rng(11)
    n = 10
    xi_t = np.clip(S.jittered_params(n * n, seed=12, rel=0.5), 0, [2, 2, 1, 1])
    ts, te, F = _tacs(xi_t)
    x = (F * (1 + 0.05 * rng.standard_normal(F.shape))).reshape(1, n, n, -1)
    maps = np.clip(xi_t.T * rng.uniform(0.7, 1.3, xi_t.T.shape), 0, [[2], [2], [1], [1]]
                   ).reshape(4, 1, n, n)
    lam = 10.0 ** rng.uniform(-6, 1, (1, n, n))
    eps_F, eps_J = 3e-7, (3e-7, 7e-7, 4e-7, 3e-7)
    b = lm.step_error_bound(x, maps, lam, ts, te, S.FENG, beta, 0.01, eps_F, eps_J)
    lin = np.all(b["step_bound"] <= 1e-2 * np.maximum(np.abs(b["trial"]), 1e-4), axis=1)
    assert lin.mean() > 0.5
    worst_s, worst_m = 0.0, 0.0
    for _ in range(8):
        step, margin = _perturbed_step(x, maps, lam, ts, te, beta, 0.01, eps_F, eps_J, rng,
                                       lm.TAU)
        ds = np.abs(step - b["step"])[lin] / b["step_bound"][lin]
        dm = np.abs(margin - b["margin"])[lin] / b["margin_bound"][lin]
        worst_s, worst_m = max(worst_s, ds.max()), max(worst_m, dm.max())
    print(f"largest perturbation / bound: step {worst_s:.3f}, margin {worst_m:.3f}")
    assert worst_s <= 1.0 and worst_m <= 1.0
    # and the bound is not vacuous: perturbations reach a fair share of it
    assert worst_s > 0.01


def _spread_case(n=12, seed=13):
    rng = np.random.default_rng(seed)
    xi_t = np.clip(S.jittered_params(n * n, seed=seed, rel=0.5), 0, [2, 2, 1, 1])
    ts, te, F = _tacs(xi_t)
    x = (F * (1 + 0.05 * rng.standard_normal(F.shape))).reshape(1, n, n, -1)
    maps = np.clip(xi_t.T * rng.uniform(0.7, 1.3, xi_t.T.shape), 0, [[2], [2], [1], [1]]
                   ).reshape(4, 1, n, n)
    lam = 10.0 ** rng.uniform(-6, 1, (1, n, n))
    f = lambda a: np.asarray(a, np.float32).astype(np.float64)   # noqa: E731
    return ts, te, f(x), f(maps), f(lam)


def test_float32_spread_vanishes_in_float64():
    # the recomputation is the same step: in float64 it reproduces step_parts
    ts, te, x, maps, lam = _spread_case()
    sp = lm.float32_spread(x, maps, lam, ts, te, S.FENG, 0.1, 0.01, dtype=np.float64)
    assert np.all(sp["dev_trial"] <= 1e-10 * np.maximum(np.abs(sp["trial"]), 1e-3))
    assert not sp["flip"].any()


@pytest.mark.parametrize("beta", [0.0, 50.0])
def test_float32_spread_within_first_order_bound(beta):
    """The float32 recomputations are one rounding pattern; step_error_bound
    with model errors of one float32 unit roundoff bounds every such pattern
    (first order), so on the voxels where that bound is small the measured
    spread must stay inside it, and decisions may flip only where the bound
    on the margin reaches zero."""
    ts, te, x, maps, lam = _spread_case()
    sp = lm.float32_spread(x, maps, lam, ts, te, S.FENG, beta, 0.01)
    u = lm.U32
    b = lm.step_error_bound(x, maps, lam, ts, te, S.FENG, beta, 0.01, u, (u, u, u, u))
    lin = np.all(b["step_bound"] <= 1e-2 * np.maximum(np.abs(b["trial"]), 1e-4), axis=1)
    assert lin.mean() > 0.8
    ratio = sp["dev_trial"][lin] / np.maximum(b["step_bound"][lin], 1e-300)
    print(f"float32 spread / bound: max {ratio.max():.3f}, median {np.median(ratio):.2e}")
    assert ratio.max() <= 1.0
    assert np.all(sp["dev_margin"][lin] <= b["margin_bound"][lin])
    assert np.all(np.abs(b["margin"][sp["flip"]]) <= b["margin_bound"][sp["flip"]])
    # the spread is real: float32 does move the steps
    assert np.median(sp["dev_trial"] / np.maximum(np.abs(sp["trial"]), 1e-6)) > 1e-9


def test_strict_voxels_rules():
    ts, te, x, maps, lam = _spread_case()
    sp = lm.float32_spread(x, maps, lam, ts, te, S.FENG, 0.1, 0.01)
    ref = np.where(sp["acc"][:, None], sp["trial"], sp["xi"]).T
    floor = 1e-2 * np.array([0.06, 0.10, 0.04, 0.03])
    st = lm.strict_voxels(sp, ref, floor)
    assert 0.5 < st.mean() < 1.0 or st.all()
    # a voxel whose spread is pushed past a quarter of the tolerance leaves the set
    v = int(np.argmax(st))
    sp2 = dict(sp, dev_trial=sp["dev_trial"].copy())
    sp2["dev_trial"][v, 2] = 0.26e-3 * max(abs(sp["trial"][v, 2]), floor[2])
    assert not lm.strict_voxels(sp2, ref, floor)[v]
    # and so does one with a flipped decision or k2 + k3 below 1e-6
    sp3 = dict(sp, flip=sp["flip"].copy())
    sp3["flip"][v] = True
    assert not lm.strict_voxels(sp3, ref, floor)[v]
    ref4 = ref.copy()
    ref4[1:3, v] = 0.0
    assert not lm.strict_voxels(sp, ref4, floor)[v]
    # a larger allowance for the model error can only shrink the set
    loose = lm.strict_voxels(sp, ref, floor, model_eps=0.0)
    tight = lm.strict_voxels(sp, ref, floor, model_eps=1e-2)
    assert np.all(loose | ~st) and np.all(st | ~tight) and tight.sum() < loose.sum()
