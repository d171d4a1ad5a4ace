"""Pins of the oracle kinetic model against independent methods (CPU only)."""
import numpy as np
import pytest

import kcs_synth as S
from oracle import kinetics as K


def _rk4_frames(xi, ts, te, feng, h):
    """Classical RK4 on C1' = K1 Cp - a C1, C2' = k3 C1 plus running integrals,
    with every frame edge on the step grid; returns frame averages of C_PET."""
    K1, k2, k3, Vb = xi
    a = k2 + k3

    def cp(t):
        return K.feng_cp(t, **feng)

    def f(t, y):
        c = cp(t)
        return np.array([K1 * c - a * y[0], k3 * y[0], y[0] + y[1], c])

    y = np.zeros(4)
    t = 0.0
    keep = {0: y.copy()}
    n = int(round(te[-1] / h))
    for i in range(n):
        k1 = f(t, y)
        k2_ = f(t + h / 2, y + h / 2 * k1)
        k3_ = f(t + h / 2, y + h / 2 * k2_)
        k4 = f(t + h, y + h * k3_)
        y = y + h / 6 * (k1 + 2 * k2_ + 2 * k3_ + k4)
        t = (i + 1) * h
        keep[i + 1] = y.copy()
    out = []
    for s_, e_ in zip(ts, te):
        A = keep[int(round(s_ / h))]
        B = keep[int(round(e_ / h))]
        out.append(((1 - Vb) * (B[2] - A[2]) + Vb * (B[3] - A[3])) / (e_ - s_))
    return np.array(out)


@pytest.mark.parametrize("xi", [(0.10, 0.13, 0.06, 0.04), (0.05, 0.10, 0.04, 0.03),
                                (0.6, 1.7, 0.9, 0.3)])
def test_matches_rk4(xi):
    ts, te = S.schedule(S.SCHEDULES["pr1"])
    F = K.model(np.array([xi]), ts, te, S.FENG, jacobian=False)[0]
    Fr = _rk4_frames(xi, ts, te, S.FENG, h=1.0 / 1200)
    np.testing.assert_allclose(F, Fr, rtol=1e-9)


def test_matches_rk4_with_gaps():
    # non-contiguous frames: the state must be carried across the gaps
    ts = np.array([0.5, 1.0, 4.0, 10.0])
    te = np.array([0.75, 2.0, 7.0, 12.5])
    xi = (0.1, 0.13, 0.06, 0.04)
    F = K.model(np.array([xi]), ts, te, S.FENG, jacobian=False)[0]
    Fr = _rk4_frames(xi, ts, te, S.FENG, h=1.0 / 1200)
    np.testing.assert_allclose(F, Fr, rtol=1e-9)


def _two_exp_feng(A2=30.0, l1=2.0, l2=0.05):
    # Feng form with A1 = A3 = 0: Cp = A2 (exp(-l2 t) - exp(-l1 t))
    return dict(A1=0.0, A2=A2, A3=0.0, l1=l1, l2=l2, l3=0.3)


def _frame_int_exp(mu, ts, te):
    """int_ts^te exp(-mu t) dt."""
    return (np.exp(-mu * ts) - np.exp(-mu * te)) / mu


def test_two_tissue_textbook_closed_form():
    # Irreversible 2TC impulse response K1 (k3 + k2 exp(-a t)) / a convolved with a
    # two-exponential input, integrated over each frame (textbook partial fractions).
    feng = _two_exp_feng()
    terms = [(feng["A2"], feng["l2"]), (-feng["A2"], feng["l1"])]
    ts, te = S.schedule(S.SCHEDULES["paper"])
    for K1, k2, k3, Vb in [(0.1, 0.13, 0.06, 0.04), (0.4, 0.3, 0.0, 0.0), (0.2, 0.5, 0.2, 0.1)]:
        a = k2 + k3
        T = np.zeros(len(ts))
        P = np.zeros(len(ts))
        for c, lam in terms:
            # int_0^t exp(-lam s) ds = (1 - exp(-lam t)) / lam
            T += c * (k3 / a) * ((te - ts) - _frame_int_exp(lam, ts, te)) / lam
            # int_0^t exp(-lam s) exp(-a (t - s)) ds = (exp(-lam t) - exp(-a t)) / (a - lam)
            T += c * (k2 / a) * (_frame_int_exp(lam, ts, te) - _frame_int_exp(a, ts, te)) / (a - lam)
            P += c * _frame_int_exp(lam, ts, te)
        ref = ((1 - Vb) * K1 * T + Vb * P) / (te - ts)
        F = K.model(np.array([[K1, k2, k3, Vb]]), ts, te, feng, jacobian=False)[0]
        np.testing.assert_allclose(F, ref, rtol=1e-10)


def test_a_to_zero_limit():
    # k2 = k3 = 0: C1 = K1 int_0^t Cp, C2 = 0
    feng = _two_exp_feng()
    ts, te = S.schedule(S.SCHEDULES["pr1"])
    K1, Vb = 0.3, 0.05
    T = np.zeros(len(ts))
    P = np.zeros(len(ts))
    for c, lam in [(feng["A2"], feng["l2"]), (-feng["A2"], feng["l1"])]:
        T += c * ((te - ts) - _frame_int_exp(lam, ts, te)) / lam
        P += c * _frame_int_exp(lam, ts, te)
    ref = ((1 - Vb) * K1 * T + Vb * P) / (te - ts)
    F = K.model(np.array([[K1, 0.0, 0.0, Vb]]), ts, te, feng, jacobian=False)[0]
    np.testing.assert_allclose(F, ref, rtol=1e-10)
    # and continuity: a = 1e-12 gives the same values
    F2 = K.model(np.array([[K1, 5e-13, 5e-13, Vb]]), ts, te, feng, jacobian=False)[0]
    np.testing.assert_allclose(F2, ref, rtol=1e-10)


def test_continuity_at_input_exponent():
    ts, te = S.schedule(S.SCHEDULES["pr2"])
    l3 = S.FENG["l3"]
    xs = np.array([[0.1, l3 - 0.05, 0.05, 0.04],
                   [0.1, l3 - 0.05 + 1e-9, 0.05, 0.04],
                   [0.1, l3 - 0.05 - 1e-9, 0.05, 0.04]])
    F = K.model(xs, ts, te, S.FENG, jacobian=False)
    # a = l3 exactly sits midway between its neighbours (no 0/0 blow-up)
    np.testing.assert_allclose(F[0], 0.5 * (F[1] + F[2]), rtol=1e-11)
    np.testing.assert_allclose(F[1], F[0], rtol=1e-7)


def test_jacobian_matches_central_differences():
    ts, te = S.schedule(S.SCHEDULES["pr2"])
    xi = S.jittered_params(5, seed=4)
    F, J = K.model(xi, ts, te, S.FENG)
    for p in range(4):
        h = 1e-4 * np.maximum(np.abs(xi[:, p]), 1e-3)
        xp, xm = xi.copy(), xi.copy()
        xp[:, p] += h
        xm[:, p] -= h
        fd = (K.model(xp, ts, te, S.FENG, jacobian=False)
              - K.model(xm, ts, te, S.FENG, jacobian=False)) / (2 * h[:, None])
        scale = np.abs(J[:, :, p]).max(axis=1, keepdims=True)
        assert np.max(np.abs(fd - J[:, :, p]) / scale) < 1e-6


def test_ki_macro_parameter():
    xi = np.array([[0.1, 0.05, 0.0], [0.13, 0.1, 0.0], [0.06, 0.04, 0.0], [0.04, 0.03, 0.0]])
    np.testing.assert_allclose(K.ki(xi), [0.1 * 0.06 / 0.19, 0.05 * 0.04 / 0.14, 0.0])


def test_blood_only_voxel_is_input():
    # Vb = 1 (blood region): the model is the frame average of Cp itself
    ts, te = S.schedule(S.SCHEDULES["pr1"])
    F = K.model(np.array([[0.0, 0.0, 0.0, 1.0]]), ts, te, S.FENG, jacobian=False)[0]
    tt = np.linspace(0, 1, 20001)
    for m in range(len(ts)):
        t = ts[m] + (te[m] - ts[m]) * tt
        avg = np.trapezoid(K.feng_cp(t, **S.FENG), t) / (te[m] - ts[m])
        assert abs(F[m] / avg - 1) < 1e-6
