"""Oracle: frame-integrated FDG two-tissue irreversible model and its Jacobian (FP64).

TEST INFRASTRUCTURE ONLY (see the package header).

The paper fits a two-tissue irreversible compartment model with blood fraction
f_v (Sec. III-A, Table I; Sec. IV-A) and evaluates its time integrals and
derivatives analytically instead of by numerical integration (Sec. II-C).
With a = k2 + k3 and Vb = f_v the model is the linear ODE

    C1' = K1 Cp - a C1,     C2' = k3 C1,     C_T = C1 + C2,
    C_PET = (1 - Vb) C_T + Vb Cp,            F_m = (1/dt_m) int_{frame m} C_PET dt

with C1(0) = C2(0) = 0 and time in minutes.  The plasma input is the Feng
three-exponential model written as the output of its own linear generator
(u_i = exp(-l_i t), v_1 = t exp(-l_1 t)).

This oracle solves that ODE exactly: all generator states, C1, C2, the running
integrals of C_T and Cp and the forward sensitivities d(C1, C2, int C_T)/d(K1,
k2, k3) form one linear system s' = Q s, propagated across every interval with
the matrix exponential s(t_e) = expm(Q (t_e - t_s)) s(t_s).  Frame values are
differences of the running integrals; gaps between frames are propagated the
same way.  No series in the parameters, no special-case formulas.

The matrix exponential is the textbook Taylor series with scaling and squaring
(Moler and Van Loan, "Nineteen dubious ways", method 3): scale Q h by 2^-s so
its 1-norm is <= 1/4, sum 20 Taylor terms (truncation < 1e-25), square s times.
(A Pade-based library expm was measured to lose ~1e-8 relative accuracy when
a = k2 + k3 comes within 1e-9 of an input exponent; this form stays at ~1e-12.)

Pins (tests/test_oracle_kinetics.py): RK4 integration of the ODE at 1e-4 min
steps, central finite differences of the Jacobian, the one-tissue closed form
(k3 = 0) with a single-exponential input, the a -> 0 limit (k2 = k3 = 0 gives
K1 times the running integral of Cp), continuity across a = l3, and the Ki
macro-parameter K1 k3 / (k2 + k3) of Sec. IV-B.
"""
from __future__ import annotations

import numpy as np

# state indices
U1, V1, U2, U3, C1, C2, QT, QP, PK, QK, RK, P2, Q2, R2, P3, Q3, R3 = range(17)
NS = 17


def expm(A, degree=20):
    """Batched matrix exponential of A [N][n][n] by Taylor scaling and squaring."""
    norm1 = np.abs(A).sum(axis=-2).max(axis=-1)
    s = np.maximum(0, np.ceil(np.log2(np.maximum(norm1, 1e-300) / 0.25))).astype(int)
    B = A / (2.0 ** s)[:, None, None]
    E = np.broadcast_to(np.eye(A.shape[-1]), A.shape).copy()
    T = E.copy()
    for k in range(1, degree + 1):
        T = T @ B / k
        E = E + T
    for i in range(int(s.max(initial=0))):
        E = np.where((i < s)[:, None, None], E @ E, E)
    return E


def feng_cp(t, A1, A2, A3, l1, l2, l3):
    """Feng plasma input Cp(t) for t >= 0 (0 before injection)."""
    t = np.asarray(t, np.float64)
    v = (A1 * t - A2 - A3) * np.exp(-l1 * t) + A2 * np.exp(-l2 * t) + A3 * np.exp(-l3 * t)
    return np.where(t >= 0, v, 0.0)


def system_matrix(xi, feng):
    """Q for a batch of parameter vectors xi [N][4] -> [N][17][17]."""
    xi = np.atleast_2d(np.asarray(xi, np.float64))
    K1, k2, k3 = xi[:, 0], xi[:, 1], xi[:, 2]
    a = k2 + k3
    A1, A2, A3 = feng["A1"], feng["A2"], feng["A3"]
    l1, l2, l3 = feng["l1"], feng["l2"], feng["l3"]
    N = xi.shape[0]
    Q = np.zeros((N, NS, NS))
    # input generator: Cp = c1 u1 + A1 v1 + A2 u2 + A3 u3
    Q[:, U1, U1] = -l1
    Q[:, V1, V1] = -l1
    Q[:, V1, U1] = 1.0
    Q[:, U2, U2] = -l2
    Q[:, U3, U3] = -l3
    cp_row = np.zeros(NS)
    cp_row[U1], cp_row[V1], cp_row[U2], cp_row[U3] = -A2 - A3, A1, A2, A3
    # tissue
    Q[:, C1, :] += K1[:, None] * cp_row[None, :]
    Q[:, C1, C1] += -a
    Q[:, C2, C1] = k3
    Q[:, QT, C1] = 1.0
    Q[:, QT, C2] = 1.0
    Q[:, QP, :] += cp_row[None, :]
    # d/dK1: PK = dC1/dK1, QK = dC2/dK1, RK = d(int C_T)/dK1
    Q[:, PK, :] += cp_row[None, :]
    Q[:, PK, PK] += -a
    Q[:, QK, PK] = k3
    Q[:, RK, PK] = 1.0
    Q[:, RK, QK] = 1.0
    # d/dk2 (a depends on k2)
    Q[:, P2, C1] = -1.0
    Q[:, P2, P2] = -a
    Q[:, Q2, P2] = k3
    Q[:, R2, P2] = 1.0
    Q[:, R2, Q2] = 1.0
    # d/dk3 (a and the C1 -> C2 rate depend on k3)
    Q[:, P3, C1] = -1.0
    Q[:, P3, P3] = -a
    Q[:, Q3, C1] = 1.0
    Q[:, Q3, P3] = k3
    Q[:, R3, P3] = 1.0
    Q[:, R3, Q3] = 1.0
    return Q


def intervals(t_start, t_end):
    """Propagation intervals [(t0, t1, frame or -1)] from t = 0 over all frames."""
    out, t = [], 0.0
    for m, (ts, te) in enumerate(zip(t_start, t_end)):
        if ts > t:
            out.append((t, ts, -1))
        if ts < t:
            raise ValueError("frames must be ordered and non-overlapping")
        out.append((ts, te, m))
        t = te
    return out


def model(xi, t_start, t_end, feng, jacobian=True):
    """Frame-averaged model TAC F [N][M] and Jacobian J [N][M][4] (K1,k2,k3,Vb)."""
    xi = np.atleast_2d(np.asarray(xi, np.float64))
    N, M = xi.shape[0], len(t_start)
    # Without the Jacobian only the first 8 states are needed: Q is block
    # lower-triangular, so the leading block of expm(Q dt) is expm of its
    # leading block.
    ns = NS if jacobian else QP + 1
    Q = system_matrix(xi, feng)[:, :ns, :ns]
    s = np.zeros((N, ns))
    s[:, U1] = s[:, U2] = s[:, U3] = 1.0
    F = np.zeros((N, M))
    J = np.zeros((N, M, 4))
    Vb = xi[:, 3]
    propagators = {}            # one expm per distinct interval length
    for t0, t1, m in intervals(t_start, t_end):
        h = t1 - t0
        if h not in propagators:
            propagators[h] = expm(Q * h)
        s_new = np.einsum("nij,nj->ni", propagators[h], s)
        if m >= 0 and not jacobian:
            dt = t1 - t0
            F[:, m] = ((1 - Vb) * (s_new[:, QT] - s[:, QT]) + Vb * (s_new[:, QP] - s[:, QP])) / dt
        elif m >= 0:
            dt = t1 - t0
            dQT = s_new[:, QT] - s[:, QT]
            dQP = s_new[:, QP] - s[:, QP]
            F[:, m] = ((1 - Vb) * dQT + Vb * dQP) / dt
            J[:, m, 0] = (1 - Vb) * (s_new[:, RK] - s[:, RK]) / dt
            J[:, m, 1] = (1 - Vb) * (s_new[:, R2] - s[:, R2]) / dt
            J[:, m, 2] = (1 - Vb) * (s_new[:, R3] - s[:, R3]) / dt
            J[:, m, 3] = (dQP - dQT) / dt
        s = s_new
    return (F, J) if jacobian else F


def ki(xi):
    """Net uptake rate Ki = K1 k3 / (k2 + k3) (Sec. IV-B); 0 where k2 + k3 = 0."""
    xi = np.asarray(xi, np.float64)
    K1, k2, k3 = xi[0], xi[1], xi[2]
    a = k2 + k3
    return np.where(a > 0, K1 * k3 / np.where(a > 0, a, 1.0), 0.0)


def model_maps(xi_maps, t_start, t_end, feng, jacobian=False, chunk=4096):
    """Apply ``model`` to maps [4][...] -> F [...][M] (and J [...][M][4])."""
    shp = xi_maps.shape[1:]
    flat = np.asarray(xi_maps, np.float64).reshape(4, -1).T
    Fs, Js = [], []
    for c in range(0, flat.shape[0], chunk):
        r = model(flat[c:c + chunk], t_start, t_end, feng, jacobian=jacobian)
        Fs.append(r[0] if jacobian else r)
        if jacobian:
            Js.append(r[1])
    F = np.concatenate(Fs).reshape(shp + (len(t_start),))
    if not jacobian:
        return F
    return F, np.concatenate(Js).reshape(shp + (len(t_start), 4))
