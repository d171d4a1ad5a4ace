"""Oracle: Huber MRF prior (Eq. 5-6) and the MAP Levenberg-Marquardt step (Eq. 4), FP64.

TEST INFRASTRUCTURE ONLY (see the package header).

Huber potential and derivative.  Eq. 5 as printed (t^2 inside) is not
continuous at |t| = delta and Eq. 6 gives -delta for t > delta; this oracle
takes the standard Huber function they approximate:

    h(t)   = t^2 / 2                   if |t| <= delta
           = delta |t| - delta^2 / 2   otherwise
    psi(t) = h'(t) = clamp(t, -delta, delta)

Neighbourhood: the 3x3 in-plane clique of Sec. II-C (8 neighbours, unit
weights, neighbours outside the image skipped, no coupling between planes);
optionally (nbhd = "3d") the 26 neighbours of the 3x3x3 cube, unit weights.
One delta and one beta serve all four maps.

    H_v(xi) = sum_p sum_{k in N8(v)} h(xi_p - xi_{k,p})
    dH_v/dxi_p = sum_{k in N8(v)} psi(xi_p - xi_{k,p})

MAP-LM step for voxel v with neighbours frozen at their start-of-step values
(all voxels advance together, Sec. II-C):

    Phi_v(xi) = 1/2 |x_v - F(xi)|^2 + beta H_v(xi)
    (J^T J + lambda I) step = J^T (x_v - F(xi)) - beta dH_v/dxi      (Eq. 4)
    trial = clamp(xi + step, lo, hi)
    accept iff Phi_v(trial) - Phi_v(xi) < -tau Phi_v(xi):  lambda <- max(lambda/10, 1e-7)
    else keep xi:                                           lambda <- min(10 lambda, 1e7)

Readings: Levenberg damping lambda I exactly as printed (not Marquardt's
diagonal); the box [lo, hi] keeps the trial physical (the paper names none);
lambda starts at 1e-2 on every fit call.  The paper states no acceptance rule.
tau is an argument: tau = 0 is the plain rule (accept any decrease, equal
objectives reject); the default tau = 1e-5 is a sufficient-decrease rule, the
usual safeguard of damped Gauss-Newton methods against steps that do not
make measurable progress (a trial that lowers the objective by less than one
part in 1e5 is treated as no progress, and the damping grows).

float32_spread() and step_error_bound() are not part of the method; they are
tools for comparing a float32 implementation with this oracle.
float32_spread() recomputes one step with the residuals, the normal equations
and the objective sums held in float32 (model values and Jacobian rounded to
float32, frames summed in three different orders, the 4x4 solve in float64)
and reports per voxel how far each recomputation moves the trial and the
decision margin from the float64 step: how well float32 arithmetic resolves
that voxel's step.  step_error_bound() bounds the same movement to first
order (componentwise, worst case) for given relative errors of the model
values and Jacobian.

Pins (tests/test_oracle_lm.py): noise-free recovery with beta = 0, a brute
force parameter grid on single voxels, accepted steps never raising Phi (each
at tau = 0 and at the default tau), tau = 1 rejecting every trial, the
accepted set shrinking as tau grows, delta -> infinity giving the quadratic
prior's Laplacian, constant maps giving zero gradient, FD of H; the error
bound against randomly perturbed models; the float32 spread inside that bound
(at the float32 unit roundoff), zero when recomputed in float64, and its
decision flips only where the bound allows them.
"""
from __future__ import annotations

import numpy as np

from . import kinetics

LAMBDA0 = 1e-2
LAMBDA_MIN, LAMBDA_MAX = 1e-7, 1e7
TAU = 1e-5          # relative objective decrease required to accept a trial
NEIGHBOURS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dy, dx) != (0, 0)]
NEIGHBOURS_3D = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                 if (dz, dy, dx) != (0, 0, 0)]


def huber(t, delta):
    a = np.abs(t)
    return np.where(a <= delta, 0.5 * t * t, delta * a - 0.5 * delta * delta)


def psi(t, delta):
    return np.clip(t, -delta, delta)


def _shifted(maps, dy, dx):
    """Neighbour values maps[..., j+dy, i+dx] and a validity mask (in-plane)."""
    Y, X = maps.shape[-2], maps.shape[-1]
    out = np.zeros_like(maps)
    valid = np.zeros(maps.shape[-2:], bool)
    ys = slice(max(0, -dy), Y - max(0, dy))
    xs = slice(max(0, -dx), X - max(0, dx))
    yn = slice(max(0, dy), Y - max(0, -dy))
    xn = slice(max(0, dx), X - max(0, -dx))
    out[..., ys, xs] = maps[..., yn, xn]
    valid[ys, xs] = True
    return out, valid


def _shifted3(maps, dz, dy, dx):
    """Neighbour values maps[:, z+dz, j+dy, i+dx] and a validity mask [Z][Y][X]."""
    Z = maps.shape[1]
    out = np.zeros_like(maps)
    valid = np.zeros(maps.shape[1:], bool)
    zs = slice(max(0, -dz), Z - max(0, dz))
    zn = slice(max(0, dz), Z - max(0, -dz))
    nb, v2 = _shifted(maps[:, zn], dy, dx)
    out[:, zs] = nb
    valid[zs] = v2
    return out, valid


def _neighbours(maps, nbhd):
    """(neighbour values, validity) for every offset of the neighbourhood:
    "2d" the 8 in-plane neighbours of Sec. II-C, "3d" the 26 of the 3x3x3 cube
    (unit weights, neighbours outside the volume skipped)."""
    if nbhd == "2d":
        for dy, dx in NEIGHBOURS:
            nb, valid = _shifted(maps, dy, dx)
            yield nb, np.broadcast_to(valid, maps.shape[1:])
    elif nbhd == "3d":
        for dz, dy, dx in NEIGHBOURS_3D:
            yield _shifted3(maps, dz, dy, dx)
    else:
        raise ValueError(nbhd)


def huber_grad(maps, delta, nbhd="2d"):
    """dH/dxi for maps [4][Z][Y][X] -> [4][Z][Y][X]."""
    g = np.zeros_like(maps, dtype=np.float64)
    for nb, valid in _neighbours(maps, nbhd):
        g += np.where(valid, psi(maps - nb, delta), 0.0)
    return g


def huber_local(trial, maps, delta, nbhd="2d"):
    """H_v evaluated at per-voxel values trial [4][Z][Y][X] against frozen maps."""
    e = np.zeros(maps.shape[1:])
    for nb, valid in _neighbours(maps, nbhd):
        e += np.where(valid, huber(trial - nb, delta).sum(axis=0), 0.0)
    return e


def huber_grad_local(trial, maps, delta, nbhd="2d", absolute=False):
    """dH_v/dxi at per-voxel values trial [4][Z][Y][X] against frozen maps
    (absolute=True: the sum of |psi| instead, a magnitude for error bounds)."""
    g = np.zeros(trial.shape)
    for nb, valid in _neighbours(maps, nbhd):
        p = psi(trial - nb, delta)
        g += np.where(valid, np.abs(p) if absolute else p, 0.0)
    return g


def step_parts(x, maps, lam, t_start, t_end, feng, beta, delta,
               lo=(0, 0, 0, 0), hi=(2, 2, 1, 1), nbhd="2d", tau=TAU, trial_jacobian=False):
    """Every quantity of one synchronous MAP-LM step (Eq. 4), per voxel [V]...:
    xi, F, J, r = x - F, A = J^T J + lambda I, rhs = J^T r - beta g, step,
    trial, Ft (and Jt when trial_jacobian), rt, phi, phi_t, g and the accept
    mask acc (phi_t - phi < -tau phi)."""
    M = x.shape[-1]
    xi = maps.reshape(4, -1).T                                   # [V][4]
    xv = x.reshape(-1, M)
    F, J = kinetics.model(xi, t_start, t_end, feng)
    r = xv - F
    phi = 0.5 * np.sum(r * r, axis=1) + beta * huber_local(maps, maps, delta, nbhd).ravel()
    g = huber_grad(maps, delta, nbhd).reshape(4, -1).T
    A = np.einsum("vmi,vmj->vij", J, J) + lam.ravel()[:, None, None] * np.eye(4)
    rhs = np.einsum("vmi,vm->vi", J, r) - beta * g
    L = np.linalg.cholesky(A)
    step = np.linalg.solve(np.swapaxes(L, 1, 2), np.linalg.solve(L, rhs[..., None]))[..., 0]
    trial = np.clip(xi + step, np.asarray(lo, float), np.asarray(hi, float))
    if trial_jacobian:
        Ft, Jt = kinetics.model(trial, t_start, t_end, feng)
    else:
        Ft, Jt = kinetics.model(trial, t_start, t_end, feng, jacobian=False), None
    rt = xv - Ft
    trial_maps = trial.T.reshape(maps.shape)
    phi_t = 0.5 * np.sum(rt * rt, axis=1) + beta * huber_local(trial_maps, maps, delta, nbhd).ravel()
    acc = (phi_t - phi) < -tau * phi
    return dict(xi=xi, F=F, J=J, r=r, A=A, rhs=rhs, step=step, trial=trial, Ft=Ft, Jt=Jt,
                rt=rt, phi=phi, phi_t=phi_t, g=g, acc=acc, trial_maps=trial_maps)


def lm_step(x, maps, lam, t_start, t_end, feng, beta, delta,
            lo=(0, 0, 0, 0), hi=(2, 2, 1, 1), nbhd="2d", tau=TAU):
    """One synchronous MAP-LM step for all voxels.

    x [Z][Y][X][M] image TACs, maps [4][Z][Y][X], lam [Z][Y][X]; tau the
    relative decrease a trial must achieve (0: any decrease).
    Returns (new maps, new lam, accepted mask, Phi at the returned maps).
    """
    sh = maps.shape[1:]
    s = step_parts(x, maps, lam, t_start, t_end, feng, beta, delta, lo, hi, nbhd, tau)
    acc = s["acc"]
    new = np.where(acc[:, None], s["trial"], s["xi"])
    lam_new = np.where(acc, np.maximum(lam.ravel() / 10, LAMBDA_MIN),
                       np.minimum(lam.ravel() * 10, LAMBDA_MAX))
    phi_new = np.where(acc, s["phi_t"], s["phi"])
    return (new.T.reshape(maps.shape), lam_new.reshape(sh), acc.reshape(sh),
            phi_new.reshape(sh))


def lm_fit(x, maps, n_steps, t_start, t_end, feng, beta, delta, lam=None, **kw):
    """n_steps synchronous MAP-LM steps; lambda starts at 1e-2 unless given
    (kw: the box lo/hi, the neighbourhood nbhd and tau of lm_step)."""
    if lam is None:
        lam = np.full(maps.shape[1:], LAMBDA0)
    for _ in range(n_steps):
        maps, lam, _, _ = lm_step(x, maps, lam, t_start, t_end, feng, beta, delta, **kw)
    return maps, lam


U32 = 2.0 ** -24      # unit roundoff of float32
U_FF = 2.0 ** -44     # a conservative unit roundoff of float-float (two float32s)


def step_error_bound(x, maps, lam, t_start, t_end, feng, beta, delta, eps_F, eps_J,
                     nbhd="2d", tau=TAU, **kw):
    """First-order bounds on how far a float32 evaluation of one MAP-LM step
    can move the step and the accept decision of each voxel (not part of the
    method: a tool for comparing a float32 implementation with this oracle).

    Error model of the float32 evaluation, per voxel: every model value F_m
    within eps_F max_m |F_m|, every Jacobian entry J_mq within eps_J[q]
    max_m |J_mq| (eps_J: 4 numbers, one per parameter); residuals, products
    and sums rounded in float32 (unit roundoff u, M-term sums within M u of the
    sum of magnitudes); the 4x4 system solved in float-float.  With
    |dJ|_mq = eps_J[q] max|J_.q| and |dr|_m = eps_F max|F| + u |r_m|, the step
    s = A^-1 b (A = J^T J + lambda I, b = J^T r - beta g) moves by at most

        |ds| <= |A^-1| w + 10 u_ff |A^-1| |A| |s| + u |xi + s|,
        w = |dJ|^T |r| + |J|^T |dr| + (|dJ|^T |J| + |J|^T |dJ|) |s|
            + M u (|J|^T |r| + |J|^T |J| |s|) + 2 n u beta sum_k |psi_k|

    (n neighbours), and the clamped trial by no more (clamping is 1-Lipschitz).
    The decision margin m = Phi(trial) - Phi + tau Phi moves by at most

        |dm| <= sum_m |r_m| |dr_m| + sum_m |rt_m| |drt_m| + 3 u (|r|^2 + |rt|^2) / 2
                + |Jt^T rt - beta gt| . |ds| + 2 n u beta (H + Ht) + u tau Phi.

    Returns dict(step_bound [V][4], margin [V], margin_bound [V], acc [V],
    trial [V][4]) with the parts of step_parts()."""
    s = step_parts(x, maps, lam, t_start, t_end, feng, beta, delta, nbhd=nbhd, tau=tau,
                   trial_jacobian=True, **kw)
    M = x.shape[-1]
    n_nb = len(NEIGHBOURS) if nbhd == "2d" else len(NEIGHBOURS_3D)
    eps_J = np.broadcast_to(np.asarray(eps_J, float), (4,))
    J, r, A, step = s["J"], s["r"], s["A"], s["step"]
    aJ, ar, astep = np.abs(J), np.abs(r), np.abs(step)
    dJ = eps_J[None, None, :] * aJ.max(axis=1, keepdims=True)            # [V][1][4]
    dJ = np.broadcast_to(dJ, J.shape)
    dr = eps_F * np.abs(s["F"]).max(axis=1, keepdims=True) + U32 * ar    # [V][M]
    JtJa = np.einsum("vmi,vmj->vij", aJ, aJ)
    gabs = huber_grad_local(maps, maps, delta, nbhd, absolute=True).reshape(4, -1).T
    w = (np.einsum("vmi,vm->vi", dJ, ar) + np.einsum("vmi,vm->vi", aJ, dr)
         + np.einsum("vij,vj->vi", np.einsum("vmi,vmj->vij", dJ, aJ)
                     + np.einsum("vmi,vmj->vij", aJ, dJ), astep)
         + M * U32 * (np.einsum("vmi,vm->vi", aJ, ar) + np.einsum("vij,vj->vi", JtJa, astep))
         + 2 * n_nb * U32 * beta * gabs)
    Ainv = np.abs(np.linalg.inv(A))
    bound = (np.einsum("vij,vj->vi", Ainv, w)
             + 10 * U_FF * np.einsum("vij,vj->vi", Ainv, np.einsum("vij,vj->vi", np.abs(A), astep))
             + U32 * np.abs(s["xi"] + step))
    # decision margin
    rt, Jt = s["rt"], s["Jt"]
    art = np.abs(rt)
    drt = eps_F * np.abs(s["Ft"]).max(axis=1, keepdims=True) + U32 * art
    gt = huber_grad_local(s["trial_maps"], maps, delta, nbhd).reshape(4, -1).T
    grad_t = np.abs(np.einsum("vmi,vm->vi", Jt, rt) - beta * gt)
    H = huber_local(maps, maps, delta, nbhd).ravel()
    Ht = huber_local(s["trial_maps"], maps, delta, nbhd).ravel()
    mb = (np.sum(ar * dr, axis=1) + np.sum(art * drt, axis=1)
          + 1.5 * U32 * (np.sum(r * r, axis=1) + np.sum(rt * rt, axis=1))
          + np.sum(grad_t * bound, axis=1) + 2 * n_nb * U32 * beta * (H + Ht)
          + U32 * tau * s["phi"])
    s.update(step_bound=bound, margin=s["phi_t"] - s["phi"] + tau * s["phi"], margin_bound=mb)
    return s


def _kahan32(v):
    """Compensated float32 sum over the last axis, in order: (s, c), value s - c."""
    f = np.float32
    s = np.zeros(v.shape[:-1], f)
    c = np.zeros(v.shape[:-1], f)
    for m in range(v.shape[-1]):
        y = v[..., m].astype(f) - c
        t = s + y
        c = (t - s) - y
        s = t
    return s, c


def float32_spread(x, maps, lam, t_start, t_end, feng, beta, delta, nbhd="2d", tau=TAU,
                   lo=(0, 0, 0, 0), hi=(2, 2, 1, 1), dtype=np.float32):
    """How far float32 arithmetic moves one MAP-LM step of each voxel.

    The step is recomputed three times with the model values F and Jacobian J
    (the float64 model's) rounded to dtype and the residuals r = x - F, the
    normal equations J^T J, J^T r and the compensated sums of r^2 formed in
    dtype, frames taken in ascending, descending and even-then-odd order; the
    4x4 system is solved in float64, the trial clamped to the box and rounded
    to dtype, and its objective formed the same way.  Returns dict(
    dev_trial [V][4]: largest |trial_f - trial| over the recomputations,
    dev_margin [V]: largest |m_f - m| of the decision margin
    m = Phi(trial) - Phi + tau Phi, flip [V]: some recomputation decides
    accept/reject differently, model_margin [V]: max|F| sum|r| + max|Ft| sum|rt|,
    the first-order change of the margin per unit relative error of the model
    values, huber_margin [V]: 2 n beta (H + Ht), its change per unit rounding
    of the n-term Huber sums) with the float64 parts of step_parts()."""
    f = dtype
    s = step_parts(x, maps, lam, t_start, t_end, feng, beta, delta, lo, hi, nbhd, tau)
    M = x.shape[-1]
    xv = x.reshape(-1, M)
    lo_, hi_ = np.asarray(lo, float), np.asarray(hi, float)
    H = huber_local(maps, maps, delta, nbhd).ravel()
    g = s["g"]
    margin = s["phi_t"] - s["phi"] + tau * s["phi"]
    M_idx = np.arange(M)
    orders = [M_idx, M_idx[::-1], np.r_[M_idx[0::2], M_idx[1::2]]]
    dev_t = np.zeros_like(s["trial"])
    dev_m = np.zeros_like(margin)
    flip = np.zeros(margin.shape, bool)
    for o in orders:
        F = s["F"][:, o].astype(f)
        J = s["J"][:, o].astype(f)
        x32 = xv[:, o].astype(f)
        r = x32 - F
        A = np.zeros((len(F), 4, 4), f)
        b = np.zeros((len(F), 4), f)
        for m in range(M):
            A += J[:, m, :, None] * J[:, m, None, :]
            b += J[:, m, :] * r[:, m, None]
        rs, rc = _kahan32(r * r)
        Ad = A.astype(np.float64) + lam.ravel()[:, None, None] * np.eye(4)
        step = np.linalg.solve(Ad, (b.astype(np.float64) - beta * g)[..., None])[..., 0]
        trial = np.clip(s["xi"] + step, lo_, hi_).astype(f).astype(np.float64)
        Ft = kinetics.model(trial, t_start, t_end, feng, jacobian=False)[:, o].astype(f)
        rt = x32 - Ft
        ts_, tc_ = _kahan32(rt * rt)
        Ht = huber_local(trial.T.reshape(maps.shape), maps, delta, nbhd).ravel()
        phi = 0.5 * (rs.astype(np.float64) - rc) + beta * H
        dphi = 0.5 * ((ts_.astype(np.float64) - rs) - (tc_.astype(np.float64) - rc))
        m_f = dphi + beta * (Ht - H) + tau * phi
        dev_t = np.maximum(dev_t, np.abs(trial - s["trial"]))
        dev_m = np.maximum(dev_m, np.abs(m_f - margin))
        flip |= (m_f < 0) != s["acc"]
    n_nb = len(NEIGHBOURS) if nbhd == "2d" else len(NEIGHBOURS_3D)
    Ht_all = huber_local(s["trial_maps"], maps, delta, nbhd).ravel()
    model_margin = (np.abs(s["F"]).max(axis=1) * np.abs(s["r"]).sum(axis=1)
                    + np.abs(s["Ft"]).max(axis=1) * np.abs(s["rt"]).sum(axis=1))
    s.update(dev_trial=dev_t, dev_margin=dev_m, flip=flip, margin=margin,
             model_margin=model_margin, huber_margin=2 * n_nb * beta * (H + Ht_all))
    return s


def strict_voxels(spread, ref_maps, floor, rel_tol=1e-3, share=0.25, margin_factor=4.0,
                  model_eps=1e-6):
    """Voxels whose step float32 arithmetic resolves well inside the parity
    tolerance, from a float32_spread() result: no recomputation flips the
    decision; the decision margin exceeds margin_factor times the sum of its
    float32 spread, of what a model evaluated within model_eps of its largest
    value (relative) can move it by, and of what float32 rounding of the Huber
    sums can; every trial parameter moves by at most share x the map
    tolerance rel_tol max(|trial_p|, floor_p); and a = k2 + k3 of the returned
    maps is at least 1e-6 (below it k2 and k3 are not identifiable).
    Boolean [V]."""
    tr = spread["trial"]
    tol = rel_tol * np.maximum(np.abs(tr), np.asarray(floor, float)[None, :])
    ok = ~spread["flip"]
    need = (spread["dev_margin"] + model_eps * spread["model_margin"]
            + U32 * spread["huber_margin"])
    ok &= np.abs(spread["margin"]) > margin_factor * need
    ok &= np.all(spread["dev_trial"] <= share * tol, axis=1)
    ref = ref_maps.reshape(4, -1)
    ok &= (ref[1] + ref[2]) >= 1e-6
    return ok
