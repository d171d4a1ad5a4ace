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
lambda starts at 1e-2 on every fit call.  The paper states no acceptance rule;
a trial must lower the voxel objective by more than tau = 1e-5 of its value,
because smaller changes are below what a float32 evaluation of the model can
resolve (they are rounding noise, and a float32 and a float64 implementation
would otherwise decide them differently); equal objectives count as reject.

Pins (tests/test_oracle_lm.py): noise-free recovery with beta = 0, a brute
force parameter grid on single voxels, delta -> infinity giving the quadratic
prior's Laplacian, constant maps giving zero gradient, FD of H, accepted steps
never raising Phi.
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


def lm_step(x, maps, lam, t_start, t_end, feng, beta, delta,
            lo=(0, 0, 0, 0), hi=(2, 2, 1, 1), nbhd="2d"):
    """One synchronous MAP-LM step for all voxels.

    x [Z][Y][X][M] image TACs, maps [4][Z][Y][X], lam [Z][Y][X].
    Returns (new maps, new lam, accepted mask, Phi at the returned maps).
    """
    sh = maps.shape[1:]
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
    Ft = kinetics.model(trial, t_start, t_end, feng, jacobian=False)
    rt = xv - Ft
    trial_maps = trial.T.reshape(maps.shape)
    phi_t = 0.5 * np.sum(rt * rt, axis=1) + beta * huber_local(trial_maps, maps, delta, nbhd).ravel()
    acc = (phi_t - phi) < -TAU * phi
    new = np.where(acc[:, None], trial, xi)
    lam_new = np.where(acc, np.maximum(lam.ravel() / 10, LAMBDA_MIN),
                       np.minimum(lam.ravel() * 10, LAMBDA_MAX))
    phi_new = np.where(acc, phi_t, phi)
    return (new.T.reshape(maps.shape), lam_new.reshape(sh), acc.reshape(sh),
            phi_new.reshape(sh))


def lm_fit(x, maps, n_steps, t_start, t_end, feng, beta, delta, lam=None, **kw):
    """n_steps synchronous MAP-LM steps; lambda starts at 1e-2 unless given
    (kw: the box lo/hi and the neighbourhood nbhd of lm_step)."""
    if lam is None:
        lam = np.full(maps.shape[1:], LAMBDA0)
    for _ in range(n_steps):
        maps, lam, _, _ = lm_step(x, maps, lam, t_start, t_end, feng, beta, delta, **kw)
    return maps, lam
