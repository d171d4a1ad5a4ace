"""Oracle: OS-MAP-OSL update with the kinetics-derived prior (Eq. 2-3), FP64.

TEST INFRASTRUCTURE ONLY (see the package header).

For subset k and every frame m, with kappa the global count calibration,
dt_m the frame duration, n_d an optional per-bin factor and r_dm randoms:

    ybar_dm = kappa dt_m n_d sum_v p_vd x_vm + r_dm          (ordinary Poisson)
    rho_dm  = s_dm / ybar_dm            (0 where ybar_dm <= 0)
    back_vm = kappa dt_m sum_{d in S_k} n_d p_vd rho_dm
    sens_v  = kappa sum_{d in S_k} n_d p_vd
    g_vm    = (beta / S) (x_vm - F_vm) / sigma^2             (dU/dx of Eq. 3)
    x_vm   <- x_vm back_vm / max(dt_m sens_v + g_vm, 1e-3 dt_m sens_v)
    (x unchanged where sens_v = 0)

Readings of the paper (Eq. 2 is printed with a minus sign before the prior
gradient and without subsets): the denominator is Green's one-step-late form
"sensitivity + beta dU/dx" with U = (F - x)^2 / (2 sigma^2), which pulls x
towards F; the subset sensitivity replaces the full one and the prior is
scaled by 1/S so that one pass over the subsets applies beta once; the
denominator is clamped at 1e-3 of the sensitivity term.

The precision form (image and ratio stored in bfloat16 or float16 with a
per-frame scale) is the same update with each store rounded to the storage
grid; quantize() is pinned against IEEE binary16 conversion, against ties and
exactly representable values of bfloat16, and against its error bound.

Pins (tests/test_oracle_osl.py): with one subset and beta = 0 it is MLEM and
the Poisson log-likelihood never decreases; x = F makes the prior vanish;
positivity is preserved; OSEM with S subsets equals S successive MLEM-like
updates on the subset matrices.
"""
from __future__ import annotations

import numpy as np


def expected_counts(geom, x, k, kappa, dt, bin_factor=None, randoms=None):
    """ybar [Z][A_k][B][M] for subset k (all angles when k is None)."""
    y = geom.forward(x, k) * (kappa * np.asarray(dt))[None, None, None, :]
    if bin_factor is not None:
        y = y * bin_factor[..., None]
    if randoms is not None:
        y = y + randoms
    return y


def loglik(geom, x, counts, kappa, dt, bin_factor=None, randoms=None):
    """Poisson log-likelihood sum s log ybar - ybar over all bins (log s! dropped)."""
    yb = expected_counts(geom, x, None, kappa, dt, bin_factor, randoms)
    pos = yb > 0
    return float(np.sum(np.where(pos, counts * np.log(np.where(pos, yb, 1.0)), 0.0) - yb))


def osl_update(geom, x, k, counts_k, kappa, dt, bin_factor_k=None, randoms_k=None,
               F=None, beta=0.0, sigma2=1.0):
    """One OS-MAP-OSL-KP update of x [Z][ny][nx][M] on subset k; returns new x."""
    dt = np.asarray(dt, np.float64)
    ybar = expected_counts(geom, x, k, kappa, dt, bin_factor_k, randoms_k)
    rho = np.where(ybar > 0, counts_k / np.where(ybar > 0, ybar, 1.0), 0.0)
    nd = np.ones(counts_k.shape[:-1]) if bin_factor_k is None else bin_factor_k
    back = geom.back(rho * nd[..., None], k) * (kappa * dt)
    sens = geom.back(np.broadcast_to(nd[..., None], nd.shape + (1,)).copy(), k)[..., 0] * kappa
    den = sens[..., None] * dt
    if F is not None and beta != 0.0:
        g = (beta / geom.n_subsets) * (x - F) / sigma2
        den = np.maximum(den + g, 1e-3 * den)
    ok = np.broadcast_to(sens[..., None] > 0, x.shape)
    return np.where(ok, x * back / np.where(ok, den, 1.0), x)


def quantize(v, kind):
    """Round float64 values to the storage grid of the precision form, to nearest
    with ties to even: kind "bf16" keeps 8 significant bits (the float32 exponent
    range, so every value here is normal), "f16" is IEEE binary16 with values
    above its largest finite number 65504 saturated; "f32" is IEEE single."""
    v = np.asarray(v, np.float64)
    if kind == "f32":
        return v.astype(np.float32).astype(np.float64)
    if kind == "f16":
        return np.minimum(v, 65504.0).astype(np.float16).astype(np.float64)
    if kind != "bf16":
        raise ValueError(kind)
    m, e = np.frexp(v)                       # v = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.round(m * 256.0) / 256.0, e)   # np.round: ties to even


def osl_update_stored(geom, xs, k, counts_k, kappa, dt, scale, kind, bin_factor_k=None,
                      randoms_k=None, F=None, beta=0.0, sigma2=1.0):
    """The same update in the precision form: the image is held as stored values
    xs (on the grid of kind) with x = xs * scale[m], the ratio rho is stored on
    that grid too, and the new image is stored as quantize(x_new / scale).
    Arithmetic stays in float64 between the stores."""
    dt = np.asarray(dt, np.float64)
    scale = np.asarray(scale, np.float64)
    x = xs * scale
    ybar = expected_counts(geom, x, k, kappa, dt, bin_factor_k, randoms_k)
    rho = quantize(np.where(ybar > 0, counts_k / np.where(ybar > 0, ybar, 1.0), 0.0), kind)
    nd = np.ones(counts_k.shape[:-1]) if bin_factor_k is None else bin_factor_k
    back = geom.back(rho * nd[..., None], k) * (kappa * dt)
    sens = geom.back(np.broadcast_to(nd[..., None], nd.shape + (1,)).copy(), k)[..., 0] * kappa
    den = sens[..., None] * dt
    if F is not None and beta != 0.0:
        g = (beta / geom.n_subsets) * (x - F) / sigma2
        den = np.maximum(den + g, 1e-3 * den)
    ok = np.broadcast_to(sens[..., None] > 0, x.shape)
    xn = np.where(ok, x * back / np.where(ok, den, 1.0), x)
    return quantize(xn / scale, kind)


def subset_slice(arr, geom, k):
    """Rows of a full sinogram [Z][A][B][...] that belong to subset k."""
    return None if arr is None else arr[:, geom.subsets[k]]


def osl_pass(geom, x, counts, kappa, dt, bin_factor=None, randoms=None,
             F=None, beta=0.0, sigma2=1.0):
    """One pass over subsets 0..S-1 in order."""
    for k in range(geom.n_subsets):
        x = osl_update(geom, x, k, subset_slice(counts, geom, k), kappa, dt,
                       subset_slice(bin_factor, geom, k), subset_slice(randoms, geom, k),
                       F, beta, sigma2)
    return x


def initial_image(geom, counts, kappa, dt, nz, bin_factor=None, randoms=None):
    """Uniform per-frame start image whose expected trues match the measured ones."""
    M = counts.shape[-1]
    ones = np.ones((nz, geom.ny, geom.nx, 1))
    proj = geom.forward(ones, None)[..., 0]                 # [Z][A][B]
    if bin_factor is not None:
        proj = proj * bin_factor
    num = counts.sum(axis=(0, 1, 2))
    if randoms is not None:
        num = num - randoms.sum(axis=(0, 1, 2))
    c = np.maximum(num, 0.0) / (kappa * np.asarray(dt) * proj.sum())
    c = np.maximum(c, 1e-6)
    return np.broadcast_to(c, (nz, geom.ny, geom.nx, M)).copy()
