"""Oracle: Iterated Conditional Modes alternation (Sec. II-D), FP64.

TEST INFRASTRUCTURE ONLY (see the package header).

Iteration n:
  a) one OS-MAP-OSL-KP pass over subsets 0..S-1 with the prior built from the
     model TACs F = F(xi) of the current kinetic maps (the prior is off in
     the first iteration unless start maps were supplied, because no fitted
     maps exist yet);
  b) n_lm MAP-LM steps on the new image series, warm-started from xi, with
     lambda reset to 1e-2.
Outputs: image series x, kinetic maps xi, Ki map, and F(xi).

The three methods compared in Sec. IV-A: INDIRECT (OSEM, then a
post-reconstruction fit), DIRECT (the ICM without the spatial prior in the
fit) and KCS DIRECT (the full ICM).

ICM on this joint objective is not convex and the paper defines no stopping
rule, so parity is on the trajectory for fixed iteration counts.

Parity status: the paper prints no trajectory, so icm() is pinned by an
invariant and by its parts: noise-free data of a phantom with uniform kinetic
maps is a fixed point of the whole alternation (every ratio is 1, the prior
term vanishes at x = F, the LM residual and the Huber gradient are zero), and
a perturbed start is not (tests/test_oracle_osl.py); it composes
osl.osl_pass and lm.lm_fit, which are pinned in tests/test_oracle_osl.py and
tests/test_oracle_lm.py, in the order the composition test checks.  The
invariant does not fix the sign of the prior term (it vanishes there); the
OSL pins do.
"""
from __future__ import annotations

import numpy as np

from . import kinetics, lm, osl


def icm(geom, counts, kappa, t_start, t_end, feng, n_iter, n_lm,
        beta_kp, beta_h, delta, x0=None, xi0=None, xi_start=(0.05, 0.10, 0.03, 0.03),
        bin_factor=None, randoms=None, sigma2=1.0, storage=None, method="kcs", nbhd="2d"):
    """storage = None runs in float64 throughout; storage = "bf16" or "f16"
    holds the image (and each subset's ratio sinogram) on that grid with the
    per-frame scale max_v x_vm of the start image (osl.osl_update_stored).

    method (Sec. IV-A): "kcs" as above; "direct" the same with beta_h = 0 (no
    spatial prior in the fit); "indirect" n_iter OSEM passes (no prior, no fit)
    followed by one post-reconstruction fit of n_lm steps with beta_h = 0."""
    if method not in ("kcs", "direct", "indirect"):
        raise ValueError(method)
    if method != "kcs":
        beta_h = 0.0
    dt = np.asarray(t_end) - np.asarray(t_start)
    Z = counts.shape[0]
    x = osl.initial_image(geom, counts, kappa, dt, Z, bin_factor, randoms) if x0 is None else x0.copy()
    if storage is not None:
        scale = x.reshape(-1, x.shape[-1]).max(axis=0)
        x = osl.quantize(x / scale, storage) * scale
    have_xi = xi0 is not None
    xi = xi0.copy() if have_xi else np.broadcast_to(
        np.asarray(xi_start, float)[:, None, None, None], (4, Z, geom.ny, geom.nx)).copy()
    for n in range(n_iter):
        F = None
        if method != "indirect" and (n > 0 or have_xi):
            F = kinetics.model_maps(xi, t_start, t_end, feng)
        if storage is None:
            x = osl.osl_pass(geom, x, counts, kappa, dt, bin_factor, randoms, F, beta_kp, sigma2)
        else:
            xs = x / scale
            for k in range(geom.n_subsets):
                xs = osl.osl_update_stored(
                    geom, xs, k, osl.subset_slice(counts, geom, k), kappa, dt, scale, storage,
                    osl.subset_slice(bin_factor, geom, k), osl.subset_slice(randoms, geom, k),
                    F, beta_kp, sigma2)
            x = xs * scale
        if method != "indirect":
            xi, _ = lm.lm_fit(x, xi, n_lm, t_start, t_end, feng, beta_h, delta, nbhd=nbhd)
    if method == "indirect":
        xi, _ = lm.lm_fit(x, xi, n_lm, t_start, t_end, feng, beta_h, delta, nbhd=nbhd)
    F = kinetics.model_maps(xi, t_start, t_end, feng)
    return x, xi, kinetics.ki(xi), F
