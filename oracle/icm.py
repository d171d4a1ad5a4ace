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

ICM on this joint objective is not convex and the paper defines no stopping
rule, so parity is on the trajectory for fixed iteration counts.
"""
from __future__ import annotations

import numpy as np

from . import kinetics, lm, osl


def icm(geom, counts, kappa, t_start, t_end, feng, n_iter, n_lm,
        beta_kp, beta_h, delta, x0=None, xi0=None, xi_start=(0.05, 0.10, 0.03, 0.03),
        bin_factor=None, randoms=None, sigma2=1.0):
    dt = np.asarray(t_end) - np.asarray(t_start)
    Z = counts.shape[0]
    x = osl.initial_image(geom, counts, kappa, dt, Z, bin_factor, randoms) if x0 is None else x0.copy()
    have_xi = xi0 is not None
    xi = xi0.copy() if have_xi else np.broadcast_to(
        np.asarray(xi_start, float)[:, None, None, None], (4, Z, geom.ny, geom.nx)).copy()
    for n in range(n_iter):
        F = None
        if n > 0 or have_xi:
            F = kinetics.model_maps(xi, t_start, t_end, feng)
        x = osl.osl_pass(geom, x, counts, kappa, dt, bin_factor, randoms, F, beta_kp, sigma2)
        xi, _ = lm.lm_fit(x, xi, n_lm, t_start, t_end, feng, beta_h, delta)
    F = kinetics.model_maps(xi, t_start, t_end, feng)
    return x, xi, kinetics.ki(xi), F
