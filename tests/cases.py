"""Shared seeded test problems: inputs from kcs_synth, expected values from the
oracle.  Nothing here calls the CUDA path."""
from __future__ import annotations

import functools

import numpy as np

import kcs_synth as S
from oracle import kinetics as OK
from oracle import lm as OL
from oracle import projector as OP

# Map tolerance floor per parameter (K1, k2, k3, Vb): 1 % of the parameter's
# grey-matter class value; a map value is held to 1e-3 max(|ref|, floor).
FLOOR = 1e-2 * np.array([0.06, 0.10, 0.04, 0.03])


@functools.lru_cache(maxsize=None)
def pr1_problem(seed=0):
    """Config PR1: 64x64 3-class slice, 12 frames, 96 x 90 sinogram, ~1e6 trues."""
    return problem("pr1", seed)


@functools.lru_cache(maxsize=None)
def problem(name, seed=0):
    """PR1, or the paper's own simulation ("paper": its 24-frame scheme and the
    concentric Table-I phantom with a blood square) on the PR1 geometry."""
    W = S.WORKLOADS[name]
    g = OP.Geometry(W.nx, W.ny, W.vox_mm, W.n_bins, W.n_angles, W.bin_mm, W.n_subsets)
    ts, te = W.frames()
    dt = te - ts
    xi = S.phantom_pr1() if name == "pr1" else S.phantom_paper()
    Ft = OK.model_maps(xi, ts, te, S.FENG)
    ybar = g.forward(Ft) * dt
    kappa = W.total_prompts / ybar.sum()
    counts = S.poisson(kappa * ybar, seed)
    return dict(W=W, g=g, ts=ts, te=te, dt=dt, xi=xi, Ftrue=Ft, kappa=kappa, counts=counts)


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def lm_step_parity(got, lam_got, lam_in, spread, min_strict, label=""):
    """Teacher-forced parity of one MAP-LM step (Eq. 4) against the oracle.

    got [4][...] and lam_got [...] are the CUDA step's maps and lambda from
    the state (maps, lam_in) the oracle's float32_spread() result `spread`
    was computed from.  The voxels the comparison holds strictly come from
    the oracle alone (oracle.lm.strict_voxels: float32 arithmetic resolves
    their step within a quarter of the map tolerance and their accept
    decision with margin): there the accept decisions must agree and the
    maps lie within 1e-3 max(|ref|, FLOOR) of the oracle's.  Everywhere, a
    voxel both sides reject keeps its maps bit for bit, and lambda follows the
    GPU's own decision exactly.  min_strict guards against a vacuous test: the
    share of strict voxels is a property of the inputs, fixed by the oracle."""
    acc_r = spread["acc"]
    ref = np.where(acc_r[:, None], spread["trial"], spread["xi"]).T      # [4][V]
    strict = OL.strict_voxels(spread, ref, FLOOR)
    lam_in = np.asarray(lam_in, np.float64).ravel()
    lam_g = np.asarray(lam_got, np.float64).ravel()
    up = np.float32(np.minimum(lam_in * 10, OL.LAMBDA_MAX)).astype(np.float64)
    down = np.float32(np.maximum(lam_in / 10, OL.LAMBDA_MIN)).astype(np.float64)
    acc_g = np.isclose(lam_g, down, rtol=1e-6, atol=0)
    assert np.all(acc_g | np.isclose(lam_g, up, rtol=1e-6, atol=0)), "lambda not /10 or x10"
    g = np.asarray(got, np.float64).reshape(4, -1)
    tol = 1e-3 * np.maximum(np.abs(ref), FLOOR[:, None])
    within = np.all(np.abs(g - ref) <= tol, axis=0)
    agree = acc_g == acc_r
    print(f"{label}: {strict.mean():.4f} of {strict.size} voxels strict "
          f"(excluded: {int(spread['flip'].sum())} decision flips in float32, "
          f"{int((~strict).sum())} in all); accepted {acc_r.mean():.3f}; outside the strict "
          f"set {int((~agree).sum())} decisions differ, {int((agree & ~within).sum())} maps "
          f"outside 1e-3")
    assert strict.mean() >= min_strict, strict.mean()
    assert np.all(agree[strict]), np.flatnonzero(strict & ~agree)[:10]
    assert np.all(within[strict]), np.flatnonzero(strict & ~within)[:10]
    xi = spread["xi"].T
    rej = ~acc_g & ~acc_r
    np.testing.assert_array_equal(g[:, rej], xi[:, rej])
    return strict


def _oracle_icm_job(job):
    """One FP64 oracle ICM run on PR1 (a process-pool worker: oracle only)."""
    from oracle import icm as OI
    weights, method, storage, n_iter = job
    P = pr1_problem()
    kappa = float(np.float32(P["kappa"]))
    return OI.icm(P["g"], P["counts"], kappa, P["ts"], P["te"], S.FENG, n_iter, 10,
                  weights["beta_kp"], weights["beta_h"], weights["delta"], method=method,
                  storage=storage)


def oracle_icm_runs(jobs):
    """Oracle ICM runs (weights, method, storage, n_iter) on PR1, in parallel
    worker processes started by spawn (safe after the CUDA context exists)."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    n = max(1, min(len(jobs), os.cpu_count() or 1))
    with ProcessPoolExecutor(n, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_oracle_icm_job, jobs))


def ulp(v, kind):
    """Spacing of the storage grid of kind ("bf16", "f16" or "f32") at |v|."""
    v = np.abs(np.asarray(v, np.float64))
    if kind == "f16":
        return np.spacing(np.float16(np.minimum(v, 32768))).astype(np.float64)
    if kind == "bf16":
        _, e = np.frexp(np.maximum(v, 1e-38))
        return np.ldexp(1.0, e - 8)
    return np.spacing(v.astype(np.float32)).astype(np.float64)
