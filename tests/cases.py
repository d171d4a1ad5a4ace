"""Shared seeded test problems: inputs from kcs_synth, expected values from the
oracle.  Nothing here calls the CUDA path."""
from __future__ import annotations

import functools

import numpy as np

import kcs_synth as S
from oracle import kinetics as OK
from oracle import projector as OP


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
