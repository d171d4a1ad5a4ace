"""Seeded synthetic inputs shared by the FP64 oracle tests and the CUDA path.

This module holds only input recipes: frame schedules, the plasma input
function's published coefficients, class-wise kinetic parameters, label maps of
the phantoms, parameter jitter and Poisson sampling.  It contains none of the
method's arithmetic (no projector, no kinetic model, no update rule), so both
the oracle and the CUDA path can consume its outputs without sharing code.

Workloads (sizes follow the paper's simulation and human-data setups, Sec. III
and Sec. IV; the numbers themselves are this library's synthetic stand-ins,
because the paper's phantom figure and the mMR data are not available):

* ``pr1``  single 64x64 slice (2 mm), 3-class phantom, 12 frames, 96 bins x 90
  angles, ~1e6 trues, 4 subsets.
* ``pr2``  stacked-2D 344x344x127 (2.09 mm), 344 bins x 252 angles, 24 frames,
  brain-like phantom with 20 lesions, ~2e8 prompts (80 % trues, 20 % uniform
  randoms), 21 subsets.
"""
from __future__ import annotations

import dataclasses
import numpy as np

# Feng et al. (1993) three-exponential FDG plasma input model, time in minutes:
#   Cp(t) = (A1 t - A2 - A3) exp(-l1 t) + A2 exp(-l2 t) + A3 exp(-l3 t),  t >= 0.
# The coefficients are those commonly quoted for this model; they only shape
# the synthetic input and are passed to both implementations as data.
FENG = dict(A1=851.1225, A2=21.8798, A3=20.8113,
            l1=4.133859, l2=0.01043449, l3=0.1190996)

# Kinetic parameter order used everywhere: (K1, k2, k3, Vb).
PARAM_NAMES = ("K1", "k2", "k3", "Vb")
XI0 = (0.05, 0.10, 0.03, 0.03)            # ICM start value of every voxel
XI_LO = (0.0, 0.0, 0.0, 0.0)              # box of the LM trial step
XI_HI = (2.0, 2.0, 1.0, 1.0)

CLASS_XI = {                               # k4 = 0 (irreversible FDG model)
    "gm": (0.10, 0.13, 0.06, 0.04),
    "wm": (0.05, 0.10, 0.04, 0.03),
    "bg": (0.03, 0.08, 0.02, 0.02),        # background / CSF class
}


def schedule(spec):
    """Frame start/end times in minutes from a list of (count, seconds)."""
    edges = [0.0]
    for n, sec in spec:
        for _ in range(n):
            edges.append(edges[-1] + sec / 60.0)
    e = np.asarray(edges, dtype=np.float64)
    return e[:-1].copy(), e[1:].copy()


SCHEDULES = {
    "pr1": [(4, 30), (4, 120), (4, 300)],
    "pr2": [(8, 15), (4, 60), (6, 180), (6, 300)],
    "paper": [(12, 10), (2, 30), (4, 60), (1, 120), (4, 300), (1, 600)],
    "m16": [(4, 15), (4, 60), (4, 180), (4, 300)],
}


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    nz: int
    vox_mm: float
    n_bins: int
    n_angles: int
    bin_mm: float
    n_subsets: int
    sched: str
    total_prompts: float
    randoms_frac: float

    @property
    def ny(self):
        return self.nx

    @property
    def n_frames(self):
        return sum(n for n, _ in SCHEDULES[self.sched])

    def frames(self):
        return schedule(SCHEDULES[self.sched])


WORKLOADS = {
    "pr1": Workload("pr1", 64, 1, 2.0, 96, 90, 2.0, 4, "pr1", 1.0e6, 0.0),
    # the paper's own simulation (Sec. IV-A): its 24-frame scheme and the
    # concentric phantom with a central blood square, on the PR1 geometry
    "paper": Workload("paper", 64, 1, 2.0, 96, 90, 2.0, 4, "paper", 1.0e6, 0.0),
    "pr2": Workload("pr2", 344, 127, 2.09, 344, 252, 2.09, 21, "pr2", 2.0e8, 0.2),
}


def _ellipse(nx, ny, ax, ay, cx=0.0, cy=0.0):
    i = np.arange(nx) - (nx - 1) / 2.0
    j = np.arange(ny) - (ny - 1) / 2.0
    X, Y = np.meshgrid(i, j, indexing="xy")        # [ny][nx]
    return ((X - cx) / ax) ** 2 + ((Y - cy) / ay) ** 2 <= 1.0


def labels_pr1(n=64):
    """Label map [ny][nx]: 0 outside, 1 background disc r=30, 2 GM ring, 3 WM core."""
    lab = np.zeros((n, n), np.int8)
    lab[_ellipse(n, n, 30, 30)] = 1
    lab[_ellipse(n, n, 24, 20)] = 2
    lab[_ellipse(n, n, 18, 14)] = 3
    return lab


def phantom_pr1(n=64):
    """Kinetic maps [4][1][n][n] float64 of the 3-class slice phantom."""
    lab = labels_pr1(n)
    xi = np.zeros((4, 1, n, n))
    for code, cls in ((1, "bg"), (2, "gm"), (3, "wm")):
        for p in range(4):
            xi[p, 0][lab == code] = CLASS_XI[cls][p]
    return xi


# Table I of the paper, read in the printed column order (f_v, K1, k2, k3) with
# f_v as a fraction (the blood row's 1.0 is pure blood); stored as (K1, k2, k3, Vb).
TABLE1_XI = {
    "blood": (0.0, 0.0, 0.0, 1.0),
    "inner": (0.75, 0.35, 0.031, 0.13),
    "middle": (0.62, 0.30, 0.026, 0.116),
    "outer": (0.51, 0.27, 0.018, 0.0985),
}


def labels_paper(n=64):
    """Label map [ny][nx] of the paper's geometrical phantom (its figure is not
    available; reading: three concentric discs and a central blood square):
    0 outside, 1 outer disc r = 0.44 n, 2 middle r = 0.31 n, 3 inner r = 0.19 n,
    4 blood square of side n / 8."""
    lab = np.zeros((n, n), np.int8)
    lab[_ellipse(n, n, 0.44 * n, 0.44 * n)] = 1
    lab[_ellipse(n, n, 0.31 * n, 0.31 * n)] = 2
    lab[_ellipse(n, n, 0.19 * n, 0.19 * n)] = 3
    h = n // 16
    c = n // 2
    lab[c - h:c + h, c - h:c + h] = 4
    return lab


def phantom_paper(n=64):
    """Kinetic maps [4][1][n][n] float64 of the paper's phantom with Table I values."""
    lab = labels_paper(n)
    xi = np.zeros((4, 1, n, n))
    for code, region in ((1, "outer"), (2, "middle"), (3, "inner"), (4, "blood")):
        for p in range(4):
            xi[p, 0][lab == code] = TABLE1_XI[region][p]
    return xi


def phantom_pr2(nx=344, nz=127, seed=0, n_lesions=20, jitter=0.10,
                dtype=np.float32):
    """Brain-like kinetic maps [4][nz][nx][nx] (head, GM shell, WM core, CSF,
    20 spherical lesions with k3 x1.5, per-voxel multiplicative N(0, jitter))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = (np.arange(nz) - (nz - 1) / 2.0)[:, None, None]
    j = (np.arange(nx) - (nx - 1) / 2.0)[None, :, None]
    i = (np.arange(nx) - (nx - 1) / 2.0)[None, None, :]

    def ell(a, b, c, ox=0.0, oy=0.0, oz=0.0):
        return ((i - ox) / a) ** 2 + ((j - oy) / b) ** 2 + ((k - oz) / c) ** 2 <= 1.0

    head = ell(80, 96, 60)
    brain = ell(70, 86, 55)
    wm = ell(58, 72, 44)
    csf = ell(8, 24, 14, ox=-12) | ell(8, 24, 14, ox=12)
    xi = np.zeros((4, nz, nx, nx), dtype)
    for p in range(4):
        xi[p][head] = CLASS_XI["bg"][p]
        xi[p][brain] = CLASS_XI["gm"][p]
        xi[p][wm] = CLASS_XI["wm"][p]
        xi[p][csf] = CLASS_XI["bg"][p]
    # lesions: centres drawn inside the brain ellipsoid
    placed = 0
    while placed < n_lesions:
        c = rng.uniform(-1, 1, 3) * np.array([60, 76, 46])
        if (c[0] / 64) ** 2 + (c[1] / 80) ** 2 + (c[2] / 50) ** 2 > 1.0:
            continue
        r = rng.uniform(3, 8)
        z0, z1 = int(max(0, np.floor(c[2] + (nz - 1) / 2 - r))), int(min(nz, np.ceil(c[2] + (nz - 1) / 2 + r) + 1))
        sl = slice(z0, z1)
        m = ((i - c[0]) ** 2 + (j - c[1]) ** 2 + (k[sl] - c[2]) ** 2 <= r * r) & brain[sl]
        xi[2, sl][m] *= 1.5
        placed += 1
    if jitter > 0:
        for p in range(4):
            noise = rng.standard_normal(xi[p].shape, dtype=np.float32)
            xi[p] *= np.maximum(1.0 + jitter * noise, 0.0).astype(dtype)
    return xi


def poisson(expected, seed):
    """Poisson counts of an expected-count array (any shape), seeded PCG64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.poisson(np.maximum(expected, 0.0)).astype(np.float64)


def uniform_randoms(n_planes, n_angles, n_bins, dt, total):
    """Uniform randoms [Z][A][B][M], proportional to frame duration, summing to total."""
    dt = np.asarray(dt, np.float64)
    per_bin_min = total / (n_planes * n_angles * n_bins * dt.sum())
    r = np.empty((n_planes, n_angles, n_bins, dt.size))
    r[...] = per_bin_min * dt
    return r


def random_images(shape, seed, lo=0.5, hi=2.0):
    """Positive smooth-ish random images for projector tests (uniform in [lo, hi])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, shape)


def jittered_params(n, seed, rel=0.3):
    """n parameter vectors around the GM class with multiplicative jitter, [n][4]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = np.array(CLASS_XI["gm"])
    return base[None, :] * rng.uniform(1 - rel, 1 + rel, (n, 4))
