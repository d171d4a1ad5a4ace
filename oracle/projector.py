"""Oracle: Joseph ray-driven system matrix of one stacked-2D plane (FP64).

TEST INFRASTRUCTURE ONLY (see the package header).

The paper writes the acquisition model through the system-matrix element
p_vd, the contribution of voxel v to bin d (Eq. 2 and the text after it), and
leaves the projector unnamed (Sec. II-B uses an in-house GPU projector).  This
library fixes a parallel-beam Joseph projector:

* voxel (i, j) has centre ((i - (nx-1)/2) h, (j - (ny-1)/2) h), h = voxel size;
* angle a has theta_a = a pi / A, a = 0..A-1 (180 degrees);
* bin b has signed offset u_b = (b - (B-1)/2) db; the ray is
  { p : p . (cos theta, sin theta) = u_b };
* if A <= 4a <= 3A (|sin| >= |cos|, ties at 45/135 degrees included) the ray is
  sampled at every column centre x_i, its y is converted to a fractional row
  index and the two bracketing rows are weighted linearly; otherwise rows and
  columns swap roles;
* the step weight is h / max(|cos|, |sin|) (path length per step, mm);
* interpolation partners outside the grid count as zero.

Back-projection is the exact transpose: the same (d, v, w) triples.
Subset k holds the angles a with a mod S == k, in increasing a.

Pins (tests/test_oracle_projector.py): adjoint identity, theta = 0 and 90
degrees reduce to plain row/column sums, a centred point's projection total,
the line integral of a constant disc against its chord length.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def x_major(a: int, n_angles: int) -> bool:
    """True when angle a is sampled column by column (|sin| >= |cos|)."""
    return n_angles <= 4 * a <= 3 * n_angles


def subset_angles(n_angles: int, n_subsets: int, k: int) -> np.ndarray:
    """Angles of ordered subset k: a = k, k+S, k+2S, ..."""
    return np.arange(k, n_angles, n_subsets, dtype=np.int64)


def system_matrix(nx, ny, vox_mm, n_bins, n_angles, bin_mm, angles=None):
    """p_vd for one plane as a CSR matrix of shape (len(angles)*B, ny*nx).

    Row d = ia * B + b for the ia-th listed angle, column v = j * nx + i.
    """
    if angles is None:
        angles = np.arange(n_angles)
    xc = (np.arange(nx) - (nx - 1) / 2.0) * vox_mm
    yc = (np.arange(ny) - (ny - 1) / 2.0) * vox_mm
    u = (np.arange(n_bins) - (n_bins - 1) / 2.0) * bin_mm
    rows, cols, vals = [], [], []
    for ia, a in enumerate(angles):
        th = a * np.pi / n_angles
        c, s = np.cos(th), np.sin(th)
        if x_major(int(a), n_angles):
            w = vox_mm / abs(s)
            ypos = (u[:, None] - xc[None, :] * c) / s          # [B][nx]
            frac = ypos / vox_mm + (ny - 1) / 2.0
            lo = np.floor(frac)
            f = frac - lo
            lo = lo.astype(np.int64)
            for jj, wt in ((lo, 1.0 - f), (lo + 1, f)):
                ok = (jj >= 0) & (jj < ny) & (wt > 0)
                b_idx, i_idx = np.nonzero(ok)
                rows.append(ia * n_bins + b_idx)
                cols.append(jj[ok] * nx + i_idx)
                vals.append(w * wt[ok])
        else:
            w = vox_mm / abs(c)
            xpos = (u[:, None] - yc[None, :] * s) / c          # [B][ny]
            frac = xpos / vox_mm + (nx - 1) / 2.0
            lo = np.floor(frac)
            f = frac - lo
            lo = lo.astype(np.int64)
            for ii, wt in ((lo, 1.0 - f), (lo + 1, f)):
                ok = (ii >= 0) & (ii < nx) & (wt > 0)
                b_idx, j_idx = np.nonzero(ok)
                rows.append(ia * n_bins + b_idx)
                cols.append(j_idx * nx + ii[ok])
                vals.append(w * wt[ok])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.csr_matrix((vals, (rows, cols)),
                         shape=(len(angles) * n_bins, ny * nx))


class Geometry:
    """Plane geometry plus per-subset system matrices (shared by all planes)."""

    def __init__(self, nx, ny, vox_mm, n_bins, n_angles, bin_mm, n_subsets):
        self.nx, self.ny, self.vox_mm = nx, ny, vox_mm
        self.n_bins, self.n_angles, self.bin_mm = n_bins, n_angles, bin_mm
        self.n_subsets = n_subsets
        self.subsets = [subset_angles(n_angles, n_subsets, k) for k in range(n_subsets)]
        self._P = {}

    def P(self, k=None):
        """System matrix of subset k (all angles when k is None)."""
        if k not in self._P:
            ang = None if k is None else self.subsets[k]
            self._P[k] = system_matrix(self.nx, self.ny, self.vox_mm,
                                       self.n_bins, self.n_angles, self.bin_mm, ang)
        return self._P[k]

    def forward(self, x, k=None):
        """x [Z][ny][nx][M] -> y [Z][A_k][B][M]  (y_dm = sum_v p_vd x_vm)."""
        P = self.P(k)
        Z, M = x.shape[0], x.shape[-1]
        out = np.empty((Z, P.shape[0] // self.n_bins, self.n_bins, M))
        for z in range(Z):
            out[z] = (P @ x[z].reshape(-1, M)).reshape(-1, self.n_bins, M)
        return out

    def back(self, y, k=None):
        """y [Z][A_k][B][M] -> x [Z][ny][nx][M]  (x_vm = sum_d p_vd y_dm)."""
        P = self.P(k)
        Z, M = y.shape[0], y.shape[-1]
        out = np.empty((Z, self.ny, self.nx, M))
        for z in range(Z):
            out[z] = (P.T @ y[z].reshape(-1, M)).reshape(self.ny, self.nx, M)
        return out
