"""Pins of the oracle projector against geometry it must reproduce (CPU only)."""
import numpy as np
import pytest

from oracle import projector as P


def _geom(nx=24, B=24, A=12, vox=2.0, db=2.0, S=3):
    return P.Geometry(nx, nx, vox, B, A, db, S)


def test_adjoint_identity():
    g = _geom(nx=20, B=29, A=17, vox=2.0, db=1.7, S=4)
    rng = np.random.default_rng(1)
    for k in [None, 0, 3]:
        nA = g.n_angles if k is None else len(g.subsets[k])
        x = rng.random((2, 20, 20, 3))
        y = rng.random((2, nA, 29, 3))
        lhs = np.sum(g.forward(x, k) * y)
        rhs = np.sum(x * g.back(y, k))
        assert abs(lhs / rhs - 1) < 1e-12


def test_angle_zero_is_column_sums():
    # theta = 0: the ray x = u_b runs along y; with B = nx and db = h, u_b hits column b.
    g = _geom(nx=16, B=16, A=8)
    x = np.random.default_rng(2).random((1, 16, 16, 2))
    y = g.forward(x)
    np.testing.assert_allclose(y[0, 0], 2.0 * x[0].sum(axis=0), rtol=1e-13)


def test_angle_ninety_is_row_sums():
    # theta = 90 deg (a = A/2): the ray y = u_b runs along x and hits row b.
    g = _geom(nx=16, B=16, A=8)
    x = np.random.default_rng(3).random((1, 16, 16, 2))
    y = g.forward(x)
    np.testing.assert_allclose(y[0, 4], 2.0 * x[0].sum(axis=1), rtol=1e-12)


def test_point_projects_onto_its_sinusoid():
    # an off-centre point at (x0, y0) projects onto u = x0 cos(theta) + y0 sin(theta):
    # the profile's centroid must follow that sinusoid (catches sign/transposition errors).
    nx, h = 64, 2.0
    g = _geom(nx=nx, B=96, A=36, vox=h, db=h)
    i0, j0 = 40, 21                      # column, row
    x = np.zeros((1, nx, nx, 1))
    x[0, j0, i0, 0] = 1.0
    y = g.forward(x)[0, :, :, 0]
    u = (np.arange(96) - 47.5) * h
    x0, y0 = (i0 - (nx - 1) / 2) * h, (j0 - (nx - 1) / 2) * h
    for a in range(36):
        th = a * np.pi / 36
        cen = np.sum(u * y[a]) / np.sum(y[a])
        assert abs(cen - (x0 * np.cos(th) + y0 * np.sin(th))) < 1e-9 + 0.5 * h


def test_mass_conserved_for_smooth_object():
    # a smooth blob's projection integrates to its mass at every angle
    nx, h = 64, 2.0
    g = _geom(nx=nx, B=96, A=30, vox=h, db=h)
    c = (np.arange(nx) - (nx - 1) / 2) * h
    X, Y = np.meshgrid(c, c, indexing="xy")
    blob = np.exp(-((X - 7) ** 2 + (Y + 5) ** 2) / (2 * 12.0 ** 2))
    x = blob[None, :, :, None]
    y = g.forward(x)[0, :, :, 0]
    mass = blob.sum() * h * h
    np.testing.assert_allclose(y.sum(axis=1) * h, mass, rtol=2e-3)


def test_subsets_partition_angles():
    g = _geom(A=90, S=4)
    allk = np.sort(np.concatenate(g.subsets))
    np.testing.assert_array_equal(allk, np.arange(90))
    assert [len(s) for s in g.subsets] == [23, 23, 22, 22]
    np.testing.assert_array_equal(g.subsets[1][:3], [1, 5, 9])


@pytest.mark.parametrize("A", [8, 90, 252])
def test_major_axis_rule_is_integer(A):
    # ties at 45 and 135 degrees step over columns
    for a in range(A):
        th = a * np.pi / A
        if 4 * a == A or 4 * a == 3 * A:
            assert P.x_major(a, A)
        elif abs(np.sin(th)) > abs(np.cos(th)) + 1e-12:
            assert P.x_major(a, A)
        elif abs(np.sin(th)) < abs(np.cos(th)) - 1e-12:
            assert not P.x_major(a, A)
