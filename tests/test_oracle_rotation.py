"""Pins of the oracle's rotation accelerations (S5: Coriolis -2 Omega x U and
centrifugal -Omega x (Omega x r) added to the velocity equation), each from a
closed form or an identity that the oracle's component-wise cross products do
not share."""
import numpy as np
import pytest

import inputs as I


@pytest.fixture(scope="module")
def O(oracle):
    return oracle


def grid(O, n, h=None):
    geom = I.geometry(n, ("periodic",) * len(n), ("periodic",) * len(n))
    return O.Grid.make(geom["n"], geom["bclo"], geom["bchi"], h=h)


def centres(g):
    ax = [(np.arange(g.n[d]) + 0.5) * g.h[d] for d in range(3)]
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return x, y, z


def test_coriolis_about_z_closed_form(O):
    g = grid(O, (6, 5, 4))
    rng = np.random.default_rng(1)
    U = [rng.normal(size=g.cell_shape) for _ in range(3)]
    w = 0.7
    F = O.rotation_forces(g, (0.0, 0.0, w), (0.5, 0.5, 0.5), U, centrifugal=False)
    np.testing.assert_allclose(F[0], 2 * w * U[1], rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(F[1], -2 * w * U[0], rtol=1e-15, atol=1e-15)
    assert np.all(F[2] == 0.0)


def test_coriolis_does_no_work(O):
    """a . U = 0 for the Coriolis acceleration, for any Omega."""
    g = grid(O, (5, 6, 7))
    rng = np.random.default_rng(2)
    U = [rng.normal(size=g.cell_shape) for _ in range(3)]
    om = rng.normal(size=3)
    F = O.rotation_forces(g, om, (0.3, 0.4, 0.5), U, centrifugal=False)
    dot = F[0] * U[0] + F[1] * U[1] + F[2] * U[2]
    scale = np.linalg.norm(om) * sum(u ** 2 for u in U)
    assert np.max(np.abs(dot) / scale) < 1e-14


def test_centrifugal_identity(O):
    """-Omega x (Omega x r) = |Omega|^2 r - Omega (Omega . r); about z it is w^2 times
    the distance vector from the axis."""
    g = grid(O, (6, 4, 5), h=(0.1, 0.2, 0.15))
    rng = np.random.default_rng(3)
    zero = [np.zeros(g.cell_shape) for _ in range(3)]
    c = (0.31, 0.42, 0.37)
    x, y, z = centres(g)
    r = [x - c[0], y - c[1], z - c[2]]
    om = rng.normal(size=3)
    F = O.rotation_forces(g, om, c, zero, centrifugal=True)
    od = om[0] * r[0] + om[1] * r[1] + om[2] * r[2]
    want = [om @ om * r[d] - om[d] * od for d in range(3)]
    for d in range(3):
        np.testing.assert_allclose(F[d], want[d], rtol=0, atol=1e-14 * np.abs(want[d]).max())
    w = 1.3
    F = O.rotation_forces(g, (0, 0, w), c, zero, centrifugal=True)
    np.testing.assert_allclose(F[0], w * w * r[0], rtol=1e-14)
    np.testing.assert_allclose(F[1], w * w * r[1], rtol=1e-14)
    assert np.all(F[2] == 0.0)


def test_accumulate_and_scale(O):
    g = grid(O, (4, 4, 4))
    rng = np.random.default_rng(4)
    U = [rng.normal(size=g.cell_shape) for _ in range(3)]
    F0 = [rng.normal(size=g.cell_shape) for _ in range(3)]
    om = (0.2, -0.5, 0.9)
    a = O.rotation_forces(g, om, (0.5,) * 3, U)
    b = O.rotation_forces(g, om, (0.5,) * 3, U, F=F0, alpha=0.25)
    for d in range(3):
        np.testing.assert_allclose(b[d], F0[d] + 0.25 * a[d], rtol=1e-14, atol=1e-15)


def test_two_dimensional_in_plane(O):
    g = grid(O, (8, 6))
    rng = np.random.default_rng(5)
    U = [rng.normal(size=g.cell_shape) for _ in range(2)]
    w = 0.4
    F = O.rotation_forces(g, (0.0, 0.0, w), (0.5, 0.5), U, centrifugal=False)
    assert len(F) == 2
    np.testing.assert_allclose(F[0], 2 * w * U[1], rtol=1e-15)
    np.testing.assert_allclose(F[1], -2 * w * U[0], rtol=1e-15)
