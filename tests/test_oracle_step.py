"""Pins of the oracle's time-step pieces (S2-S3 loop around the two
projections): face velocities from cell velocities and the upwind advective
derivative, against closed forms, the textbook upwind difference and the
telescoping of the flux form; and the composition of one step."""
import numpy as np
import pytest

import inputs as I


@pytest.fixture(scope="module")
def O(oracle):
    return oracle


def G(O, n, lo, hi, h=None):
    geom = I.geometry(n, lo, hi)
    return O.Grid.make(geom["n"], geom["bclo"], geom["bchi"], h=h)


def test_face_average_linear_field(O):
    g = G(O, (8, 5, 4), ("neumann", "periodic", "periodic"), ("dirichlet", "periodic", "periodic"))
    hx = g.h[0]
    x = (np.arange(8) + 0.5) * hx
    Ux = np.broadcast_to(2.0 * x + 1.0, g.cell_shape).copy()
    Uf = O.face_average(g, [Ux, np.zeros(g.cell_shape), np.zeros(g.cell_shape)])
    xf = np.arange(9) * hx
    want = 2.0 * xf + 1.0
    want[0] = 0.0                    # wall
    want[8] = 2.0 * x[7] + 1.0       # outflow: interior value
    np.testing.assert_allclose(Uf[0][0, 0, :], want, rtol=1e-15, atol=1e-15)
    # periodic y: a constant component gives the constant on every face, wrap face included
    Uy = np.full(g.cell_shape, 3.5)
    Uf = O.face_average(g, [np.zeros(g.cell_shape), Uy, np.zeros(g.cell_shape)])
    assert np.all(Uf[1] == 3.5)


def test_advect_uniform_field_is_zero(O):
    g = G(O, (6, 5, 4), ("periodic", "neumann", "dirichlet"), ("periodic", "dirichlet", "neumann"))
    rng = np.random.default_rng(1)
    Uf = [rng.normal(size=g.face_shape(d)) for d in range(3)]
    A = O.advect(g, Uf, np.full(g.cell_shape, 2.25))
    assert np.all(A == 0.0)


def test_advect_linear_field_closed_form(O):
    g = G(O, (10, 3, 3), ("dirichlet", "periodic", "periodic"), ("dirichlet", "periodic", "periodic"))
    hx = g.h[0]
    q = np.broadcast_to((np.arange(10) + 0.5) * hx * 3.0, g.cell_shape).copy()
    for u in (0.7, -0.4):
        Uf = [np.full(g.face_shape(0), u), np.zeros(g.face_shape(1)), np.zeros(g.face_shape(2))]
        A = O.advect(g, Uf, q)
        want = np.full(g.cell_shape, u * 3.0)
        if u > 0:
            want[..., 0] = 0.0       # upwind cell outside: zero gradient
        else:
            want[..., -1] = 0.0
        np.testing.assert_allclose(A, want, rtol=1e-12, atol=1e-12)


def test_advect_textbook_upwind_periodic(O):
    g = G(O, (12, 4, 4), ("periodic",) * 3, ("periodic",) * 3)
    rng = np.random.default_rng(2)
    q = rng.normal(size=g.cell_shape)
    u = 0.9
    Uf = [np.full(g.face_shape(0), u), np.zeros(g.face_shape(1)), np.zeros(g.face_shape(2))]
    A = O.advect(g, Uf, q)
    want = u * (q - np.roll(q, 1, axis=2)) / g.h[0]
    np.testing.assert_allclose(A, want, rtol=1e-13, atol=1e-13)


def test_advect_flux_form_telescopes(O):
    """A + q div(U_adv) is the divergence of upwind fluxes: it sums to 0 on a periodic grid."""
    g = G(O, (6, 7, 5), ("periodic",) * 3, ("periodic",) * 3, h=(0.1, 0.2, 0.3))
    rng = np.random.default_rng(3)
    Uf = [rng.normal(size=g.face_shape(d)) for d in range(3)]
    for d in range(3):   # periodic: face n is face 0
        sl_last = [slice(None)] * 3
        sl_first = [slice(None)] * 3
        sl_last[2 - d], sl_first[2 - d] = -1, 0
        Uf[d][tuple(sl_last)] = Uf[d][tuple(sl_first)]
    q = rng.normal(size=g.cell_shape)
    A = O.advect(g, Uf, q)
    div = sum((np.diff(Uf[d], axis=2 - d)) / g.h[d] for d in range(3))
    total = np.sum(A + q * div)
    assert abs(total) < 1e-12 * np.sum(np.abs(A))


def test_step_composition(O):
    """dt = 0: the step is the nodal projection of U^n; U = 0, S = 0 stays 0; the
    face velocities of a step satisfy the MAC constraint."""
    p = I.stratified(16, seed=5, contrast=1e2)
    g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"])
    r = O.time_step(g, p["sigma"], p["beta0"], p["beta0_face"], p["U_cell"], p["S"], dt=0.0)
    ref = O.nodal_project(g, p["sigma"], p["beta0"], p["U_cell"], p["S"])
    for d in range(3):
        np.testing.assert_allclose(r["U"][d], ref["U"][d], rtol=1e-12, atol=1e-14)
    assert r["mac"]["constraint"] < 1e-9
    z = [np.zeros(g.cell_shape) for _ in range(3)]
    r0 = O.time_step(g, p["sigma"], p["beta0"], p["beta0_face"], z, np.zeros(g.cell_shape), dt=0.1)
    assert all(np.all(u == 0.0) for u in r0["U"])
