"""Pins for the source term of the constraint, Eq. 6 (S2): div(beta0 U) = beta0 S.

The right-hand side of both projections is f = D(beta0 U) - beta0 S (nodal: the
source lumped to the nodes), and the update is U <- U - (sigma/beta0) G phi.
None of the expected values below is formed by the oracle's own right-hand-side
routines; each follows from Eq. 6 and the mathematics alone:

  * with U = 0 the right-hand side is minus the weighted source, cell by cell
    (MAC) or as the plain sum over the cells that touch a node divided by 2^d
    (nodal, written out here with loops);
  * with U = W/beta0_face for a linear field W, D(beta0 U) is the constant
    divergence of W, so f = div W - beta0 S;
  * a laterally uniform column (periodic x and y, slip wall at z = 0, outflow
    at z = 1; sigma, beta0 and S functions of z only, S > 0, U = 0) is a 1-D
    problem: after the projection Eq. 6 says d(beta0 U_z)/dz = beta0 S with zero
    flux through the wall, so the flux at height z is the discrete integral of
    beta0 S from the wall up to z -- positive, i.e. the heated column flows
    upward.  For the MAC projection the flux at z-face k is
    h * sum_{k' < k} beta0_k' S_k'.  For the nodal projection a potential that
    depends on z alone sees L = D_N sigma G_N exactly (the Q1 stiffness of a
    z-only function reduces to the 1-D three-point form), so the projection is
    exact here too and the cell-centred flux of layer k is
    h * (sum_{k' < k} g_k' + g_k / 2), g = beta0 S.

A flipped sign of the source, a dropped or misplaced beta0 weight, a wrong
lumping weight or an update that forgets the division by beta0 each fails one
of these tests.
"""
import itertools

import numpy as np
import pytest


def _column(O, n=(4, 4, 8), seed=0):
    """Laterally uniform column with z-dependent sigma, beta0, S > 0."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    g = O.Grid.make(n, ("periodic", "periodic", "neumann"), ("periodic", "periodic", "dirichlet"))
    h = 1.0 / nz
    zc = (np.arange(nz) + 0.5) * h
    zf = np.arange(nz + 1) * h
    rho = lambda z: 10.0 ** (-2.0 * z)                       # density contrast 1e2
    beta0 = lambda z: rho(z) ** 0.6 * (1.0 + 0.3 * z)          # any positive profile
    s_c = 0.5 + rng.random(nz)                                 # S > 0, one value per layer
    lat = lambda v: np.broadcast_to(v[:, None, None], (v.size, ny, nx)).copy()
    sigma = lat(beta0(zc) / rho(zc))
    b0c = lat(beta0(zc))
    S = lat(s_c)
    b0f = [lat(beta0(zc))[:, :, np.r_[0:nx, 0]],              # x faces: cell value on either side
           lat(beta0(zc))[:, np.r_[0:ny, 0], :],
           lat(beta0(zf))]
    return g, h, sigma, b0c, b0f, S, beta0(zc) * s_c, beta0(zf)


def test_mac_rhs_of_zero_velocity_is_minus_beta0_S(oracle):
    O = oracle
    rng = np.random.default_rng(1)
    for lo, hi in [(("periodic",) * 3, ("periodic",) * 3),
                   (("neumann", "dirichlet", "periodic"), ("dirichlet", "neumann", "periodic"))]:
        g = O.Grid.make((5, 4, 3), lo, hi)
        b0c = np.exp(rng.normal(size=g.cell_shape))
        b0f = [np.exp(rng.normal(size=g.face_shape(d))) for d in range(3)]
        S = rng.normal(size=g.cell_shape)
        U = [np.zeros(g.face_shape(d)) for d in range(3)]
        f = O.mac_rhs(g, b0c, b0f, U, S)
        np.testing.assert_allclose(f, -b0c * S, rtol=0, atol=1e-15)


def test_mac_rhs_of_linear_flux(oracle):
    """beta0_face U = W with W_d = a_d x_d + c_d: D(W) = a_x + a_y + a_z on every
    cell of a fully Neumann box (boundary faces carry the field's own value)."""
    O = oracle
    rng = np.random.default_rng(2)
    n = (4, 5, 6)
    h = tuple(1.0 / v for v in n)
    g = O.Grid.make(n, ("neumann",) * 3, ("neumann",) * 3)
    a = np.array([0.7, -1.3, 2.1])
    c = np.array([0.2, 0.4, -0.1])
    U, b0f = [], []
    for d in range(3):
        shp = g.face_shape(d)
        pos = np.indices(shp)[2 - d] * h[d]                     # face coordinate along d
        W = a[d] * pos + c[d]
        bf = np.exp(rng.normal(size=shp))
        b0f.append(bf)
        U.append(W / bf)
    b0c = np.exp(rng.normal(size=g.cell_shape))
    S = rng.normal(size=g.cell_shape)
    f = O.mac_rhs(g, b0c, b0f, U, S)
    np.testing.assert_allclose(f, a.sum() - b0c * S, rtol=0, atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_nodal_rhs_of_zero_velocity_is_minus_lumped_beta0_S(oracle, dim):
    O = oracle
    rng = np.random.default_rng(3)
    combos = [(("periodic",) * dim, ("periodic",) * dim),
              (("neumann", "dirichlet", "periodic")[:dim], ("dirichlet", "neumann", "periodic")[:dim])]
    for lo, hi in combos:
        g = O.Grid.make((4, 3, 5)[:dim], lo, hi)
        b0 = np.exp(rng.normal(size=g.cell_shape))
        S = rng.normal(size=g.cell_shape)
        U = [np.zeros(g.cell_shape) for _ in range(dim)]
        f = O.nodal_rhs(g, b0, U, S)
        # brute force: every node gathers beta0 S / 2^d from each cell it touches
        want = np.zeros(g.node_shape)
        n = g.n
        for k, j, i in itertools.product(range(n[2]), range(n[1]), range(n[0])):
            for oz, oy, ox in itertools.product(range(2 if dim == 3 else 1), range(2), range(2)):
                p = [i + ox, j + oy, k + oz]
                for d in range(dim):
                    if g.bclo[d] == "periodic":
                        p[d] %= n[d]
                want[p[2], p[1], p[0]] += b0[k, j, i] * S[k, j, i] / 2 ** dim
        for d in range(dim):                                     # Dirichlet nodes are not unknowns
            sl = [slice(None)] * 3
            if g.bclo[d] == "dirichlet":
                sl[2 - d] = 0
                want[tuple(sl)] = 0.0
            if g.bchi[d] == "dirichlet":
                sl[2 - d] = -1
                want[tuple(sl)] = 0.0
        np.testing.assert_allclose(f, -want, rtol=0, atol=1e-14)


def test_mac_column_flux_is_integral_of_beta0_S(oracle):
    O = oracle
    g, h, sigma, b0c, b0f, S, g1d, b0zf = _column(O)
    U = [np.zeros(g.face_shape(d)) for d in range(3)]
    r = O.mac_project(g, sigma, b0c, b0f, U, S, dense=True)
    flux = h * np.concatenate([[0.0], np.cumsum(g1d)])          # at z-faces 0..nz
    want_uz = flux / b0zf
    Uz = r["U"][2]
    assert Uz.shape[0] == flux.size
    for k in range(flux.size):
        np.testing.assert_allclose(Uz[k], want_uz[k], rtol=1e-12, atol=1e-15)
    assert (Uz[1:] > 0).all()                                   # heated column rises
    np.testing.assert_allclose(r["U"][0], 0.0, atol=1e-13)
    np.testing.assert_allclose(r["U"][1], 0.0, atol=1e-13)


def test_nodal_column_flux_is_integral_of_beta0_S(oracle):
    O = oracle
    g, h, sigma, b0c, b0f, S, g1d, _ = _column(O, seed=1)
    U = [np.zeros(g.cell_shape) for _ in range(3)]
    r = O.nodal_project(g, sigma, b0c, U, S, dense=True)
    flux_c = h * (np.concatenate([[0.0], np.cumsum(g1d)[:-1]]) + 0.5 * g1d)   # at cell centres
    want_uz = flux_c / b0c[:, 0, 0]
    Uz = r["U"][2]
    for k in range(g.n[2]):
        np.testing.assert_allclose(Uz[k], want_uz[k], rtol=1e-12, atol=1e-15)
    assert (Uz > 0).all()
    np.testing.assert_allclose(r["U"][0], 0.0, atol=1e-13)
    np.testing.assert_allclose(r["U"][1], 0.0, atol=1e-13)
    # the approximate projection is exact for a z-only potential
    assert r["constraint"] < 1e-12
