"""Pins for the oracle's cell-centred (MAC) system, each independent of the oracle itself.

The operator is the reading of Eq. 6 (S2) described in oracle/mg_oracle.c.  What
pins it here:
  * closed-form discrete eigenfunctions for every boundary kind (operator,
    boundary treatment and h scaling, anisotropic spacing included);
  * second-order convergence to a manufactured smooth solution (S3: the
    projection method is second order) with a variable coefficient, which also
    pins the harmonic face coefficients;
  * closed forms for D (divergence of a linear field) and G (gradient of a
    linear potential);
  * brute force: dense LU versus multigrid on tiny grids, all boundary mixes;
  * invariants: symmetry, constant null space, L = D B G, exactness and
    idempotence of the MAC projection.
"""
import itertools

import numpy as np
import pytest

import inputs as I

BCS = ["periodic", "neumann", "dirichlet"]


def _grid(O, n, lo, hi, h=None):
    return O.Grid.make(n, lo, hi, h)


def _axis_mode(kind_lo, kind_hi, m, n, h):
    """(1-D mode at cell centres, eigenvalue contribution) for a cell-centred
    second difference with the given boundary pair."""
    x = (np.arange(n) + 0.5) * h
    L = n * h
    if kind_lo == "periodic":
        v = np.cos(2 * np.pi * m * x / L)
        lam = -(4 / h ** 2) * np.sin(np.pi * m * h / L) ** 2
    elif (kind_lo, kind_hi) == ("neumann", "neumann"):
        v = np.cos(m * np.pi * x / L)
        lam = -(4 / h ** 2) * np.sin(m * np.pi * h / (2 * L)) ** 2
    elif (kind_lo, kind_hi) == ("dirichlet", "dirichlet"):
        v = np.sin(m * np.pi * x / L)
        lam = -(4 / h ** 2) * np.sin(m * np.pi * h / (2 * L)) ** 2
    elif (kind_lo, kind_hi) == ("neumann", "dirichlet"):
        k = (m + 0.5) * np.pi / L
        v = np.cos(k * x)
        lam = -(4 / h ** 2) * np.sin(k * h / 2) ** 2
    else:  # dirichlet lo, neumann hi
        k = (m + 0.5) * np.pi / L
        v = np.sin(k * x)
        lam = -(4 / h ** 2) * np.sin(k * h / 2) ** 2
    return v, lam


PAIRS = [("periodic", "periodic"), ("neumann", "neumann"), ("dirichlet", "dirichlet"),
         ("neumann", "dirichlet"), ("dirichlet", "neumann")]


@pytest.mark.parametrize("dim", [2, 3])
def test_eigenfunctions_every_boundary_pair(oracle, dim):
    O = oracle
    rng = np.random.default_rng(1)
    n = (8, 6, 4)[:dim]
    h = (0.125, 0.2, 0.3)[:dim]
    for combo in itertools.product(PAIRS, repeat=dim):
        lo = tuple(c[0] for c in combo)
        hi = tuple(c[1] for c in combo)
        g = _grid(O, n, lo, hi, h)
        sigma = np.full(g.cell_shape, 2.5)
        B = O.mac_faces(g, sigma)
        phi = np.ones(g.cell_shape)
        lam = 0.0
        for d in range(dim):
            m = int(rng.integers(1, 3))
            v, l = _axis_mode(lo[d], hi[d], m, n[d], h[d])
            shape = [1, 1, 1]
            shape[2 - d] = n[d]
            phi = phi * v.reshape(shape)
            lam += l
        Lphi = O.mac_apply(g, B, phi)
        np.testing.assert_allclose(Lphi, 2.5 * lam * phi, rtol=0, atol=1e-10 * abs(lam))


def test_eigenfunction_solution_is_exact(oracle):
    """For f an eigenfunction, the discrete solution is f / lambda (dense and MG)."""
    O = oracle
    n, h = 16, 1 / 16
    g = _grid(O, (n, n, n), ("periodic", "periodic", "neumann"), ("periodic", "periodic", "dirichlet"))
    B = O.mac_faces(g, np.ones(g.cell_shape))
    vx, lx = _axis_mode("periodic", "periodic", 1, n, h)
    vy, ly = _axis_mode("periodic", "periodic", 2, n, h)
    vz, lz = _axis_mode("neumann", "dirichlet", 0, n, h)
    f = vz[:, None, None] * vy[None, :, None] * vx[None, None, :]
    phi, st = O.mac_solve_mg(g, B, f)
    exact = f / (lx + ly + lz)
    assert st["relres"] < 1e-13
    np.testing.assert_allclose(phi, exact, atol=1e-12 * np.abs(exact).max())


def test_manufactured_second_order(oracle):
    """2-D stratified manufactured solution: error falls ~4x per refinement."""
    O = oracle
    errs = []
    for n in (16, 32, 64, 128):
        p = I.manufactured_2d(n)
        g = _grid(O, (n, n), ("periodic", "neumann"), ("periodic", "neumann"))
        B = O.mac_faces(g, p["sigma"])
        phi, st = O.mac_solve_mg(g, B, p["f"])
        assert st["relres"] < 1e-12
        ex = p["phi_exact"] - p["phi_exact"].mean()
        errs.append(np.sqrt(np.mean((phi - phi.mean() - ex) ** 2)))
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(orders) > 1.9, orders


def test_div_and_grad_closed_forms(oracle):
    """D of a linear face field is its constant slope; G of a linear potential
    (Dirichlet-free, interior faces) is its slope."""
    O = oracle
    n = (6, 5, 4)
    h = (0.5, 0.25, 0.2)
    g = _grid(O, n, ("neumann",) * 3, ("neumann",) * 3, h)
    a = (1.5, -2.0, 0.75)
    V = []
    for d in range(3):
        xf = np.arange(n[d] + 1) * h[d]
        shape = [1, 1, 1]
        shape[2 - d] = n[d] + 1
        V.append(np.broadcast_to((a[d] * xf).reshape(shape), g.face_shape(d)).copy())
    np.testing.assert_allclose(O.mac_div(g, V), sum(a), rtol=1e-13)
    xc = [(np.arange(n[d]) + 0.5) * h[d] for d in range(3)]
    phi = (a[0] * xc[0][None, None, :] + a[1] * xc[1][None, :, None] + a[2] * xc[2][:, None, None]) * np.ones(g.cell_shape)
    B = [np.ones(g.face_shape(d)) for d in range(3)]
    U0 = [np.zeros(g.face_shape(d)) for d in range(3)]
    Un = O.mac_grad_update(g, B, B, phi, U0)   # = -G phi with B = beta0 = 1
    for d in range(3):
        sl = [slice(None)] * 3
        sl[2 - d] = slice(1, n[d])
        np.testing.assert_allclose(-Un[d][tuple(sl)], a[d], rtol=1e-12)
        # wall (Neumann) faces carry no gradient
        sl[2 - d] = 0
        assert np.all(Un[d][tuple(sl)] == 0.0)


def test_harmonic_faces(oracle):
    O = oracle
    g = _grid(O, (3, 2), ("periodic", "dirichlet"), ("periodic", "neumann"))
    s = np.array([[[1.0, 2.0, 4.0], [3.0, 5.0, 7.0]]])
    Bx, By = O.mac_faces(g, s)
    hm = lambda a, b: 2 * a * b / (a + b)
    assert Bx[0, 0, 1] == pytest.approx(hm(1, 2))
    assert Bx[0, 0, 0] == pytest.approx(hm(4, 1)) and Bx[0, 0, 3] == pytest.approx(hm(4, 1))
    assert By[0, 0, 2] == pytest.approx(4.0)          # boundary face: interior sigma
    assert By[0, 1, 1] == pytest.approx(hm(2, 5))
    assert By[0, 2, 0] == pytest.approx(3.0)


@pytest.mark.parametrize("n", [(4, 4), (8, 8), (4, 4, 4), (6, 6, 6)])
def test_dense_matches_multigrid(oracle, n):
    O = oracle
    dim = len(n)
    rng = np.random.default_rng(sum(n))
    combos = list(itertools.product(PAIRS, repeat=dim))
    for combo in combos[:: (1 if dim == 2 else 7)]:
        lo = tuple(c[0] for c in combo)
        hi = tuple(c[1] for c in combo)
        g = _grid(O, n, lo, hi)
        sigma = np.exp(rng.normal(size=g.cell_shape))
        B = O.mac_faces(g, sigma)
        f = rng.normal(size=g.cell_shape)
        pd = O.mac_solve_dense(g, B, f)
        pm, st = O.mac_solve_mg(g, B, f)
        if g.singular:
            pm = pm - pm.mean()
        assert np.linalg.norm(pd - pm) <= 1e-12 * np.linalg.norm(pd), (lo, hi)


def test_symmetry_and_null_space(oracle):
    O = oracle
    rng = np.random.default_rng(7)
    for combo in itertools.product(PAIRS, repeat=3):
        lo = tuple(c[0] for c in combo)
        hi = tuple(c[1] for c in combo)
        g = _grid(O, (5, 4, 6), lo, hi, (0.2, 0.3, 0.1))
        B = O.mac_faces(g, np.exp(rng.normal(size=g.cell_shape)))
        u, v = rng.normal(size=(2,) + g.cell_shape)
        a = np.sum(O.mac_apply(g, B, u) * v)
        b = np.sum(u * O.mac_apply(g, B, v))
        assert abs(a - b) <= 1e-13 * (abs(a) + abs(b) + 1)
        one = O.mac_apply(g, B, np.ones(g.cell_shape))
        if g.singular:
            assert np.abs(one).max() < 1e-12
        else:
            assert np.abs(one).max() > 1e-3


def test_L_equals_D_B_G(oracle):
    O = oracle
    rng = np.random.default_rng(3)
    for combo in itertools.product(PAIRS, repeat=3):
        lo = tuple(c[0] for c in combo)
        hi = tuple(c[1] for c in combo)
        g = _grid(O, (4, 5, 3), lo, hi, (0.25, 0.2, 1 / 3))
        B = O.mac_faces(g, np.exp(rng.normal(size=g.cell_shape)))
        phi = rng.normal(size=g.cell_shape)
        ones = [np.ones(g.face_shape(d)) for d in range(3)]
        zero = [np.zeros(g.face_shape(d)) for d in range(3)]
        BG = [-u for u in O.mac_grad_update(g, B, ones, phi, zero)]
        np.testing.assert_allclose(O.mac_div(g, BG), O.mac_apply(g, B, phi), atol=1e-11 * np.abs(phi).max() * 100)


def test_projection_exact_and_idempotent(oracle):
    """Post-MAC D(beta0 U) - beta0 S equals the solver residual; with the
    dense solve it vanishes to round-off; a second projection is a no-op."""
    O = oracle
    p = I.stratified(8, seed=11, contrast=1e3)
    g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"])
    r = O.mac_project(g, p["sigma"], p["beta0"], p["beta0_face"], p["U_mac"], p["S"], dense=True)
    assert r["constraint"] < 1e-11
    r2 = O.mac_project(g, p["sigma"], p["beta0"], p["beta0_face"], r["U"], p["S"], dense=True)
    for u1, u2 in zip(r["U"], r2["U"]):
        assert np.abs(u1 - u2).max() <= 1e-12 * np.abs(u1).max()
    # MG projection reaches the same U
    rm = O.mac_project(g, p["sigma"], p["beta0"], p["beta0_face"], p["U_mac"], p["S"], dense=False)
    assert rm["relres"] < 1e-13
    for u1, u2 in zip(r["U"], rm["U"]):
        assert np.abs(u1 - u2).max() <= 1e-11 * np.abs(u1).max()
    # the constraint residual equals the solver residual in norm
    Bf = O.mac_faces(g, p["sigma"])
    f = O.mac_rhs(g, p["beta0"], p["beta0_face"], p["U_mac"], p["S"])
    res = f - O.mac_apply(g, Bf, rm["phi"])
    div = O.mac_rhs(g, p["beta0"], p["beta0_face"], rm["U"], p["S"])
    np.testing.assert_allclose(div, res, atol=1e-9 * np.abs(f).max())
