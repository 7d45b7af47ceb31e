"""Pins for the oracle's nodal (Q1 finite-element) system.

Reading of the nodal projection of the second-order projection method (S3):
Q1 elements with sigma constant per cell; see oracle/mg_oracle.c.  What pins it:
  * the textbook constant-coefficient Q1 stencils (3-D: centre -8/3, face
    neighbours 0, edges 1/6, corners 1/12; 2-D: (1/3)[1 1 1; 1 -8 1; 1 1 1]);
  * closed-form discrete eigenvalues (tensor product of the 1-D stiffness
    symbol 2 - 2 cos(theta) and mass symbol (2 + cos(theta))/3), for every
    boundary kind, with the half-weight rows of natural-boundary nodes;
  * closed forms for D_N of a linear field and G_N of a linear potential;
  * the adjoint relation D_N = -G_N^T and conservation of the lumped source;
  * second-order convergence to a manufactured solution;
  * brute force (dense LU) against multigrid; symmetry; constant null space.
"""
import itertools

import numpy as np
import pytest

PAIRS = [("periodic", "periodic"), ("neumann", "neumann"), ("dirichlet", "dirichlet"),
         ("neumann", "dirichlet"), ("dirichlet", "neumann")]


def _delta_row(O, g, sigma, pos):
    phi = np.zeros(g.node_shape)
    phi[pos] = 1.0
    return O.nodal_apply(g, sigma, phi)


def test_q1_stencil_3d(oracle):
    O = oracle
    n, h, s = 6, 0.5, 3.0
    g = O.Grid.make((n, n, n), ("periodic",) * 3, ("periodic",) * 3, (h, h, h))
    row = _delta_row(O, g, np.full(g.cell_shape, s), (3, 3, 3))
    want = np.zeros_like(row)
    for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
        m = abs(dx) + abs(dy) + abs(dz)
        want[3 + dz, 3 + dy, 3 + dx] = {0: -8 / 3, 1: 0.0, 2: 1 / 6, 3: 1 / 12}[m] * s / h ** 2
    np.testing.assert_allclose(row, want, atol=1e-13)


def test_q1_stencil_2d(oracle):
    O = oracle
    n, h, s = 6, 0.25, 0.7
    g = O.Grid.make((n, n), ("periodic",) * 2, ("periodic",) * 2, (h, h))
    row = _delta_row(O, g, np.full(g.cell_shape, s), (0, 2, 2))
    want = np.zeros_like(row)
    want[0, 1:4, 1:4] = s / (3 * h ** 2)
    want[0, 2, 2] = -8 * s / (3 * h ** 2)
    np.testing.assert_allclose(row, want, atol=1e-12)


def _node_mode(lo, hi, m, n, h):
    x = np.arange(n + (0 if lo == "periodic" else 1)) * h
    L = n * h
    w = np.ones_like(x)
    if lo == "periodic":
        th = 2 * np.pi * m / n
        return np.cos(2 * np.pi * m * x / L), th, w
    if (lo, hi) == ("neumann", "neumann"):
        v, th = np.cos(m * np.pi * x / L), m * np.pi / n
    elif (lo, hi) == ("dirichlet", "dirichlet"):
        v, th = np.sin(m * np.pi * x / L), m * np.pi / n
    elif (lo, hi) == ("neumann", "dirichlet"):
        v, th = np.cos((m + 0.5) * np.pi * x / L), (m + 0.5) * np.pi / n
    else:
        v, th = np.sin((m + 0.5) * np.pi * x / L), (m + 0.5) * np.pi / n
    if lo == "neumann":
        w[0] = 0.5
    if hi == "neumann":
        w[-1] = 0.5
    return v, th, w


@pytest.mark.parametrize("dim", [2, 3])
def test_nodal_eigenfunctions(oracle, dim):
    O = oracle
    rng = np.random.default_rng(5)
    n = (8, 6, 4)[:dim]
    h = (0.125, 0.2, 0.3)[:dim]
    for combo in itertools.product(PAIRS, repeat=dim):
        lo = tuple(c[0] for c in combo)
        hi = tuple(c[1] for c in combo)
        g = O.Grid.make(n, lo, hi, h)
        phi = np.ones(g.node_shape)
        wt = np.ones(g.node_shape)
        ths = []
        for d in range(dim):
            m = int(rng.integers(1, 3))
            v, th, w = _node_mode(lo[d], hi[d], m, n[d], h[d])
            shape = [1, 1, 1]
            shape[2 - d] = len(v)
            phi = phi * v.reshape(shape)
            wt = wt * w.reshape(shape)
            ths.append(th)
        lam = 0.0
        for d in range(dim):
            t = (2 - 2 * np.cos(ths[d])) / h[d] ** 2
            for e in range(dim):
                if e != d:
                    t *= (2 + np.cos(ths[e])) / 3
            lam -= t
        sig = 1.7
        Lphi = O.nodal_apply(g, np.full(g.cell_shape, sig), phi)
        want = sig * lam * wt * phi
        want[g.dirichlet_node_mask()] = 0.0
        np.testing.assert_allclose(Lphi, want, atol=1e-10 * abs(lam) * sig)


def test_div_grad_lump_closed_forms(oracle):
    O = oracle
    n, h = (5, 4, 6), (0.2, 0.25, 0.5)
    g = O.Grid.make(n, ("neumann", "dirichlet", "neumann"), ("neumann", "neumann", "dirichlet"), h)
    a = (0.5, -1.25, 2.0)
    xc = [(np.arange(n[d]) + 0.5) * h[d] for d in range(3)]
    shp = lambda d, v: v.reshape([len(v) if 2 - k == d else 1 for k in range(3)])
    V = [np.broadcast_to(shp(d, a[d] * xc[d]), g.cell_shape).copy() for d in range(3)]
    D = O.nodal_div(g, V)
    np.testing.assert_allclose(D[1:-1, 1:-1, 1:-1], sum(a), rtol=1e-12)
    xn = [np.arange(n[d] + 1) * h[d] for d in range(3)]
    phi = sum(np.broadcast_to(shp(d, a[d] * xn[d]), g.node_shape) for d in range(3)).copy()
    # G_N treats Dirichlet nodes as 0: check cells away from the Dirichlet faces
    G = O.nodal_grad(g, phi)
    for d in range(3):
        np.testing.assert_allclose(G[d][:-1, 1:, :], a[d], rtol=1e-12)
    lump = O.nodal_lump(g, np.full(g.cell_shape, 2.5))
    np.testing.assert_allclose(lump[1:-1, 1:-1, 1:-1], 2.5, rtol=1e-14)


def test_adjoint_and_conservation(oracle):
    O = oracle
    rng = np.random.default_rng(2)
    for combo in itertools.product(PAIRS, repeat=3):
        lo = tuple(c[0] for c in combo)
        hi = tuple(c[1] for c in combo)
        g = O.Grid.make((4, 5, 4), lo, hi, (0.25, 0.2, 0.25))
        V = [rng.normal(size=g.cell_shape) for _ in range(3)]
        phi = rng.normal(size=g.node_shape)
        phi[g.dirichlet_node_mask()] = 0.0
        a = np.sum(O.nodal_div(g, V) * phi)
        G = O.nodal_grad(g, phi)
        b = -sum(np.sum(v * gg) for v, gg in zip(V, G))
        assert abs(a - b) <= 1e-12 * (abs(a) + 1)
        if g.singular:
            gc = rng.normal(size=g.cell_shape)
            assert abs(O.nodal_lump(g, gc).sum() - gc.sum()) < 1e-12
            assert abs(O.nodal_div(g, V).sum()) < 1e-11


def test_symmetry_and_null_space(oracle):
    O = oracle
    rng = np.random.default_rng(9)
    for combo in itertools.product(PAIRS, repeat=3):
        lo = tuple(c[0] for c in combo)
        hi = tuple(c[1] for c in combo)
        g = O.Grid.make((4, 4, 6), lo, hi, (0.25, 0.25, 0.25))
        sig = np.exp(rng.normal(size=g.cell_shape))
        mask = g.dirichlet_node_mask()
        u, v = rng.normal(size=(2,) + g.node_shape)
        u[mask] = 0
        v[mask] = 0
        a = np.sum(O.nodal_apply(g, sig, u) * v)
        b = np.sum(u * O.nodal_apply(g, sig, v))
        assert abs(a - b) <= 1e-13 * (abs(a) + abs(b) + 1)
        if g.singular:
            assert np.abs(O.nodal_apply(g, sig, np.ones(g.node_shape))).max() < 1e-12


@pytest.mark.parametrize("n", [(4, 4), (8, 8), (4, 4, 4), (6, 6, 6)])
def test_dense_matches_multigrid(oracle, n):
    O = oracle
    dim = len(n)
    rng = np.random.default_rng(31 + sum(n))
    combos = list(itertools.product(PAIRS, repeat=dim))
    for combo in combos[:: (1 if dim == 2 else 11)]:
        lo = tuple(c[0] for c in combo)
        hi = tuple(c[1] for c in combo)
        g = O.Grid.make(n, lo, hi)
        sig = np.exp(rng.normal(size=g.cell_shape))
        f = rng.normal(size=g.node_shape)
        f[g.dirichlet_node_mask()] = 0.0
        pd = O.nodal_solve_dense(g, sig, f)
        pm, st = O.nodal_solve_mg(g, sig, f)
        mask = ~g.dirichlet_node_mask()
        if g.singular:
            pm = pm - pm[mask].mean()
        assert np.linalg.norm(pd - pm) <= 1e-12 * np.linalg.norm(pd), (lo, hi)


def test_manufactured_second_order(oracle):
    """phi = cos(2 pi x) cos(2 pi y), sigma = exp(1.6 y), periodic x / natural y:
    nodal error falls ~4x per refinement."""
    O = oracle
    errs = []
    for n in (16, 32, 64, 128):
        g = O.Grid.make((n, n), ("periodic", "neumann"), ("periodic", "neumann"))
        h = 1.0 / n
        yc = (np.arange(n) + 0.5) * h
        sig = np.broadcast_to(np.exp(1.6 * yc)[None, :, None], g.cell_shape).copy()
        xn = np.arange(n) * h
        yn = np.arange(n + 1) * h
        X, Y = xn[None, None, :], yn[None, :, None]
        phi = np.cos(2 * np.pi * X) * np.cos(2 * np.pi * Y)
        s = np.exp(1.6 * Y)
        f = -8 * np.pi ** 2 * s * phi + 1.6 * s * (-2 * np.pi * np.cos(2 * np.pi * X) * np.sin(2 * np.pi * Y))
        w = np.ones(n + 1)
        w[0] = w[-1] = 0.5
        f = f * w[None, :, None]
        ph, st = O.nodal_solve_mg(g, sig, f)
        assert st["relres"] < 1e-12
        wt = np.broadcast_to(w[None, :, None], g.node_shape)
        ex = phi - np.sum(phi * wt) / np.sum(wt)
        ph = ph - np.sum(ph * wt) / np.sum(wt)
        errs.append(np.sqrt(np.mean((ph - ex) ** 2)))
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(orders) > 1.9, orders


def test_projection_update(oracle):
    import inputs as I
    O = oracle
    p = I.stratified(8, seed=21, contrast=1e2)
    g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"])
    r = O.nodal_project(g, p["sigma"], p["beta0"], p["U_cell"], p["S"], dense=True)
    rm = O.nodal_project(g, p["sigma"], p["beta0"], p["U_cell"], p["S"], dense=False)
    assert rm["relres"] < 1e-13
    np.testing.assert_allclose(rm["phi"], r["phi"], atol=1e-12 * np.abs(r["phi"]).max())
    G = O.nodal_grad(g, r["phi"])
    for d in range(3):
        np.testing.assert_allclose(r["U"][d], p["U_cell"][d] - p["sigma"] / p["beta0"] * G[d], atol=1e-15)
    f = O.nodal_rhs(g, p["beta0"], p["U_cell"], p["S"])
    assert np.linalg.norm(f - O.nodal_apply(g, p["sigma"], r["phi"])) < 1e-11 * np.linalg.norm(f)
    # approximate projection: the nodal divergence constraint falls a lot but not to round-off
    assert r["constraint"] < 0.5 * np.linalg.norm(f[~g.dirichlet_node_mask()]) / r["src_norm"]
