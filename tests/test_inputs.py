"""Pins for the seeded input generators.

* beta0 of Eq. 5 (S2): the closed form used by the generators,
  rho0(0) (p0/p0(0))^(1/Gamma1), against a trapezoid quadrature of the
  integral in Eq. 5 for the isothermal and polytropic base states;
* hydrostatic equilibrium (Eq. 4) of the isothermal profile;
* the Lane-Emden integrator against its closed-form solutions for n = 0, 1, 5
  and the classical first zero xi_1 = 6.89685 of n = 3 (Chandrasekhar 1939,
  "An Introduction to the Study of Stellar Structure", ch. IV, table 4);
* seeded determinism, periodic face copies and wall faces of the velocities.
"""
import math

import numpy as np
import pytest

import inputs as I


def _beta0_quadrature(r, p0, rho0_0, gamma1):
    """Eq. 5 evaluated by the trapezoid rule on the tabulated p0(r)."""
    dpdr = np.gradient(p0, r, edge_order=2)
    integrand = dpdr / (gamma1 * p0)
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (integrand[1:] + integrand[:-1]) * np.diff(r))])
    return rho0_0 * np.exp(cum)


def test_beta0_closed_form_isothermal():
    # isothermal: p0 = c^2 rho0, rho0 = exp(-z/H); hydrostatic with g = c^2 / H
    H, c2 = 0.25, 2.0
    z = np.linspace(0.0, 1.0, 10001)
    rho0 = np.exp(-z / H)
    p0 = c2 * rho0
    # Eq. 4: dp0/dz = -rho0 g
    g = c2 / H
    assert np.max(np.abs(np.gradient(p0, z, edge_order=2) + rho0 * g)) < 1e-6
    quad = _beta0_quadrature(z, p0, 1.0, I.GAMMA1)
    closed = rho0 ** (1.0 / I.GAMMA1)
    assert np.max(np.abs(quad - closed) / closed) < 1e-6
    # the generator's beta0
    p = I.manufactured_2d(64, H)
    y = (np.arange(64) + 0.5) / 64
    np.testing.assert_allclose(p["beta0"][0, :, 0], np.exp(-y / H) ** (1 / I.GAMMA1), rtol=1e-14)


def test_beta0_closed_form_polytrope():
    xe, xi, th = I.polytrope_profile(1e4, 3.0)
    r = xi / xe * 0.5
    rho = th ** 3
    p0 = rho ** (4.0 / 3.0)
    quad = _beta0_quadrature(r[10:], p0[10:], rho[10] ** 0.8, I.GAMMA1)
    closed = rho[10:] ** 0.8
    assert np.max(np.abs(quad - closed) / closed) < 1e-6
    assert th[-1] ** 3 == pytest.approx(1e-4, rel=1e-3)


@pytest.mark.parametrize("n,exact", [
    (0.0, lambda x: 1 - x ** 2 / 6),
    (1.0, lambda x: np.sin(x) / x),
    (5.0, lambda x: 1 / np.sqrt(1 + x ** 2 / 3)),
])
def test_lane_emden_closed_forms(n, exact):
    xi, th = I.lane_emden(n, 2.4, 1e-3)
    m = xi > 0
    np.testing.assert_allclose(th[m], exact(xi[m]), atol=1e-9)


def test_lane_emden_n3_first_zero():
    xi, th = I.lane_emden(3.0, 7.0, 1e-4)
    assert xi[-1] == pytest.approx(6.89685, abs=2e-4)


def test_stratified_fields():
    a = I.stratified(8, seed=3, contrast=1e3)
    b = I.stratified(8, seed=3, contrast=1e3)
    for u, v in zip(a["U_mac"], b["U_mac"]):
        assert np.array_equal(u, v)
    rho = a["rho"][:, 0, 0]
    # contrast between the bottom and top faces of the domain
    assert math.exp(math.log(rho[0]) + (math.log(rho[0]) - math.log(rho[1])) / 2) / \
        math.exp(math.log(rho[-1]) - (math.log(rho[0]) - math.log(rho[1])) / 2) == pytest.approx(1e3)
    np.testing.assert_allclose(a["sigma"], a["beta0"] / a["rho"])
    Ux, Uy, Uz = a["U_mac"]
    assert np.array_equal(Ux[:, :, 0], Ux[:, :, -1]) and np.array_equal(Uy[:, 0, :], Uy[:, -1, :])
    assert np.all(Uz[0] == 0.0) and np.any(Uz[-1] != 0.0)
    assert abs(np.std(Ux) - 1e-2) < 2e-3
    # beta0 at z faces follows the closed form at the face heights
    ze = np.arange(9) / 8
    np.testing.assert_allclose(a["beta0_face"][2][:, 0, 0], 1e3 ** (-ze / I.GAMMA1), rtol=1e-13)


def test_polytrope_star_fields():
    p = I.polytrope_star(16, seed=5)
    r = p["rho"]
    assert r.max() < 1.0 and r.max() > 0.5
    assert r.min() == pytest.approx(1e-4, rel=1e-2)
    for u, d in zip(p["U_mac"], range(3)):
        sl = [slice(None)] * 3
        sl[2 - d] = 0
        # phi = 0 (outflow) on every face: boundary faces carry random flux
        assert np.any(u[tuple(sl)] != 0.0)


def test_batch_specs_and_arrivals():
    s = I.batch_specs(64, seed=4)
    assert len(s) == 64 and {x["n"] for x in s} <= {32, 64, 96, 128}
    assert all(10.0 <= x["contrast"] <= 1e4 for x in s)
    assert s == I.batch_specs(64, seed=4)
    t, ns = I.poisson_arrivals(100.0, 512, seed=5)
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0) and abs(np.mean(np.diff(t)) - 0.01) < 0.002
