"""Pins for the base-state oracle (Eq. 5 and the radial mapping).

* constant Gamma1: the trapezoid rule in ln p0 telescopes, so beta0 equals the
  closed form rho0(0) (p0/p0(0))^(1/Gamma1) of Eq. 5 to round-off (isothermal
  and polytropic base states);
* variable Gamma1 with a closed-form integral: second-order convergence;
* mapping: a linear radial table is interpolated exactly; points beyond the
  table take its end values; spherical and plane-parallel radii.
"""
import numpy as np
import pytest


def test_beta0_closed_forms(oracle):
    O = oracle
    r = np.linspace(0.0, 1.0, 1001)
    rho = np.exp(-r / 0.25)                      # isothermal, p0 = c^2 rho
    b = O.beta0_eq5(3.0 * rho, 1.0)
    np.testing.assert_allclose(b, rho ** 0.6, rtol=1e-13)
    th = 1.0 - 0.9 * r ** 2                      # any rho profile, p0 = K rho^(4/3)
    rho_p = th ** 3
    b = O.beta0_eq5(2.0 * rho_p ** (4.0 / 3.0), rho_p[0], g1=5.0 / 3.0)
    np.testing.assert_allclose(b, rho_p[0] * (rho_p / rho_p[0]) ** 0.8, rtol=1e-12)


def test_beta0_variable_gamma_second_order(oracle):
    O = oracle
    a, c = 0.6, 0.3                               # 1/Gamma1 = a + c r, ln p0 = -r^2
    errs = []
    for nr in (101, 201, 401, 801):
        r = np.linspace(0.0, 1.0, nr)
        b = O.beta0_eq5(np.exp(-r ** 2), 2.0, gamma1=1.0 / (a + c * r))
        exact = 2.0 * np.exp(-(a * r ** 2 + 2.0 * c * r ** 3 / 3.0))
        errs.append(np.abs(b - exact).max())
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert min(orders) > 1.95, orders


def test_map_radial(oracle):
    O = oracle
    g = O.Grid.make((8, 6, 4), ("neumann",) * 3, ("neumann",) * 3, (0.125, 0.125, 0.25))
    nr, r0, dr = 41, 0.0, 0.025
    rt = r0 + dr * np.arange(nr)
    beta = 1.0 + 3.0 * rt
    rho = 2.0 + rt
    # plane-parallel: radius = height z
    sig, bc, bf = O.map_radial(g, False, (0, 0, 0), r0, dr, beta, rho)
    z = (np.arange(4) + 0.5) * 0.25
    np.testing.assert_allclose(bc[:, 0, 0], np.minimum(1 + 3 * z, beta[-1]), rtol=1e-14)
    np.testing.assert_allclose(sig[:, 3, 5], np.minimum(1 + 3 * z, beta[-1]) / np.minimum(2 + z, rho[-1]), rtol=1e-14)
    ze = np.arange(5) * 0.25
    np.testing.assert_allclose(bf[2][:, 2, 2], np.minimum(1 + 3 * ze, beta[-1]), rtol=1e-14)
    # spherical: radius = distance to the centre
    c = (0.5, 0.375, 0.5)
    sig, bc, bf = O.map_radial(g, True, c, r0, dr, beta, rho)
    x, y, zz = (3 + 0.5) * 0.125, (1 + 0.5) * 0.125, (2 + 0.5) * 0.25
    rr = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (zz - c[2]) ** 2)
    assert bc[2, 1, 3] == pytest.approx(1 + 3 * rr, rel=1e-14)
    xf = 3 * 0.125
    rf = np.sqrt((xf - c[0]) ** 2 + (y - c[1]) ** 2 + (zz - c[2]) ** 2)
    assert bf[0][2, 1, 3] == pytest.approx(1 + 3 * rf, rel=1e-14)
