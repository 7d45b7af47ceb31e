"""Seeded synthetic inputs for the projection solve (shared by tests, smoke and bench).

This module holds no arithmetic of the solve itself (no operator, divergence,
gradient, smoother or norm): it only draws and tabulates the fields that the
solver receives -- density, the base-state buoyancy term beta0 of Eq. 5 in its
closed form, sigma = beta0/rho, random velocities and the heating source S.
Both the GPU path and the CPU oracle consume exactly these arrays.

The paper's own workloads (the ``reacting_bubble`` problem and stellar models,
S6) are not available; the generators below stand in for them:

* ``manufactured_2d``: 2-D stratified square, rho = exp(-y/H), H = 0.25,
  beta0 = rho^(1/gamma), gamma = 5/3, and the right-hand side of the smooth
  solution phi = cos(2 pi x) cos(2 pi y); periodic in x, Neumann in y.
* ``stratified``: 3-D plane-parallel isothermal atmosphere with a given
  bottom-to-top density contrast, Gaussian random velocity and a Gaussian
  heating blob; periodic in x and y, slip wall at the bottom, outflow
  (phi = 0) at the top.
* ``polytrope_star``: 3-D star of polytropic index 3 centred in the unit cube,
  Lane-Emden profile with a given centre-to-edge density contrast, phi = 0 on
  every boundary.

Layouts follow the solver's: x fastest, arrays shaped (nz, ny, nx); faces of
axis d have one more entry along d; 2-D arrays use nz = 1.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA1 = 5.0 / 3.0


def _centres(n):
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def _edges(n):
    return np.arange(n + 1, dtype=np.float64) / n


def geometry(n, bclo, bchi):
    """Plain description of the grid on the unit domain: cells, spacing, boundaries."""
    dim = len(n)
    return {"dim": dim, "n": tuple(int(v) for v in n), "h": tuple(1.0 / v for v in n),
            "bclo": tuple(bclo), "bchi": tuple(bchi)}


# --------------------------------------------------------------------------- 2-D

def manufactured_2d(n: int = 64, H: float = 0.25):
    """2-D stratified solve with a manufactured smooth solution.

    rho(y) = exp(-y/H), beta0 = rho^(1/gamma) (Eq. 5 for an isothermal p ~ rho
    with rho(0) = 1), sigma = beta0/rho = exp(y (1 - 1/gamma) / H).  For
    phi = cos(2 pi x) cos(2 pi y),
        div(sigma grad phi) = -8 pi^2 sigma phi + sigma' dphi/dy,
    tabulated at cell centres.  Returns a dict with the geometry, rho, beta0,
    sigma, f and the exact phi (all shaped (1, n, n)).
    """
    x = _centres(n)[None, None, :]
    y = _centres(n)[None, :, None]
    a = (1.0 - 1.0 / GAMMA1) / H                 # sigma = exp(a y)
    rho = np.exp(-y / H) * np.ones((1, n, n))
    beta0 = rho ** (1.0 / GAMMA1)
    sigma = beta0 / rho
    phi = np.cos(2 * np.pi * x) * np.cos(2 * np.pi * y)
    dphidy = -2 * np.pi * np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y)
    f = -8 * np.pi ** 2 * sigma * phi + a * sigma * dphidy
    return {"geom": geometry((n, n), ("periodic", "neumann"), ("periodic", "neumann")),
            "rho": rho, "beta0": beta0, "sigma": sigma, "f": f, "phi_exact": phi * np.ones((1, n, n))}


# ------------------------------------------------------------------ 3-D fields

def _gaussian_blob(n, centre, width):
    x = _centres(n)
    gx = np.exp(-((x - centre[0]) ** 2) / width ** 2)
    gy = np.exp(-((x - centre[1]) ** 2) / width ** 2)
    gz = np.exp(-((x - centre[2]) ** 2) / width ** 2)
    return gz[:, None, None] * gy[None, :, None] * gx[None, None, :]


def _mac_velocity(rng, n, u_std, bclo, bchi):
    """Random face velocities, one array per axis; periodic copies equal, wall faces 0."""
    U = []
    for d in range(3):
        shape = [n, n, n]
        shape[2 - d] += 1
        u = rng.normal(0.0, u_std, size=shape)
        idx_lo = [slice(None)] * 3
        idx_hi = [slice(None)] * 3
        idx_lo[2 - d] = 0
        idx_hi[2 - d] = n
        if bclo[d] == "periodic":
            u[tuple(idx_hi)] = u[tuple(idx_lo)]
        else:
            if bclo[d] == "neumann":
                u[tuple(idx_lo)] = 0.0
            if bchi[d] == "neumann":
                u[tuple(idx_hi)] = 0.0
        U.append(u)
    return U


def stratified(n: int, seed: int, contrast: float = 1e3, u_std: float = 1e-2, width: float = 0.1,
               centre=(0.5, 0.5, 0.5), mac: bool = True, nodal: bool = True):
    """3-D plane-parallel isothermal atmosphere on the unit cube.

    rho(z) = contrast^(-z) (so rho(0)/rho(1) = contrast), beta0 = rho^(1/gamma),
    sigma = beta0/rho.  beta0 is also tabulated at the MAC face centres for the
    face update.  U ~ N(0, u_std^2) independently per face value (MAC) and per
    cell component (nodal); wall-normal faces are zero.  S = exp(-|x-c|^2/w^2).
    Boundaries: periodic x, y; slip wall (Neumann) at z = 0; outflow (phi = 0)
    at z = 1.
    """
    bclo = ("periodic", "periodic", "neumann")
    bchi = ("periodic", "periodic", "dirichlet")
    rng = np.random.default_rng(seed)
    lnc = math.log(contrast)
    zc = _centres(n)
    ze = _edges(n)
    rho_z = np.exp(-lnc * zc)
    rho = np.broadcast_to(rho_z[:, None, None], (n, n, n)).copy()
    beta0 = rho ** (1.0 / GAMMA1)
    sigma = beta0 / rho
    bz_c = np.exp(-lnc * zc / GAMMA1)
    bz_e = np.exp(-lnc * ze / GAMMA1)
    beta0_face = [np.broadcast_to(bz_c[:, None, None], (n, n, n + 1)).copy(),
                  np.broadcast_to(bz_c[:, None, None], (n, n + 1, n)).copy(),
                  np.broadcast_to(bz_e[:, None, None], (n + 1, n, n)).copy()]
    S = _gaussian_blob(n, centre, width)
    out = {"geom": geometry((n, n, n), bclo, bchi), "rho": rho, "beta0": beta0, "sigma": sigma,
           "beta0_face": beta0_face, "S": S}
    if mac:
        out["U_mac"] = _mac_velocity(rng, n, u_std, bclo, bchi)
    if nodal:
        out["U_cell"] = [rng.normal(0.0, u_std, size=(n, n, n)) for _ in range(3)]
    return out


# ------------------------------------------------------------------ polytrope

def lane_emden(index: float, xi_max: float, step: float = 1e-3):
    """Tabulate theta(xi) of the Lane-Emden equation theta'' + 2 theta'/xi = -theta^n.

    Classical RK4 from a series start at xi0 = step (theta = 1 - xi^2/6 +
    n xi^4/120).  Stops at xi_max or just before theta reaches 0.  Returns
    (xi, theta) arrays.
    """
    def rhs(xi, y):
        th, dth = y
        return np.array([dth, -max(th, 0.0) ** index - 2.0 * dth / xi])

    xi = step
    y = np.array([1 - xi ** 2 / 6 + index * xi ** 4 / 120, -xi / 3 + index * xi ** 3 / 30])
    xs, ths = [0.0, xi], [1.0, y[0]]
    while xi < xi_max:
        k1 = rhs(xi, y)
        k2 = rhs(xi + step / 2, y + step / 2 * k1)
        k3 = rhs(xi + step / 2, y + step / 2 * k2)
        k4 = rhs(xi + step, y + step * k3)
        y_new = y + step / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        if y_new[0] <= 0.0:
            break
        xi += step
        y = y_new
        xs.append(xi)
        ths.append(y[0])
    return np.array(xs), np.array(ths)


def polytrope_profile(contrast: float = 1e4, index: float = 3.0):
    """(xi_edge, xi table, theta table) with theta(xi_edge)^index = 1/contrast."""
    xi, th = lane_emden(index, 7.0, 1e-4)
    target = contrast ** (-1.0 / index)
    k = int(np.nonzero(th < target)[0][0])
    # linear interpolation for the crossing (the table step is 1e-4)
    xe = xi[k - 1] + (th[k - 1] - target) * (xi[k] - xi[k - 1]) / (th[k - 1] - th[k])
    return xe, xi[: k + 1], th[: k + 1]


def polytrope_star(n: int, seed: int, contrast: float = 1e4, u_std: float = 1e-2, width: float = 0.1,
                   centre=None, index: float = 3.0, mac: bool = True, nodal: bool = False):
    """Star of polytropic index 3 centred in the unit cube, phi = 0 on every face.

    rho(r) = theta(xi)^n with xi = xi_edge * r / 0.5, clamped to the edge value
    for r > 0.5 (the cube corners); p ~ rho^(1 + 1/n), so beta0 of Eq. 5 with
    constant Gamma1 is rho^((1 + 1/n)/Gamma1) (rho_c = 1).  The heating blob
    centre is drawn uniformly in [0.3, 0.7]^3 from ``seed`` unless given.
    """
    rng = np.random.default_rng(seed)
    if centre is None:
        centre = tuple(rng.uniform(0.3, 0.7, size=3))
    xe, xi_t, th_t = polytrope_profile(contrast, index)
    expo = (1.0 + 1.0 / index) / GAMMA1

    def rho_at(x, y, z):
        r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
        xi = xe * np.minimum(r, 0.5) / 0.5
        return np.interp(xi, xi_t, th_t) ** index

    c, e = _centres(n), _edges(n)
    rho = rho_at(c[None, None, :], c[None, :, None], c[:, None, None])
    beta0 = rho ** expo
    sigma = beta0 / rho
    beta0_face = [rho_at(e[None, None, :], c[None, :, None], c[:, None, None]) ** expo,
                  rho_at(c[None, None, :], e[None, :, None], c[:, None, None]) ** expo,
                  rho_at(c[None, None, :], c[None, :, None], e[:, None, None]) ** expo]
    S = _gaussian_blob(n, centre, width)
    bc = ("dirichlet",) * 3
    out = {"geom": geometry((n, n, n), bc, bc), "rho": rho, "beta0": beta0, "sigma": sigma,
           "beta0_face": beta0_face, "S": S, "centre": centre}
    if mac:
        out["U_mac"] = _mac_velocity(rng, n, u_std, bc, bc)
    if nodal:
        out["U_cell"] = [rng.normal(0.0, u_std, size=(n, n, n)) for _ in range(3)]
    return out


# ---------------------------------------------------------------- batch / serve

def batch_specs(count: int = 64, seed: int = 4, sizes=(32, 64, 96, 128), contrast_range=(1e1, 1e4)):
    """Per-solve parameters of an uneven batch: size, density contrast
    (log-uniform), heating centre in [0.3, 0.7]^3 and a per-solve seed."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        lc = rng.uniform(math.log(contrast_range[0]), math.log(contrast_range[1]))
        centre = tuple(float(v) for v in rng.uniform(0.3, 0.7, size=3))
        out.append({"n": n, "contrast": float(math.exp(lc)), "centre": centre, "seed": int(seed * 100003 + i)})
    return out


def batch_problem(spec):
    """The stratified MAC problem of one batch entry."""
    return stratified(spec["n"], spec["seed"], contrast=spec["contrast"], centre=spec["centre"],
                      mac=True, nodal=False)


def poisson_arrivals(rate: float, count: int, seed: int = 5, sizes=(64, 96, 128, 192, 256)):
    """Arrival times (s) of a Poisson stream and a uniformly drawn size per request."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps) - gaps[0]
    ns = rng.choice(sizes, size=count)
    return t, [int(v) for v in ns]
