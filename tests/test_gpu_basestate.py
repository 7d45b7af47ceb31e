"""Device-resident base state (Eq. 5 quadrature and radial mapping) against the oracle."""
import numpy as np
import pytest

import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1910_12979_gb300 import native as N  # noqa: E402

DEV = "cuda:0"


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


@pytest.mark.parametrize("nr", [1, 2, 1000, 5003])
def test_beta0_matches_oracle(oracle, nr):
    r = np.linspace(0.0, 1.0, max(nr, 1))
    p0 = np.exp(-3.0 * r) * (1.0 + 0.1 * np.sin(7 * r))
    g1 = 1.4 + 0.3 * r
    out = torch.zeros(nr, dtype=torch.float64, device=DEV)
    p0d, gd = T(p0), T(g1)
    N.mg_base_state_beta0(p0d.data_ptr(), gd.data_ptr(), 0.0, 0.7, nr, out.data_ptr())
    torch.cuda.synchronize()
    ref = oracle.beta0_eq5(p0, 0.7, gamma1=g1)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-13)
    out2 = torch.zeros(nr, dtype=torch.float64, device=DEV)
    N.mg_base_state_beta0(p0d.data_ptr(), None, 5.0 / 3.0, 0.7, nr, out2.data_ptr())
    torch.cuda.synchronize()
    np.testing.assert_allclose(out2.cpu().numpy(), oracle.beta0_eq5(p0, 0.7), rtol=1e-13)


@pytest.mark.parametrize("spherical", [True, False])
def test_map_matches_oracle(oracle, spherical):
    O = oracle
    n = (24, 16, 32)
    g = O.Grid.make(n, ("dirichlet",) * 3, ("dirichlet",) * 3)
    xe, xi, th = I.polytrope_profile(1e4, 3.0)
    nr = 2000
    dr = 0.9 / (nr - 1)
    rt = dr * np.arange(nr)
    rho_r = np.interp(np.minimum(rt, 0.5) / 0.5 * xe, xi, th) ** 3
    beta_r = rho_r ** 0.8
    center = (0.5, 0.45, 0.55)
    ref = O.map_radial(g, spherical, center, 0.0, dr, beta_r, rho_r)
    geo = N.mg_geometry(3, n, tuple(1.0 / v for v in n), N.MG_LOC_CELL)
    sig = torch.zeros(g.cell_shape, dtype=torch.float64, device=DEV)
    bc = torch.zeros_like(sig)
    bf = [torch.zeros(g.face_shape(d), dtype=torch.float64, device=DEV) for d in range(3)]
    br, rr = T(beta_r), T(rho_r)
    N.mg_base_state_map(geo, spherical, center, 0.0, dr, nr, br.data_ptr(), rr.data_ptr(), sig.data_ptr(),
                        bc.data_ptr(), [b.data_ptr() for b in bf])
    torch.cuda.synchronize()
    np.testing.assert_allclose(sig.cpu().numpy(), ref[0], rtol=1e-14)
    np.testing.assert_allclose(bc.cpu().numpy(), ref[1], rtol=1e-14)
    for d in range(3):
        np.testing.assert_allclose(bf[d].cpu().numpy(), ref[2][d], rtol=1e-14)


@pytest.mark.parametrize("spherical", [True, False])
def test_map_2d_matches_oracle(oracle, spherical):
    # 2-D: the plane-parallel radius is y; rows of 40 cells (41 x-faces) leave lanes idle and the
    # 25 y-face rows end in a partial group of rows
    O = oracle
    n = (40, 24)
    g = O.Grid.make(n, ("periodic", "neumann"), ("periodic", "dirichlet"))
    nr = 700
    dr = 1.2 / (nr - 1)
    rt = dr * np.arange(nr)
    rho_r = np.exp(-4.0 * rt) * (1.0 + 0.05 * np.cos(9.0 * rt))
    beta_r = rho_r ** 0.6
    center = (0.4, 0.55)
    ref = O.map_radial(g, spherical, center, 0.0, dr, beta_r, rho_r)
    geo = N.mg_geometry(2, n, tuple(1.0 / v for v in n), N.MG_LOC_CELL)
    sig = torch.zeros(g.cell_shape, dtype=torch.float64, device=DEV)
    bc = torch.zeros_like(sig)
    bf = [torch.zeros(g.face_shape(d), dtype=torch.float64, device=DEV) for d in range(2)]
    br, rr = T(beta_r), T(rho_r)
    N.mg_base_state_map(geo, spherical, center + (0.0,), 0.0, dr, nr, br.data_ptr(), rr.data_ptr(), sig.data_ptr(),
                        bc.data_ptr(), [b.data_ptr() for b in bf] + [None])
    torch.cuda.synchronize()
    np.testing.assert_allclose(sig.cpu().numpy(), ref[0], rtol=1e-14)
    np.testing.assert_allclose(bc.cpu().numpy(), ref[1], rtol=1e-14)
    for d in range(2):
        np.testing.assert_allclose(bf[d].cpu().numpy(), ref[2][d], rtol=1e-14)
