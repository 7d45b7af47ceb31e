"""Coriolis and centrifugal accelerations (S5) through the C ABI against the oracle."""
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


def geom_c(n, h):
    dim = len(n)
    nn = list(n) + [1] * (3 - dim)
    hh = list(h) + [1.0] * (3 - dim)
    return N.mg_geometry(dim, tuple(nn), tuple(hh), N.MG_LOC_CELL)


@pytest.mark.parametrize("n,h", [((40, 24, 16), (0.025, 0.03, 0.04)), ((33, 20), (0.03, 0.05))])
@pytest.mark.parametrize("centrifugal", [False, True])
def test_rotation_matches_oracle(oracle, n, h, centrifugal):
    O = oracle
    dim = len(n)
    geom = I.geometry(n, ("periodic",) * dim, ("periodic",) * dim)
    g = O.Grid.make(geom["n"], geom["bclo"], geom["bchi"], h=h)
    rng = np.random.default_rng(7 + dim)
    U = [rng.normal(size=g.cell_shape) for _ in range(dim)]
    F0 = [rng.normal(size=g.cell_shape) for _ in range(dim)]
    om = tuple(rng.normal(size=3))
    c = (0.41, 0.37, 0.52)
    want = O.rotation_forces(g, om, c[:dim], U, F=F0, alpha=0.3, centrifugal=centrifugal)
    Ud = [T(u) for u in U]
    Fd = [T(f) for f in F0]
    N.mg_rotation_forces(geom_c(n, h), om, c, centrifugal, 0.3, [u.data_ptr() for u in Ud],
                         [f.data_ptr() for f in Fd])
    torch.cuda.synchronize()
    for d in range(dim):
        got = Fd[d].cpu().numpy()
        assert np.max(np.abs(got - want[d])) <= 1e-14 * np.max(np.abs(want[d]))


def test_rotation_in_place_update(oracle):
    """F aliasing U: the explicit update U += dt a."""
    O = oracle
    n, h = (32, 16, 8), (1 / 32, 1 / 16, 1 / 8)
    geom = I.geometry(n, ("periodic",) * 3, ("periodic",) * 3)
    g = O.Grid.make(geom["n"], geom["bclo"], geom["bchi"], h=h)
    rng = np.random.default_rng(11)
    U = [rng.normal(size=g.cell_shape) for _ in range(3)]
    om, c, dt = (0.0, 0.3, 1.1), (0.5, 0.5, 0.5), 0.05
    want = O.rotation_forces(g, om, c, U, F=U, alpha=dt)
    Ud = [T(u) for u in U]
    N.mg_rotation_forces(geom_c(n, h), om, c, True, dt, [u.data_ptr() for u in Ud], [u.data_ptr() for u in Ud])
    torch.cuda.synchronize()
    for d in range(3):
        assert np.max(np.abs(Ud[d].cpu().numpy() - want[d])) <= 1e-14 * np.max(np.abs(want[d]))


def test_rotation_rejects_missing_components():
    with pytest.raises(N.MGError):
        N.mg_rotation_forces(geom_c((8, 8, 8), (0.1, 0.1, 0.1)), (0, 0, 1), None, True, 1.0, [None] * 3, [None] * 3)
