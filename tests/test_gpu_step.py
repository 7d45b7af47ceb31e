"""One time step around the two projections (mg_step) against the oracle's
composition of the same pieces."""
import numpy as np
import pytest

import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1910_12979_gb300 import ProjectionSolver  # noqa: E402
from paper_1910_12979_gb300 import native as N  # noqa: E402
from paper_1910_12979_gb300.solver import time_step  # noqa: E402

DEV = "cuda:0"
TOL = {"fp64": 1e-9, "mixed": 1e-8}


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("rot", [False, True])
def test_step_matches_oracle(oracle, prec, rot):
    O = oracle
    p = I.stratified(32, seed=6, contrast=1e2)
    g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"])
    rng = np.random.default_rng(3)
    U = [u + 0.05 * rng.normal(size=u.shape) for u in p["U_cell"]]
    dt = 0.02
    kw = {"omega": (0.0, 0.4, 1.1), "center": (0.5, 0.5, 0.5)} if rot else {}
    ref = O.time_step(g, p["sigma"], p["beta0"], p["beta0_face"], U, p["S"], dt, centrifugal=True, **kw)
    mac = ProjectionSolver(p["geom"], T(p["sigma"]), loc="cell", prec=prec)
    nod = ProjectionSolver(p["geom"], T(p["sigma"]), loc="nodal", prec=prec)
    Ud = [T(u) for u in U]
    Un = [torch.empty_like(u) for u in Ud]
    Ua = [torch.empty(mac.face_shape(d), dtype=torch.float64, device=DEV) for d in range(3)]
    sm, sn = time_step(mac, nod, Ud, Un, Ua, T(p["beta0"]), [T(b) for b in p["beta0_face"]], T(p["S"]), dt,
                       centrifugal=True, tol=1e-12, **kw)
    for d in range(3):
        assert relerr(Ua[d].cpu().numpy(), ref["Uadv"][d]) <= TOL[prec]
        assert relerr(Un[d].cpu().numpy(), ref["U"][d]) <= TOL[prec]
        assert torch.equal(Ud[d], T(U[d]))            # U^n untouched
    assert sm["rel_constraint"] < 1e-8
    assert sn["rel_constraint"] == pytest.approx(ref["nodal"]["constraint"], rel=1e-6)
    mac.close()
    nod.close()


def test_step_rejects_mismatched_handles():
    p = I.stratified(32, seed=6, contrast=1e2, mac=False, nodal=False)
    q = I.stratified(16, seed=6, contrast=1e2, mac=False, nodal=False)
    mac = ProjectionSolver(p["geom"], T(p["sigma"]), loc="cell", prec="mixed")
    nod = ProjectionSolver(q["geom"], T(q["sigma"]), loc="nodal", prec="mixed")
    z = lambda shp: torch.zeros(shp, dtype=torch.float64, device=DEV)
    with pytest.raises(N.MGError):
        time_step(mac, nod, [z(mac.cell_shape)] * 3, [z(mac.cell_shape) for _ in range(3)],
                  [z(mac.face_shape(d)) for d in range(3)], z(mac.cell_shape),
                  [z(mac.face_shape(d)) for d in range(3)], z(mac.cell_shape), 0.1)
    mac.close()
    nod.close()
