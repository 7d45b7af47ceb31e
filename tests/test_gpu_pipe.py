"""The pipelined legs of the cell V-cycle (one launch per leg on the finest
FP32 level, its colour passes pipelined through L2) against the pass-by-pass
kernels and against the oracle.

The pipelined kernel runs every pass on the values the pass-by-pass launches
would see, so phi must be identical bit for bit: same iterations, same
residual, same bits, for every smoothing count the kernel takes, every boundary
kind of the lateral axes, row counts that leave a ragged band, a y-periodic
grid (bands wrap), solves started from zero (the first red pass takes x = 0
without loading it) and from a warm start, and both the host-driven and the
graph-resident refinement loops.  The end result is also compared with the
oracle (rel-L2 <= 1e-8, the mixed-precision bound).
"""
import numpy as np
import pytest

import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1910_12979_gb300 import ProjectionSolver  # noqa: E402
from paper_1910_12979_gb300 import native as N  # noqa: E402

DEV = "cuda:0"


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


GRIDS = [
    # (nx, ny, nz), (lo, hi): ny = 20 leaves a last band of 4 rows; with y periodic the bands also wrap
    ((32, 20, 32), (("periodic", "neumann", "neumann"), ("periodic", "dirichlet", "dirichlet"))),
    ((32, 20, 40), (("dirichlet", "periodic", "dirichlet"), ("neumann", "periodic", "neumann"))),
    ((128, 64, 48), (("periodic", "periodic", "neumann"), ("periodic", "periodic", "dirichlet"))),
]


@pytest.mark.parametrize("n,bcs", GRIDS)
@pytest.mark.parametrize("nu", [(2, 1), (1, 1), (3, 2), (4, 4)])
def test_pipe_matches_pass_by_pass(n, bcs, nu):
    rng = np.random.default_rng(21)
    sigma = T(np.exp(rng.uniform(0.0, np.log(1e3), size=n[::-1])))
    geom = dict(I.geometry(n, bcs[0], bcs[1]), h=(1.0 / max(n),) * 3)
    f = T(np.random.default_rng(8).normal(size=n[::-1]))
    guess = T(np.random.default_rng(9).normal(size=n[::-1]) * 1e-3)
    for extra in (0, N.MG_FLAG_ZERO_GUESS, N.MG_FLAG_NO_GRAPH):
        out = []
        for flags in (extra | N.MG_FLAG_CELL_PIPE, extra):
            s = ProjectionSolver(geom, sigma, loc="cell", prec="mixed", flags=flags, nu1=nu[0], nu2=nu[1],
                                 max_iters=5)
            phi = guess.clone()
            st = s.solve(f, phi, tol=1e-11, allow_not_converged=True)
            out.append((phi, st["iters"], st["rel_resid"], st["vcycles"]))
            s.close()
        (p0, *s0), (p1, *s1) = out
        assert s0 == s1, (extra, s0, s1)
        assert torch.equal(p0, p1), (extra, float((p0 - p1).abs().max()))


def test_pipe_projection_matches_oracle(oracle):
    """A stratified 48^3 MAC projection (pipelined legs on the finest level)
    against the oracle's solve of the same system."""
    O = oracle
    p = I.stratified(48, seed=31, contrast=1e3, nodal=False)
    g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"], p["geom"]["h"])
    ref = O.mac_project(g, p["sigma"], p["beta0"], p["beta0_face"], p["U_mac"], p["S"], tol=1e-13)
    s = ProjectionSolver(p["geom"], T(p["sigma"]), loc="cell", prec="mixed", nu1=2, nu2=1,
                         flags=N.MG_FLAG_CELL_PIPE)
    U = [T(u) for u in p["U_mac"]]
    phi = torch.zeros(s.vec_shape, dtype=torch.float64, device=DEV)
    st = s.project(U, T(p["beta0"]), T(p["S"]), beta0_face=[T(b) for b in p["beta0_face"]], phi=phi, tol=1e-12)
    s.close()
    ph = phi.cpu().numpy()
    assert np.linalg.norm(ph - ref["phi"]) / np.linalg.norm(ref["phi"]) <= 1e-8
    for d in range(3):
        u, r = U[d].cpu().numpy(), ref["U"][d]
        assert np.linalg.norm(u - r) <= 1e-8 * np.linalg.norm(r)
    assert st["rel_constraint"] <= 1e-10
