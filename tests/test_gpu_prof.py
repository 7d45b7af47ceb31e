"""Live per-kernel timing (mg_prof_*): launch and byte accounting of the timed classes.

The benchmark's roofline divides the algorithmic bytes of a class by its
event-timed launches, so the counts must be exact: a mixed MAC solve with
V(nu1, nu2) cycles runs, on the finest level, 2 (nu1 + nu2) colour passes and
one residual + restriction per V-cycle -- or, with the pipelined legs
(MG_FLAG_CELL_PIPE), one down leg (nu1 sweeps at 4 words per cell and the
residual restriction at 3 + 1/8) and one up leg (prolongation fused into the
first of nu2 sweeps: 4 + 1/8 words per cell, then 4 per sweep) --
and the nodal solve nu1 + nu2 Jacobi sweeps per V-cycle.
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


@pytest.mark.parametrize("pipe", [True, False])
def test_prof_counts_match_vcycles(pipe):
    p = I.stratified(64, seed=4, contrast=1e3)
    n = 64 ** 3
    mac = ProjectionSolver(p["geom"], T(p["sigma"]), loc="cell", prec="mixed", nu1=2, nu2=1,
                           flags=N.MG_FLAG_CELL_PIPE if pipe else 0)
    nod = ProjectionSolver(p["geom"], T(p["sigma"]), loc="nodal", prec="mixed", nu1=2, nu2=2)
    fm = T(np.random.default_rng(3).normal(size=mac.vec_shape))
    fn = T(np.random.default_rng(4).normal(size=nod.vec_shape))
    pm, pn = torch.zeros_like(fm), torch.zeros_like(fn)
    torch.cuda.synchronize()
    N.mg_prof_enable(True)
    try:
        sm = mac.solve(fm, pm, tol=1e-10)
        sn = nod.solve(fn, pn, tol=1e-10)
        torch.cuda.synchronize()
        q = {name: N.mg_prof_query(k) for k, name in N.PROF_NAMES.items()}
    finally:
        N.mg_prof_enable(False)
    cs, rr, ns = q["cell_smooth_fine"], q["cell_restrict_fine"], q["node_smooth_fine"]
    dn, up = q["cell_pipe_down"], q["cell_pipe_up"]
    if pipe:
        assert cs["launches"] == 0 and rr["launches"] == 0
        assert dn["launches"] == sm["vcycles"] and up["launches"] == sm["vcycles"]
        assert dn["bytes"] == pytest.approx(dn["launches"] * (4 * 2 + 3 + 1 / 8) * 4 * n)
        assert up["bytes"] == pytest.approx(up["launches"] * (4 * 1 + 1 / 8) * 4 * n)
    else:
        assert dn["launches"] == 0 and up["launches"] == 0
        assert cs["launches"] == 2 * 3 * sm["vcycles"]
        assert cs["bytes"] == pytest.approx(cs["launches"] * 2 * 4 * n)
        assert rr["launches"] == sm["vcycles"]
    assert ns["launches"] == 4 * sn["vcycles"]
    assert ns["bytes"] == pytest.approx(ns["launches"] * 4 * 4 * nod.vec_shape[0] * nod.vec_shape[1] * nod.vec_shape[2])
    assert q["cell_resid64"]["launches"] >= sm["iters"] and q["node_resid64"]["launches"] >= sn["iters"]
    for v in q.values():
        assert (v["ms"] > 0.0) == (v["launches"] > 0)
    mac.close()
    nod.close()
