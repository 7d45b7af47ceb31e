"""The smoother autotuner (MG_FLAG_AUTOTUNE): every candidate kernel computes
the same arithmetic, so an autotuned handle returns the same phi, bit for bit,
as the default choice and as the forced alternatives; the choices are reported
per level and cached per grid."""
import numpy as np
import pytest

import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1910_12979_gb300 import ProjectionSolver, solve_batch  # noqa: E402
from paper_1910_12979_gb300 import native as N  # noqa: E402

DEV = "cuda:0"


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


@pytest.mark.parametrize("loc", ["cell", "nodal"])
def test_autotuned_equals_default(loc):
    p = I.stratified(64, seed=12, contrast=1e3, mac=False, nodal=False)
    out, kinds = [], []
    for flags in (0, N.MG_FLAG_AUTOTUNE, N.MG_FLAG_AUTOTUNE):   # the second tuned handle hits the cache
        s = ProjectionSolver(p["geom"], T(p["sigma"]), loc=loc, prec="mixed", flags=flags)
        f = T(np.random.default_rng(3).normal(size=s.vec_shape))
        phi = torch.zeros_like(f)
        st = s.solve(f, phi, tol=1e-11)
        out.append((phi, st["iters"]))
        kinds.append([N.mg_smoother_kind(s.handle, l) for l in range(4)])
        s.close()
    assert all(0 <= k <= 11 for k in kinds[1])
    if loc == "cell":
        assert all(k in (0, 1, 2, 3, 4, 8) for k in kinds[1])
    else:
        assert all(k in (0, 1, 2, 3, 4, 5, 6, 7, 9, 10, 11) for k in kinds[1])
    assert kinds[1] == kinds[2]
    assert kinds[1][0] != 0                       # the finest level was timed
    for phi, it in out[1:]:
        assert it == out[0][1] and torch.equal(phi, out[0][0])


def test_autotuned_batch_equals_alone():
    specs = [(32, "cell"), (64, "cell"), (32, "nodal"), (48, "cell")]
    solvers, rhs = [], []
    for i, (n, loc) in enumerate(specs):
        p = I.stratified(n, seed=40 + i, contrast=10.0 ** (1 + i), mac=False, nodal=False)
        solvers.append(ProjectionSolver(p["geom"], T(p["sigma"]), loc=loc, prec="mixed", flags=N.MG_FLAG_AUTOTUNE))
        rhs.append(T(np.random.default_rng(i).normal(size=solvers[-1].vec_shape)))
    alone = []
    for s, f in zip(solvers, rhs):
        phi = torch.zeros_like(f)
        s.solve(f, phi, tol=1e-10)
        alone.append(phi)
    phis = [torch.zeros_like(f) for f in rhs]
    solve_batch(solvers, rhs, phis, [1e-10] * len(rhs))
    for a, b in zip(alone, phis):
        assert torch.equal(a, b)
    for s in solvers:
        s.close()
