"""Serving on the GPU: every request's result is the same in the mix as alone.

Requests of three grid sizes arrive together: their problems are uploaded from
pinned host memory into resident hierarchies on their own streams, the requests
admitted together run as one batch (their solves in one graph launch), and the
projected velocities come back to pinned host memory.  They must equal, bit for
bit, those of the same problems each projected alone on a fresh solver (the
kernels' arithmetic does not depend on what else runs on the device).  The
post-projection constraint of each request is also checked against the
oracle's definition of D(beta0 U) - beta0 S.
"""
import numpy as np
import pytest

import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1910_12979_gb300 import ProjectionSolver  # noqa: E402
from paper_1910_12979_gb300.serve import GpuBackend, Request, Scheduler, host_problem, latency_stats  # noqa: E402


def test_alone_equals_mix(oracle):
    dev = "cuda:0"
    sizes = (32, 48, 64)
    problems = {n: [host_problem(I.polytrope_star(n, seed=50 + 3 * n + k)) for k in range(2)] for n in sizes}
    order = [32, 64, 48, 32, 64, 48, 48, 32, 64, 32]
    reqs = [Request(i, n, 0.0, (n, i % 2), keep=True) for i, n in enumerate(order)]
    be = GpuBackend(problems, device=dev, tol=1e-11)
    sch = Scheduler(be, budget_bytes=2 * 10 ** 9, max_inflight=6)
    done = sch.run_stream(reqs, timeout=300)
    assert all(not isinstance(r.status, Exception) for r in done)
    st = latency_stats(done)
    assert st["count"] == len(order)
    assert max(sch.batches) > 1      # requests admitted together ran as a batch
    sch.close()
    D = lambda t: t.to(dev)
    for r in done:
        n, k = r.payload
        p = problems[n][k]
        s = ProjectionSolver(p["geom"], D(p["sigma"]), loc="cell", prec="mixed")
        U = [D(u) for u in p["U"]]
        phi = torch.zeros(s.vec_shape, dtype=torch.float64, device=dev)
        s.project(U, D(p["beta0"]), D(p["S"]), beta0_face=[D(b) for b in p["beta0_face"]], phi=phi, tol=1e-11)
        for a, b in zip(U, r.result):
            assert torch.equal(a.cpu(), b), (r.rid, n)
        s.close()
    # one projected field checked with the oracle's own divergence
    O = oracle
    r = done[0]
    n, k = r.payload
    g = O.Grid.make((n, n, n), ("dirichlet",) * 3, ("dirichlet",) * 3)
    p = problems[n][k]
    H = lambda t: t.cpu().numpy()
    div = O.mac_rhs(g, H(p["beta0"]), [H(b) for b in p["beta0_face"]], [H(u) for u in r.result], H(p["S"]))
    src = np.linalg.norm(H(p["beta0"]) * H(p["S"]))
    assert np.linalg.norm(div) / src < 1e-8
