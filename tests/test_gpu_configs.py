"""Error against the oracle for the workloads that the element-by-element
parity tests of test_gpu_parity.py do not already cover: the 128^3 nodal
projection of the stratified step, entries of the uneven batch solved inside
one batch launch, and polytrope-star requests that went through the serving
scheduler.  Each is compared with a full oracle solve of the same system
(rel-L2 of phi or of the projected velocity <= 1e-8, the mixed-precision bound;
<= 1e-9 for FP64), with the GPU solved to 1e-12 so that the solver tolerance
cannot hide a discrepancy.
"""
import numpy as np
import pytest

import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1910_12979_gb300 import ProjectionSolver, solve_batch  # noqa: E402
from paper_1910_12979_gb300 import native as N  # noqa: E402
from paper_1910_12979_gb300.serve import GpuBackend, Request, Scheduler, host_problem  # noqa: E402

DEV = "cuda:0"
TOL = {"fp64": 1e-9, "mixed": 1e-8}
_CACHE = {}


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def H(t):
    return t.detach().cpu().numpy()


def relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _nodal_128(O):
    if "n128" not in _CACHE:
        p = I.stratified(128, seed=2, contrast=1e3, mac=False)
        g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"])
        ref = O.nodal_project(g, p["sigma"], p["beta0"], p["U_cell"], p["S"], tol=1e-13)
        _CACHE["n128"] = (p, g, ref)
    return _CACHE["n128"]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_config2_128_nodal_full_parity(oracle, prec):
    """The nodal projection of the 128^3 stratified step against a full oracle
    solve: phi over the unknown nodes and the projected cell velocities."""
    p, g, ref = _nodal_128(oracle)
    s = ProjectionSolver(p["geom"], T(p["sigma"]), loc="nodal", prec=prec)
    U = [T(u) for u in p["U_cell"]]
    phi = torch.zeros(s.vec_shape, dtype=torch.float64, device=DEV)
    st = s.project(U, T(p["beta0"]), T(p["S"]), phi=phi, tol=1e-12, allow_not_converged=True)
    s.close()
    live = ~g.dirichlet_node_mask()
    assert relerr(H(phi)[live], ref["phi"][live]) <= TOL[prec]
    for d in range(3):
        assert relerr(H(U[d]), ref["U"][d]) <= TOL[prec]
    assert st["rel_constraint"] == pytest.approx(ref["constraint"], rel=1e-6)


def test_batch_entries_vs_oracle(oracle):
    """Three entries of the seeded uneven batch -- 32^3, 96^3 (coarsest level
    3^3) and 128^3, each with its own density contrast and heating centre --
    solved together in one mg_solve_batch launch in the benchmark's
    configuration (mixed, autotuned smoother shapes, solves started from
    zero), each against the oracle's multigrid solve of its system."""
    O = oracle
    specs = I.batch_specs(64, seed=4)
    pick = []
    for n in (32, 96, 128):
        pick.append(next(sp for sp in specs if sp["n"] == n))
    solvers, rhs, phis, refs = [], [], [], []
    for sp in pick:
        p = I.batch_problem(sp)
        s = ProjectionSolver(p["geom"], T(p["sigma"]), loc="cell", prec="mixed",
                             flags=N.MG_FLAG_AUTOTUNE | N.MG_FLAG_ZERO_GUESS)
        f = s.rhs([T(u) for u in p["U_mac"]], T(p["beta0"]), T(p["S"]), beta0_face=[T(b) for b in p["beta0_face"]])
        g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"])
        fo = O.mac_rhs(g, p["beta0"], p["beta0_face"], p["U_mac"], p["S"])
        assert relerr(H(f), fo) <= 1e-13            # the right-hand side itself
        ref, _ = O.mac_solve_mg(g, O.mac_faces(g, p["sigma"]), fo, tol=1e-13)
        solvers.append(s)
        rhs.append(f)
        phis.append(torch.zeros_like(f))
        refs.append(ref)
    st = solve_batch(solvers, rhs, phis, [1e-12] * len(solvers))
    for sp, ph, ref, s_ in zip(pick, phis, refs, st):
        assert s_["status"] == N.MG_OK
        assert relerr(H(ph), ref) <= 1e-8, (sp["n"], relerr(H(ph), ref))
    for s in solvers:
        s.close()


def test_served_requests_vs_oracle(oracle):
    """Polytrope-star MAC projections (64^3 and 128^3, phi = 0 on every face)
    admitted and run by the serving scheduler, against oracle projections."""
    O = oracle
    sizes = (64, 128)
    host = {n: I.polytrope_star(n, seed=70 + n) for n in sizes}
    problems = {n: [host_problem(host[n])] for n in sizes}
    reqs = [Request(i, n, 0.0, (n, 0), keep=True) for i, n in enumerate(sizes)]
    sch = Scheduler(GpuBackend(problems, device=DEV, tol=1e-12), budget_bytes=8 * 10 ** 9, max_inflight=2)
    done = sch.run_stream(reqs, timeout=300)
    sch.close()
    for r in done:
        assert not isinstance(r.status, Exception), r.status
        n = r.n
        p = host[n]
        g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"])
        ref = O.mac_project(g, p["sigma"], p["beta0"], p["beta0_face"], p["U_mac"], p["S"], tol=1e-13)
        num = np.sqrt(sum(np.sum((H(u) - v) ** 2) for u, v in zip(r.result, ref["U"])))
        den = np.sqrt(sum(np.sum(v ** 2) for v in ref["U"]))
        assert num / den <= 1e-8, (n, num / den)
