"""Graph-resident solve loop and the one-launch batch, through the C ABI.

The graph path makes the convergence decisions on the device with the same
formulas as the host loop (MG_FLAG_NO_GRAPH), so both must return the same phi
bit for bit after the same number of iterations.  mg_solve_batch runs every
solve as a branch of one graph, and mg_project_batch every projection's solve;
each branch must equal the solve (or projection) run alone.
"""
import numpy as np
import pytest

import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1910_12979_gb300 import ProjectionSolver, project_batch, solve_batch  # noqa: E402
from paper_1910_12979_gb300 import native as N  # noqa: E402

DEV = "cuda:0"


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


@pytest.mark.parametrize("loc", ["cell", "nodal"])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_graph_equals_host_loop(loc, prec):
    p = I.stratified(32, seed=21, contrast=1e3)
    res = []
    for flags in (0, N.MG_FLAG_NO_GRAPH):
        s = ProjectionSolver(p["geom"], T(p["sigma"]), loc=loc, prec=prec, flags=flags)
        f = T(np.random.default_rng(8).normal(size=s.vec_shape))
        phi = torch.zeros_like(f)
        st = s.solve(f, phi, tol=1e-11)
        res.append((phi, st))
        s.close()
    (a, sa), (b, sb) = res
    assert sa["iters"] == sb["iters"] and sa["rel_resid"] == sb["rel_resid"]
    assert torch.equal(a, b)


@pytest.mark.parametrize("loc", ["cell", "nodal"])
def test_graph_projection_equals_host_loop(loc):
    p = I.stratified(32, seed=22, contrast=1e2)
    out = []
    for flags in (0, N.MG_FLAG_NO_GRAPH):
        s = ProjectionSolver(p["geom"], T(p["sigma"]), loc=loc, prec="mixed", flags=flags)
        U = [T(u) for u in (p["U_mac"] if loc == "cell" else p["U_cell"])]
        kw = {"beta0_face": [T(b) for b in p["beta0_face"]]} if loc == "cell" else {}
        st = s.project(U, T(p["beta0"]), T(p["S"]), tol=1e-10, **kw)
        out.append((U, st))
    (ua, sa), (ub, sb) = out
    assert sa["iters"] == sb["iters"] and sa["rel_constraint"] == sb["rel_constraint"]
    for x, y in zip(ua, ub):
        assert torch.equal(x, y)


def test_batch_one_launch_equals_alone():
    """Uneven sizes, both locations and both precisions in one graph launch."""
    specs = [(16, "cell", "mixed"), (32, "cell", "mixed"), (24, "nodal", "mixed"), (32, "cell", "fp64"),
             (48, "cell", "mixed"), (16, "nodal", "fp64")]
    solvers, rhs = [], []
    for i, (n, loc, prec) in enumerate(specs):
        p = I.stratified(n, seed=30 + i, contrast=10.0 ** (1 + i % 3), mac=False, nodal=False)
        s = ProjectionSolver(p["geom"], T(p["sigma"]), loc=loc, prec=prec)
        solvers.append(s)
        rhs.append(T(np.random.default_rng(i).normal(size=s.vec_shape)))
    alone = []
    for s, f in zip(solvers, rhs):
        phi = torch.zeros_like(f)
        st = s.solve(f, phi, tol=1e-10)
        alone.append((phi, st))
    for _ in range(2):  # the second call replays the cached batch graph
        phis = [torch.full_like(f, 7.0) * 0 for f in rhs]
        stats = solve_batch(solvers, rhs, phis, [1e-10] * len(rhs))
        for (pa, sa), pb, sb in zip(alone, phis, stats):
            assert sb["iters"] == sa["iters"] and sb["status"] == N.MG_OK
            assert torch.equal(pa, pb)


def test_batch_reports_per_solve_status():
    p = I.stratified(32, seed=3, contrast=1e3, mac=False, nodal=False)
    a = ProjectionSolver(p["geom"], T(p["sigma"]), loc="cell", prec="mixed")
    b = ProjectionSolver(p["geom"], T(p["sigma"]), loc="cell", prec="mixed", max_iters=2)
    f = T(np.random.default_rng(1).normal(size=a.vec_shape))
    pa, pb = torch.zeros_like(f), torch.zeros_like(f)
    st = solve_batch([a, b], [f, f], [pa, pb], [1e-10, 1e-12], allow_not_converged=True)
    assert st[0]["status"] == N.MG_OK and st[1]["status"] == N.MG_ERR_NOT_CONVERGED and st[1]["iters"] == 2
    with pytest.raises(N.MGError):
        solve_batch([a, a], [f, f], [pa, pb], [1e-10, 1e-10])


def test_graph_zero_rhs_and_warm_start():
    p = I.stratified(32, seed=4, contrast=1e3, mac=False, nodal=False)
    s = ProjectionSolver(p["geom"], T(p["sigma"]), loc="cell", prec="mixed")
    phi = torch.ones(s.vec_shape, dtype=torch.float64, device=DEV)
    st = s.solve(torch.zeros_like(phi), phi, tol=1e-10)
    assert st["iters"] == 0 and float(phi.abs().max()) == 0.0
    f = T(np.random.default_rng(2).normal(size=s.vec_shape))
    phi = torch.zeros_like(f)
    s.solve(f, phi, tol=1e-10)
    st2 = s.solve(f, phi, tol=1e-10)   # warm start at the solution: no iteration needed
    assert st2["iters"] == 0


@pytest.mark.parametrize("loc", ["cell", "nodal"])
def test_zero_guess_flag(loc):
    """MG_FLAG_ZERO_GUESS ignores phi's input and skips the operator in the first
    residual; the FP32 residual it feeds the V-cycles is the same, so the solve
    returns the same phi as a solve started from an explicit zero, on the graph
    path and on the host-driven loop."""
    p = I.stratified(32, seed=23, contrast=1e3, mac=False, nodal=False)
    res = []
    for flags in (0, N.MG_FLAG_ZERO_GUESS, N.MG_FLAG_ZERO_GUESS | N.MG_FLAG_NO_GRAPH):
        s = ProjectionSolver(p["geom"], T(p["sigma"]), loc=loc, prec="mixed", flags=flags)
        f = T(np.random.default_rng(9).normal(size=s.vec_shape))
        phi = torch.zeros_like(f) if flags == 0 else torch.full_like(f, 7.0)
        st = s.solve(f, phi, tol=1e-11)
        res.append((phi, st["iters"]))
        s.close()
    for phi, it in res[1:]:
        assert it == res[0][1] and torch.equal(phi, res[0][0])


@pytest.mark.parametrize("loc", ["cell", "nodal"])
def test_graph_launch_count_matches_host_loop(loc):
    # the graph path counts its replayed kernels (the loop body per iteration, each conditional
    # extra V-cycle when it ran); the host loop counts its launches one by one.  The two run the
    # same kernels plus a few control kernels on the graph side.
    p = I.stratified(48, seed=5, contrast=1e3)
    counts = []
    for flags in (0, N.MG_FLAG_NO_GRAPH):
        s = ProjectionSolver(p["geom"], T(p["sigma"]), loc=loc, prec="mixed", flags=flags)
        f = T(np.random.default_rng(2).normal(size=s.vec_shape))
        phi = torch.zeros_like(f)
        s.solve(f, phi, tol=1e-10)   # builds the graph and the cached sub-graphs
        torch.cuda.synchronize()
        phi.zero_()
        c0 = N.mg_launch_count()
        st = s.solve(f, phi, tol=1e-10)
        torch.cuda.synchronize()
        counts.append((N.mg_launch_count() - c0, st["vcycles"], st["iters"]))
        s.close()
    (g, vg, ig), (h, vh, ih) = counts
    assert vg == vh and ig == ih
    # a check kernel and two condition kernels per refinement step, a few per solve
    assert abs(g - h) <= 4 * (ih + 1) + 12, (g, h)


def test_project_batch_equals_alone(oracle):
    """mg_project_batch: MAC and nodal projections of uneven sizes and both
    precisions, their solves as one graph launch, give the same projected
    velocities and statistics as each projection alone; the 48^3 MAC entry is
    also checked against the oracle's projection."""
    specs = [(32, "cell", "mixed"), (48, "cell", "mixed"), (24, "nodal", "mixed"), (32, "cell", "fp64"),
             (16, "nodal", "fp64")]
    probs, solvers = [], []
    for i, (n, loc, prec) in enumerate(specs):
        p = I.stratified(n, seed=60 + i, contrast=10.0 ** (1 + i % 3))
        probs.append(p)
        solvers.append(ProjectionSolver(p["geom"], T(p["sigma"]), loc=loc, prec=prec))

    def inputs(p, loc):
        U = [T(u) for u in (p["U_mac"] if loc == "cell" else p["U_cell"])]
        return U, T(p["beta0"]), T(p["S"]), ([T(b) for b in p["beta0_face"]] if loc == "cell" else None)

    alone = []
    for (n, loc, prec), p, s in zip(specs, probs, solvers):
        U, b0, S, bf = inputs(p, loc)
        st = s.project(U, b0, S, beta0_face=bf, tol=1e-11)
        alone.append((U, st))
    for _ in range(2):   # the second call replays the cached batch graph
        ins = [inputs(p, loc) for (n, loc, prec), p in zip(specs, probs)]
        st = project_batch(solvers, [x[0] for x in ins], [x[1] for x in ins], [x[2] for x in ins],
                           beta0_face=[x[3] for x in ins], tols=[1e-11] * len(specs))
        for (Ua, sa), x, sb in zip(alone, ins, st):
            assert sb["status"] == N.MG_OK and sb["iters"] == sa["iters"]
            assert sb["rel_constraint"] == sa["rel_constraint"]
            for a, b in zip(Ua, x[0]):
                assert torch.equal(a, b)
    O = oracle
    p = probs[1]
    g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"])
    ref = O.mac_project(g, p["sigma"], p["beta0"], p["beta0_face"], p["U_mac"], p["S"], tol=1e-13)
    U = ins[1][0]
    num = np.sqrt(sum(np.sum((u.cpu().numpy() - r) ** 2) for u, r in zip(U, ref["U"])))
    den = np.sqrt(sum(np.sum(r ** 2) for r in ref["U"]))
    assert num / den <= 1e-8
    for s in solvers:
        s.close()
