"""The batched solve loop of mg_solve_batch / mg_project_batch, through the C ABI.

The 3-D mixed-precision cell solves of a batch with at most 2^18 cells share
one lockstep iteration loop whose steps are shared launches driven by
per-solve work items (level passes, coarse ends, FP64 residuals, norms,
updates, convergence checks).  Each solve keeps its own decisions, so it must
iterate as often as alone and return the same phi bit for bit -- against the
solve run alone and against the batch run as per-solve graph branches
(MG_FLAG_BATCH_BRANCHES) -- while using far fewer launches.  Solves that stop
early (converged, or out of iterations) drop out without disturbing the rest.
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


# (cells per axis, low / high boundary kinds): cubic and ragged grids, levels
# launched by the batched kernels from one (16^3, 24^3) to three (96^3), and
# boundary mixes with and without a Dirichlet side (singular problems too)
P_N = ("periodic", "periodic", "neumann")
P_D = ("periodic", "periodic", "dirichlet")
D3 = ("dirichlet",) * 3
N3 = ("neumann",) * 3
GRIDS = [
    ((16, 16, 16), P_N, P_D),
    ((24, 24, 24), D3, D3),
    ((32, 32, 32), P_N, P_D),
    ((48, 48, 48), N3, N3),
    ((40, 24, 32), D3, ("neumann", "dirichlet", "neumann")),
    ((64, 32, 48), ("periodic", "neumann", "neumann"), ("periodic", "neumann", "dirichlet")),
    ((96, 96, 96), P_N, P_D),
    ((32, 64, 32), ("periodic", "periodic", "periodic"), ("periodic", "periodic", "periodic")),
]


def problem(i, shape, lo, hi):
    rng = np.random.default_rng(100 + i)
    geom = I.geometry(shape, lo, hi)
    sigma = np.exp(rng.uniform(-0.5, 0.5) * 4.0 * rng.random(shape[::-1]))   # contrast up to e^2 per cell
    return geom, sigma


def make(specs, flags=0, **kw):
    out = []
    for i, (shape, lo, hi) in enumerate(specs):
        geom, sigma = problem(i, shape, lo, hi)
        out.append(ProjectionSolver(geom, T(sigma), loc="cell", prec="mixed", flags=flags, **kw))
    return out


def rhs_of(solvers):
    return [T(np.random.default_rng(7 + i).normal(size=s.vec_shape)) for i, s in enumerate(solvers)]


def test_batched_loop_equals_alone_and_branches():
    solvers = make(GRIDS)
    branch = make(GRIDS, flags=N.MG_FLAG_BATCH_BRANCHES)
    host = make(GRIDS, flags=N.MG_FLAG_NO_GRAPH)   # the batched loop driven from the host
    rhs = rhs_of(solvers)
    alone = []
    for s, f in zip(solvers, rhs):
        phi = torch.zeros_like(f)
        alone.append((phi, s.solve(f, phi, tol=1e-10)))
    its = {st["iters"] for _, st in alone}
    assert len(its) > 1   # the solves stop after different numbers of iterations
    launches = {}
    for name, group in (("batched", solvers), ("branches", branch), ("host", host)):
        for rep in range(2):   # the second call replays the cached graph
            phis = [torch.zeros_like(f) for f in rhs]   # the same initial guess as alone
            l0 = N.mg_launch_count()
            st = solve_batch(group, rhs, phis, [1e-10] * len(rhs))
            launches[name] = N.mg_launch_count() - l0
            for (pa, sa), pb, sb in zip(alone, phis, st):
                assert sb["status"] == N.MG_OK
                assert sb["iters"] == sa["iters"] and sb["vcycles"] == sa["vcycles"]
                assert torch.equal(pa, pb), name
    # one launch per step for the seven solves of at most 64^3 cells instead of
    # one per step and solve (the 96^3 solve runs as its own branch)
    assert launches["batched"] * 2 < launches["branches"], launches
    for s in solvers + branch + host:
        s.close()


def test_batch_groups_do_not_change_results():
    """The batch split into 1, 3 or 8 concurrent lockstep loops: the same phi."""
    solvers = make(GRIDS)
    rhs = rhs_of(solvers)
    out = []
    try:
        for g in (1, 3, 8):
            N.mg_set_batch_groups(g)
            phis = [torch.zeros_like(f) for f in rhs]
            st = solve_batch(solvers, rhs, phis, [1e-10] * len(rhs))
            out.append((phis, [x["iters"] for x in st]))
    finally:
        N.mg_set_batch_groups(0)
    for phis, its in out[1:]:
        assert its == out[0][1]
        for a, b in zip(phis, out[0][0]):
            assert torch.equal(a, b)
    with pytest.raises(N.MGError):
        N.mg_set_batch_groups(-1)
    for s in solvers:
        s.close()


def test_batched_loop_dropouts_and_zero_guess():
    """A solve that runs out of iterations, one with a zero right-hand side and
    solves started from zero (MG_FLAG_ZERO_GUESS) share the loop with solves
    that run on; each result is its result alone."""
    specs = GRIDS[:6]
    solvers = make(specs, flags=N.MG_FLAG_ZERO_GUESS)
    solvers[1].close()
    geom, sigma = problem(1, *specs[1])
    solvers[1] = ProjectionSolver(geom, T(sigma), loc="cell", prec="mixed", flags=N.MG_FLAG_ZERO_GUESS, max_iters=2)
    rhs = rhs_of(solvers)
    rhs[3] = torch.zeros_like(rhs[3])
    tols = [1e-10, 1e-12, 1e-10, 1e-10, 1e-9, 1e-11]
    alone = []
    for s, f, t in zip(solvers, rhs, tols):
        phi = torch.zeros_like(f)
        alone.append((phi, s.solve(f, phi, tol=t, allow_not_converged=True)))
    assert alone[1][1]["status"] == N.MG_ERR_NOT_CONVERGED and alone[1][1]["iters"] == 2
    phis = [torch.full_like(f, -1.0) for f in rhs]
    st = solve_batch(solvers, rhs, phis, tols, allow_not_converged=True)
    for (pa, sa), pb, sb in zip(alone, phis, st):
        assert sb["status"] == sa["status"] and sb["iters"] == sa["iters"]
        assert torch.equal(pa, pb)
    assert torch.count_nonzero(phis[3]) == 0
    for s in solvers:
        s.close()


def test_batched_projection_equals_alone(oracle):
    """mg_project_batch of stratified MAC projections of uneven sizes: the
    projected velocities and statistics equal each projection alone; one entry
    is checked against the oracle's projection."""
    sizes = (32, 48, 24, 64)
    probs = [I.stratified(n, seed=80 + n, contrast=10.0 ** (1 + k), mac=True, nodal=False)
             for k, n in enumerate(sizes)]
    solvers = [ProjectionSolver(p["geom"], T(p["sigma"]), loc="cell", prec="mixed") for p in probs]

    def inputs(p):
        return [T(u) for u in p["U_mac"]], T(p["beta0"]), T(p["S"]), [T(b) for b in p["beta0_face"]]

    alone = []
    for p, s in zip(probs, solvers):
        U, b0, S, bf = inputs(p)
        alone.append((U, s.project(U, b0, S, beta0_face=bf, tol=1e-11)))
    ins = [inputs(p) for p in probs]
    l0 = N.mg_launch_count()
    st = project_batch(solvers, [x[0] for x in ins], [x[1] for x in ins], [x[2] for x in ins],
                       beta0_face=[x[3] for x in ins], tols=[1e-11] * len(sizes))
    assert N.mg_launch_count() > l0
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


def test_mixed_batch_falls_back_to_branches():
    """A nodal or FP64 solve in the batch makes it a graph of per-solve
    branches; the results still equal the solves alone."""
    solvers = make(GRIDS[:3])
    p = I.stratified(24, seed=5, contrast=1e2, mac=False, nodal=False)
    solvers.append(ProjectionSolver(p["geom"], T(p["sigma"]), loc="nodal", prec="mixed"))
    rhs = rhs_of(solvers)
    alone = []
    for s, f in zip(solvers, rhs):
        phi = torch.zeros_like(f)
        alone.append((phi, s.solve(f, phi, tol=1e-10)))
    phis = [torch.zeros_like(f) for f in rhs]
    st = solve_batch(solvers, rhs, phis, [1e-10] * len(rhs))
    for (pa, sa), pb, sb in zip(alone, phis, st):
        assert sb["iters"] == sa["iters"]
        assert torch.equal(pa, pb)
    for s in solvers:
        s.close()


def test_batched_loop_over_96_solves():
    """More solves than one launch's parameter table holds (96 items): every
    step is split over several launches; each result is its result alone."""
    specs = [((16, 16, 16), P_N, P_D), ((24, 24, 24), D3, D3), ((32, 16, 16), N3, N3)] * 34   # 102 solves
    solvers = make(specs)
    rhs = rhs_of(solvers)
    alone = []
    for s, f in zip(solvers, rhs):
        phi = torch.zeros_like(f)
        alone.append((phi, s.solve(f, phi, tol=1e-10)))
    phis = [torch.zeros_like(f) for f in rhs]
    st = solve_batch(solvers, rhs, phis, [1e-10] * len(rhs))
    for (pa, sa), pb, sb in zip(alone, phis, st):
        assert sb["status"] == sa["status"] and sb["iters"] == sa["iters"]
        assert torch.equal(pa, pb)
    for s in solvers:
        s.close()


def test_host_driven_projection_batch_equals_alone():
    """mg_project_batch with graphs off runs the batched loop from the host
    (one read-back per iteration): the same velocities as each projection alone."""
    sizes = (32, 24, 48)
    probs = [I.stratified(n, seed=90 + n, contrast=10.0 ** (1 + k), mac=True, nodal=False)
             for k, n in enumerate(sizes)]
    alone_s = [ProjectionSolver(p["geom"], T(p["sigma"]), loc="cell", prec="mixed") for p in probs]
    host_s = [ProjectionSolver(p["geom"], T(p["sigma"]), loc="cell", prec="mixed", flags=N.MG_FLAG_NO_GRAPH)
              for p in probs]

    def inputs(p):
        return [T(u) for u in p["U_mac"]], T(p["beta0"]), T(p["S"]), [T(b) for b in p["beta0_face"]]

    alone = []
    for p, s in zip(probs, alone_s):
        U, b0, S, bf = inputs(p)
        alone.append((U, s.project(U, b0, S, beta0_face=bf, tol=1e-11)))
    ins = [inputs(p) for p in probs]
    st = project_batch(host_s, [x[0] for x in ins], [x[1] for x in ins], [x[2] for x in ins],
                       beta0_face=[x[3] for x in ins], tols=[1e-11] * len(sizes))
    for (Ua, sa), x, sb in zip(alone, ins, st):
        assert sb["status"] == N.MG_OK and sb["iters"] == sa["iters"]
        for a, b in zip(Ua, x[0]):
            assert torch.equal(a, b)
    for s in alone_s + host_s:
        s.close()


def test_ineligible_solves_run_as_branches_beside_the_loop():
    """A batch mixing solves the batched kernels take (16^3, 24^3, 32x40x32)
    with cell solves they do not (40^3: its 10^3 level has nx % 4 != 0; a 2-D
    grid): the first share the loop, the others run as branches of the same
    graph; every result equals the solve alone."""
    specs = [((16, 16, 16), P_N, P_D), ((40, 40, 40), D3, D3), ((24, 24, 24), N3, N3), ((32, 40, 32), P_N, P_D)]
    solvers = make(specs)
    rng = np.random.default_rng(3)
    g2 = I.geometry((64, 48), ("periodic", "neumann"), ("periodic", "dirichlet"))
    solvers.append(ProjectionSolver(g2, T(np.exp(rng.random((1, 48, 64)))), loc="cell", prec="mixed"))
    rhs = rhs_of(solvers)
    alone = []
    for s, f in zip(solvers, rhs):
        phi = torch.zeros_like(f)
        alone.append((phi, s.solve(f, phi, tol=1e-10)))
    for rep in range(2):
        phis = [torch.zeros_like(f) for f in rhs]
        st = solve_batch(solvers, rhs, phis, [1e-10] * len(rhs))
        for (pa, sa), pb, sb in zip(alone, phis, st):
            assert sb["status"] == N.MG_OK and sb["iters"] == sa["iters"]
            assert torch.equal(pa, pb)
    for s in solvers:
        s.close()
