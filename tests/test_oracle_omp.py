"""The all-core CPU baseline (oracle/mg_oracle_omp.c: the oracle with colour-ordered
smoothers and OpenMP loops), which the benchmark times beside the one-thread
oracle.  It is not used for parity, but what it reports must be a real solve:
its result does not depend on the thread count (bit for bit), and it reaches the
one-thread oracle's solution of the same system."""
import os

import numpy as np
import pytest

import inputs as I


@pytest.mark.parametrize("n", [16, 24])
def test_all_cores_is_thread_count_independent_and_converged(oracle, n):
    O = oracle
    p = I.stratified(n, seed=3, contrast=1e3)
    g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"])
    ref_m = O.mac_project(g, p["sigma"], p["beta0"], p["beta0_face"], p["U_mac"], p["S"], tol=1e-13)
    ref_n = O.nodal_project(g, p["sigma"], p["beta0"], p["U_cell"], p["S"], tol=1e-13)
    cores = max(2, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else 2)
    out = []
    for th in (1, cores):
        with O.all_cores(th):
            a = O.mac_project(g, p["sigma"], p["beta0"], p["beta0_face"], p["U_mac"], p["S"], tol=1e-13)
            b = O.nodal_project(g, p["sigma"], p["beta0"], p["U_cell"], p["S"], tol=1e-13)
        out.append((a, b))
    (a1, b1), (a2, b2) = out
    assert np.array_equal(a1["phi"], a2["phi"]) and np.array_equal(b1["phi"], b2["phi"])
    for u1, u2 in zip(a1["U"] + b1["U"], a2["U"] + b2["U"]):
        assert np.array_equal(u1, u2)
    assert np.linalg.norm(a1["phi"] - ref_m["phi"]) <= 1e-10 * np.linalg.norm(ref_m["phi"])
    live = ~g.dirichlet_node_mask()
    assert np.linalg.norm((b1["phi"] - ref_n["phi"])[live]) <= 1e-10 * np.linalg.norm(ref_n["phi"][live])
