"""Write oracle_small.json: small results of the FP64 oracle kept as regression values.

The paper prints no worked numerical example of the projection (its only numbers are
timings of its own port), so no fixture here carries a value from the paper.  These are
regression values only: they pin nothing about the method by themselves (the oracle's pins
are the closed forms and invariants of tests/test_oracle_*.py) but they make any later change
of the oracle's arithmetic visible.  Every value is computed by oracle/ alone, with the dense
direct solves, so it is the exact discrete solution up to round-off.

    python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import inputs as I  # noqa: E402
import oracle as O  # noqa: E402


def cases():
    O.build()
    out = {}
    # MAC projection (the projection of Eq. 6 with the base state frozen; harmonic face
    # coefficients of beta0/rho, the velocity update of the gradient form of Eq. 2)
    p = I.stratified(6, seed=11, contrast=1e3)
    g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"], p["geom"]["h"])
    r = O.mac_project(g, p["sigma"], p["beta0"], p["beta0_face"], p["U_mac"], p["S"], tol=1e-14, dense=True)
    out["mac_project_6"] = {"cite": "Eq. 6 and Eq. 2 (MAC projection), stratified recipe n=6 seed 11, dense solve",
                            "phi": r["phi"].ravel().tolist(), "constraint": r["constraint"]}
    # nodal projection (approximate projection of the same constraint on the Q1 node grid)
    p = I.stratified(4, seed=12, contrast=1e3)
    g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"], p["geom"]["h"])
    r = O.nodal_project(g, p["sigma"], p["beta0"], p["U_cell"], p["S"], tol=1e-14, dense=True)
    out["nodal_project_4"] = {"cite": "Eq. 6 and Eq. 2 (nodal projection), stratified recipe n=4 seed 12, dense solve",
                              "phi": r["phi"].ravel().tolist(), "constraint": r["constraint"],
                              "U0": r["U"][0].ravel().tolist()}
    # beta0 of Eq. 5 by the oracle's quadrature for a non-isothermal p0 and a varying Gamma1
    rr = np.linspace(0.0, 1.0, 33)
    p0 = np.exp(-3.0 * rr) * (1.0 + 0.1 * np.sin(7.0 * rr))
    out["beta0_eq5_33"] = {"cite": "Eq. 5, trapezoidal quadrature of (1/Gamma1) d ln p0",
                           "beta0": O.beta0_eq5(p0, 0.7, gamma1=1.4 + 0.3 * rr).tolist()}
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_small.json"), "w") as f:
        json.dump(cases(), f, indent=0)
        f.write("\n")
