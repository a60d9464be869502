"""Iteration counts of the oracle's own solves of the benchmark workloads.

TEST INFRASTRUCTURE (like everything under oracle/): the benchmark's CPU
leg times the oracle's solve phase at full size on a bounded number of PCG
iterations and scales that time to the number of iterations the oracle
needs to reach the tolerance.  That number is a property of the workload
and the oracle alone; this script computes it with a complete oracle solve
(k-d tree contact search checked against the brute-force rule, eq. (1)
blocks, Prim, TreeLDLT, PCG from a zero guess) and stores it in
``calibration.json`` beside this file.

    python -m oracle.calibrate [ball1m cube1k ...]

A full solve of the 1e6-cell spheroid takes about two minutes on one core.
"""
from __future__ import annotations

import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402

OUT = os.path.join(HERE, "calibration.json")

# the benchmark's workloads (rank 0's replica seed) and tolerances
WORKLOADS = {
    "ball1m": (lambda: workloads.ball(n=1_000_000, seed=2000, gamma0=1e-3), 1e-8),
    "cube1k": (lambda: workloads.cube(n=1000, side=8.886, seed=2000), 1e-8),
}


def calibrate(name: str) -> dict:
    make, tol = WORKLOADS[name]
    c = make()
    F = c.forces()
    t0 = time.perf_counter()
    ij = oracle.contacts_kdtree(c.pos, c.radii)
    sysm = oracle.build_system(c.pos, c.radii, c.gammas_np, c.gamma0, ij=ij)
    t1 = time.perf_counter()
    forest = oracle.prim_msf(sysm.n, sysm.ij, sysm.w)
    fac = oracle.tree_ldlt(forest, sysm.blocks, sysm.gamma0)
    t2 = time.perf_counter()
    res = oracle.pcg(sysm.n, sysm.ij, sysm.blocks, sysm.gamma0, F, oracle.PRECOND_TREE, fac, tol=tol)
    t3 = time.perf_counter()
    return {"n_cells": int(c.n), "edges": int(ij.shape[0]), "tol": tol, "iterations": int(res.iters),
            "rel_residual": float(res.relres), "setup_s": round(t1 - t0, 3), "factor_s": round(t2 - t1, 3),
            "pcg_s": round(t3 - t2, 3), "host": platform.machine()}


def main(argv):
    names = argv or sorted(WORKLOADS)
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name in names:
        data[name] = calibrate(name)
        print(name, data[name], flush=True)
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:])
