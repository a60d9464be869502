"""The one-block mixed-precision solve of small systems (every contraction
level in the tree solve's one-block tail): against the multi-launch path on
the same system, against the oracle's FP64 solution, and its edge cases."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
import paper_2410_04512_gb300 as sgp
import workloads
from gpu_common import GpuSystem, dev_tensor, oracle_system, rel_err, small_cube

pytestmark = pytest.mark.gpu


def _ctx(small=True):
    if small:
        return sgp.Context(0)
    os.environ["SGP_NO_SMALL"] = "1"
    try:
        return sgp.Context(0)
    finally:
        del os.environ["SGP_NO_SMALL"]


def _solve(cx, s, F, **kw):
    cx.launch_count(reset=True)
    v, info = cx.pcg_solve(s.M, s.Fac, dev_tensor(F), precision=sgp.PREC_MIXED, **kw)
    return v.cpu().numpy(), info, cx.launch_count()


@pytest.mark.parametrize("n,seed", [(1000, 1200), (300, 1201), (3000, 1202)])
def test_small_solve_matches_multi_launch_and_oracle(cuda_device, n, seed):
    """Up to about a thousand cells the one-block solve runs (one launch for
    the whole solve); beyond, the multi-launch path does."""
    c = small_cube(n, seed=seed)
    F = c.forces()
    a, b = _ctx(True), _ctx(False)
    sa, sb = GpuSystem(a, c, precision=sgp.PREC_MIXED), GpuSystem(b, c, precision=sgp.PREC_MIXED)
    xa, ia, la = _solve(a, sa, F, tol=1e-10)
    xb, ib, lb = _solve(b, sb, F, tol=1e-10)
    assert ia.status == 0 and ib.status == 0
    if n <= 1000:
        assert la <= 4 < lb, (la, lb)
    else:
        assert la == lb > 4, (la, lb)
    assert ia.true_rel_residual <= 1e-10 and ib.true_rel_residual <= 1e-10
    assert abs(ia.iterations - ib.iterations) <= max(3, ib.iterations // 20), (ia.iterations, ib.iterations)
    assert ia.outer_iterations == ib.outer_iterations
    o = oracle_system(c)
    want = oracle.solve_system(o, F, tol=1e-13)[0].x
    assert rel_err(xa, want) <= 1e-8
    assert rel_err(xa, xb) <= 1e-8


def test_small_solve_edge_cases(cuda_device):
    c = small_cube(500, seed=1203)
    cx = _ctx(True)
    s = GpuSystem(cx, c, precision=sgp.PREC_MIXED)
    F = c.forces()
    # zero right-hand side: v = 0 at once
    x0, i0, _ = _solve(cx, s, np.zeros_like(F), tol=1e-8)
    assert i0.iterations == 0 and not x0.any() and i0.status == 0
    # a given initial guess near the solution needs fewer iterations
    x1, i1, _ = _solve(cx, s, F, tol=1e-8)
    v0 = dev_tensor(x1 * (1 + 1e-6))
    cx.launch_count(reset=True)
    v2, i2 = cx.pcg_solve(s.M, s.Fac, dev_tensor(F), v=v0, x0_given=True, precision=sgp.PREC_MIXED, tol=1e-8)
    assert i2.status == 0 and i2.iterations < i1.iterations and i2.true_rel_residual <= 1e-8
    # an iteration cap: NO_CONVERGENCE with the cap's count
    _, i3, _ = _solve(cx, s, F, tol=1e-14, maxit=9, raise_on_error=False)
    assert i3.status == sgp.ERR_NO_CONVERGENCE and i3.iterations == 9
    # isolated cells (no contacts): P = Gamma = gamma0 I
    pos = np.random.default_rng(3).uniform(0, 400, size=(200, 3))
    iso = workloads.Cells("isolated", pos, np.full(200, 0.5), 9, 0.1, 10.0, 0.25)
    si = GpuSystem(cx, iso, precision=sgp.PREC_MIXED)
    Fi = iso.forces()
    xi, ii, _ = _solve(cx, si, Fi, tol=1e-10)
    assert ii.status == 0
    np.testing.assert_allclose(xi, Fi / 0.25, rtol=1e-9)
