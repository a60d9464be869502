"""The binned tree solve (three launches per application: the contraction
tree's bottom subtrees one thread block each, the top part in one block)
against the level-by-level solve of the same factor and against the oracle,
and the PCG step fused around it against the unfused step."""
from __future__ import annotations


import numpy as np
import pytest
import torch

import oracle
import paper_2410_04512_gb300 as sgp
import workloads
from gpu_common import GpuSystem, dev_tensor, oracle_system, rel_err, small_cube

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda_device):
    return sgp.Context(0)


def _ctx(bin_cap):
    c = sgp.Context(0)
    c.set_tuning(bin_cap=bin_cap)
    return c


def _chain(n=20000):
    pos = np.zeros((n, 3))
    pos[:, 0] = 0.9 * np.arange(n)
    pos[:, 1] = 0.02 * np.sin(0.1 * np.arange(n))
    return workloads.Cells("chain", pos, np.full(n, 0.5), 9, 0.1, 10.0, 1e-3)


def _cases():
    return {
        "cube1k": small_cube(1000, seed=1000),
        "ball60k": workloads.ball(n=60000, seed=2001, gamma0=1e-3),
        "chain20k": _chain(),
        "hex": workloads.hex_sheet(nx=120, ny=90, seed=3000),
    }


def _kappa_bound(s, c):
    """Gershgorin bound on kappa(P): lambda_min(P) >= gamma0 (Lemma 2.4),
    lambda_max(P) <= gamma0 + 2 max_i sum_j |Upsilon_ij| over tree edges."""
    te = s.T.edge_ids().cpu().numpy()
    ij = s.ij.cpu().numpy()[te]
    blocks = s.M.edge_blocks()[0].cpu().numpy()[te]
    norms = np.abs(blocks).sum(axis=2).max(axis=1)
    rowsum = np.zeros(c.n)
    np.add.at(rowsum, ij[:, 0], norms)
    np.add.at(rowsum, ij[:, 1], norms)
    return (c.gamma0 + 2 * rowsum.max()) / c.gamma0


def _apply(ctx, c, bin_cap, precision=sgp.PREC_F64, seed=0):
    cx = _ctx(bin_cap)
    s = GpuSystem(cx, c, precision=precision)
    b = np.random.default_rng(seed).standard_normal((c.n, 3))
    x = cx.tree_apply(s.Fac, dev_tensor(b)).cpu().numpy()
    return x, s, b


@pytest.mark.parametrize("name", ["cube1k", "ball60k", "chain20k", "hex"])
@pytest.mark.parametrize("cap", [64, 256, 1024])
def test_binned_apply_equals_level_apply(name, cap):
    """Same factor, same operator: the binned solve differs from the level
    kernels only in the order in which a top receiver subtracts its leaks
    (the bins' values are computed in the same order), so the two agree
    within the forward-error bound of two backward-stable solves,
    64 eps kappa(P)."""
    c = _cases()[name]
    xl, sl, b = _apply(None, c, -1)
    xb, sb, _ = _apply(None, c, cap)
    lay = sb.Fac.layout()
    assert lay["bin_cap"] == cap and lay["bins"] >= 1, lay
    # small bins always fit in shared memory in FP64; large FP64 bins of a
    # chain (two L blocks per vertex) may not, and then the level kernels run
    assert lay["fp64"] == 1 or cap > 256, lay
    assert sl.Fac.layout()["fp64"] == 0
    assert lay["top"] < c.n
    tol = 64 * np.finfo(float).eps * _kappa_bound(sb, c)
    assert rel_err(xb, xl) <= tol, (name, cap, rel_err(xb, xl), tol, lay)


@pytest.mark.parametrize("cap", [64, 1024])
def test_binned_apply_matches_oracle(cap):
    """Forward error against the oracle's Prim-order solve within
    64 eps kappa(P) (both are backward-stable solves of P x = b)."""
    c = small_cube(1000, seed=1001)
    x, s, b = _apply(None, c, cap, seed=3)
    o = oracle_system(c)
    f = oracle.prim_msf(c.n, o.ij, o.w)
    fac = oracle.tree_ldlt(f, o.blocks, c.gamma0)
    want = oracle.tree_solve(fac, b)
    te = np.sort(f.tree_edges)
    norms = np.abs(o.blocks[te]).sum(axis=2).max(axis=1)
    rowsum = np.zeros(c.n)
    np.add.at(rowsum, o.ij[te, 0], norms)
    np.add.at(rowsum, o.ij[te, 1], norms)
    kappa = (c.gamma0 + 2 * rowsum.max()) / c.gamma0
    assert rel_err(x, want) <= 64 * np.finfo(float).eps * kappa


def test_binned_layout_of_a_forest_of_many_trees():
    """Isolated cells, pairs and a few clusters: every tree small, all of
    them bottom subtrees (no top part)."""
    rng = np.random.default_rng(5)
    pos = np.concatenate([rng.uniform(0, 400, size=(300, 3)),
                          rng.uniform(0, 6, size=(200, 3)) + 500.0])
    cells = workloads.Cells("forest", pos, np.full(pos.shape[0], 0.5), 8, 0.1, 10.0, 1e-2)
    xl, _, b = _apply(None, cells, -1)
    xb, s, _ = _apply(None, cells, 1024)
    assert s.Fac.layout()["top"] == 0
    assert rel_err(xb, xl) <= 1e-14


def test_binned_mixed_factor_layouts():
    """A MIXED factor gets the FP32 layout (the inner solve's); its FP64
    apply (the public call) uses the FP64 layout when it fits, else the
    level kernels, and stays the FP64 solve either way."""
    c = workloads.ball(n=60000, seed=2001, gamma0=1e-3)
    xl, _, b = _apply(None, c, -1, precision=sgp.PREC_MIXED)
    xb, s, _ = _apply(None, c, 1024, precision=sgp.PREC_MIXED)
    lay = s.Fac.layout()
    assert lay["fp32"] == 1, lay
    assert rel_err(xb, xl) <= 64 * np.finfo(float).eps * _kappa_bound(s, c)


@pytest.mark.parametrize("precision", [sgp.PREC_F64, sgp.PREC_MIXED])
def test_fused_step_matches_unfused(precision):
    """The PCG step fused around the binned solve (r -= alpha q and |r|^2 in
    the bins and the top, r^T z in the backward launch) reaches the same
    solution as the unfused step on the level kernels."""
    c = workloads.ball(n=20000, seed=2003, gamma0=1e-3)
    F = c.forces()
    tol, agree = (1e-13, 1e-9) if precision == sgp.PREC_F64 else (1e-12, 1e-8)
    cf = _ctx(1024)
    sf = GpuSystem(cf, c, precision=precision)
    assert sf.Fac.layout()["top"] > 0
    vf, inf_f = cf.pcg_solve(sf.M, sf.Fac, dev_tensor(F), tol=tol, precision=precision)
    cu = _ctx(-1)
    su = GpuSystem(cu, c, precision=precision)
    vu, inf_u = cu.pcg_solve(su.M, su.Fac, dev_tensor(F), tol=tol, precision=precision)
    assert inf_f.status == 0 and inf_u.status == 0
    assert abs(inf_f.iterations - inf_u.iterations) <= max(3, inf_u.iterations // 50)
    # the recursive residual reaches tol; the true one stalls at rounding
    # level (eps kappa(Gamma)) in FP64, and the mixed loop checks it exactly
    assert inf_f.true_rel_residual <= (1e-11 if precision == sgp.PREC_F64 else 2 * tol)
    assert inf_f.true_rel_residual <= max(4 * inf_u.true_rel_residual, 2 * tol)
    assert rel_err(vf.cpu().numpy(), vu.cpu().numpy()) <= agree


def test_fused_step_iterates_at_equal_k():
    """FP64 iterates of the fused step after k = 1, 5, 30 iterations agree
    with the oracle's PCG to 1e-9 (x += alpha p is applied in the step's
    last launch, also on the step that stops)."""
    c = small_cube(3000, seed=1004)
    cx = _ctx(128)
    s = GpuSystem(cx, c)
    assert s.Fac.layout()["top"] > 0
    o = oracle_system(c)
    F = c.forces()
    f = oracle.prim_msf(c.n, o.ij, o.w)
    fac = oracle.tree_ldlt(f, o.blocks, c.gamma0)
    for k in (1, 5, 30):
        v, info = cx.pcg_solve(s.M, s.Fac, dev_tensor(F), tol=1e-300, maxit=k, raise_on_error=False)
        assert info.iterations == k and info.status == sgp.ERR_NO_CONVERGENCE
        r = oracle.pcg(c.n, o.ij, o.blocks, c.gamma0, F, oracle.PRECOND_TREE, fac, fixed_iters=k)
        assert rel_err(v.cpu().numpy(), r.x) <= 1e-9, k


def test_fused_step_bitwise_reproducible():
    c = workloads.ball(n=30000, seed=2004, gamma0=1e-3)
    F = dev_tensor(c.forces())
    out = []
    for _ in range(2):
        cx = _ctx(512)
        s = GpuSystem(cx, c, precision=sgp.PREC_MIXED)
        v, info = cx.pcg_solve(s.M, s.Fac, F, tol=1e-8, precision=sgp.PREC_MIXED)
        out.append((v, info.iterations))
    assert out[0][1] == out[1][1]
    assert torch.equal(out[0][0], out[1][0])
