"""The partitioned spanning-forest preconditioner (Section 6) through the C
ABI against the oracle: leaf labels and the union of the leaves' forests
bit for bit, the factor and PCG on it, and its binned layout (leaves as
independent bins, no top part)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import oracle.local_forest as lf
import paper_2410_04512_gb300 as sgp
import workloads
from gpu_common import GpuSystem, dev_tensor, oracle_system, rel_err, small_cube

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda_device):
    return sgp.Context(0)


def test_grid_leaves_bit_exact(ctx):
    rng = np.random.default_rng(11)
    pos = np.concatenate([rng.uniform(-3000.0, 3000.0, size=(20000, 3)),
                          rng.normal(0.0, 5.0, size=(5000, 3)),
                          np.array([[2.75, 0, 0], [np.nextafter(2.75, 0), 0, 0], [-1e-300, 0, 0], [0, 0, 0]])])
    for h in (2.75, 0.3, 7.67, 1e9):
        got = ctx.grid_leaves(dev_tensor(pos), h).cpu().numpy()
        np.testing.assert_array_equal(got, lf.grid_leaves(pos, h))
    with pytest.raises(sgp.SgpError):
        ctx.grid_leaves(dev_tensor(pos), 0.0)
    with pytest.raises(sgp.SgpError):
        ctx.grid_leaves(dev_tensor(pos), float("nan"))
    assert ctx.grid_leaves(dev_tensor(np.zeros((0, 3))), 1.0).shape == (0,)


CASES = {
    "cube3k": lambda: small_cube(3000, seed=1101),
    "ball60k": lambda: workloads.ball(n=60000, seed=2101, gamma0=1e-3),
    "hex": lambda: workloads.paper_hex(n=20000, seed=6301),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("h", [3.0, 7.67])
def test_local_forest_bit_exact(ctx, name, h):
    c = CASES[name]()
    s = GpuSystem(ctx, c, tree=False)
    o = oracle_system(c)
    leaf = ctx.grid_leaves(s.pos, h)
    np.testing.assert_array_equal(leaf.cpu().numpy(), lf.grid_leaves(c.pos, h))
    T = ctx.local_spanning_forest(s.M, leaf)
    want = np.sort(lf.local_msf(c.n, o.ij, o.w, lf.grid_leaves(c.pos, h)).tree_edges)
    np.testing.assert_array_equal(T.edge_ids().cpu().numpy(), want)
    ne, ncomp = T.info()[:2]
    assert ne == want.shape[0] and ncomp == c.n - ne


def test_local_forest_degenerate_leaves(ctx):
    c = small_cube(2000, seed=1102)
    s = GpuSystem(ctx, c, tree=False)
    o = oracle_system(c)
    # one leaf: the global forest
    one = torch.zeros(c.n, dtype=torch.int32, device="cuda")
    T1 = ctx.local_spanning_forest(s.M, one)
    np.testing.assert_array_equal(T1.edge_ids().cpu().numpy(), np.sort(oracle.prim_msf(c.n, o.ij, o.w).tree_edges))
    # every cell its own leaf: no edges; P = gamma0 I
    own = torch.arange(c.n, dtype=torch.int32, device="cuda")
    T0 = ctx.local_spanning_forest(s.M, own)
    assert T0.info()[0] == 0
    Fh = ctx.tree_factor(s.M, T0)
    b = np.random.default_rng(2).standard_normal((c.n, 3))
    x = ctx.tree_apply(Fh, dev_tensor(b)).cpu().numpy()
    np.testing.assert_allclose(x, b / c.gamma0, rtol=1e-15)
    with pytest.raises(ValueError):
        ctx.local_spanning_forest(s.M, own[:-1])


@pytest.mark.parametrize("precision", [sgp.PREC_F64, sgp.PREC_MIXED])
def test_local_forest_pcg_matches_oracle(ctx, precision):
    """PCG preconditioned by P_loc: the oracle's iteration count (FP64) and
    solution; the leaves of a small grid are independent bins (no top)."""
    c = workloads.ball(n=60000, seed=2102, gamma0=1e-3)
    cx = sgp.Context(0)
    cx.set_tuning(bin_cap=1024)
    s = GpuSystem(cx, c, precision=precision, tree=False)
    o = oracle_system(c)
    h = 5.0
    leaf = cx.grid_leaves(s.pos, h)
    T = cx.local_spanning_forest(s.M, leaf)
    Fh = cx.tree_factor(s.M, T)
    lay = Fh.layout()
    assert lay["bins"] >= 1 and lay["top"] == 0, lay
    F = c.forces()
    v, info = cx.pcg_solve(s.M, Fh, dev_tensor(F), tol=1e-10, precision=precision)
    assert info.status == 0
    f = lf.local_msf(c.n, o.ij, o.w, lf.grid_leaves(c.pos, h))
    fac = oracle.tree_ldlt(f, o.blocks, c.gamma0)
    r = oracle.pcg(c.n, o.ij, o.blocks, c.gamma0, F, oracle.PRECOND_TREE, fac, tol=1e-10)
    assert r.status == oracle.OK
    if precision == sgp.PREC_F64:
        assert abs(info.iterations - r.iters) <= max(3, r.iters // 50), (info.iterations, r.iters)
    assert rel_err(v.cpu().numpy(), r.x) <= 1e-7
    # error-bound stopping keeps its guarantee (mu = 1: the forest is a subgraph)
    if precision == sgp.PREC_F64:
        v2, info2 = cx.pcg_solve(s.M, Fh, dev_tensor(F), tol=1e-6, stop=sgp.STOP_ERROR)
        xs = r.x
        e = xs - v2.cpu().numpy()
        num = np.sum(e * oracle.matvec(c.n, o.ij, o.blocks, c.gamma0, e))
        den = np.sum(v2.cpu().numpy() * oracle.matvec(c.n, o.ij, o.blocks, c.gamma0, v2.cpu().numpy()))
        assert np.sqrt(num / den) <= 1e-6 * (1 + 1e-3)
