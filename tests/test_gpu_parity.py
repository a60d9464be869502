"""Parity of the CUDA path (called through the C ABI) with the CPU oracle.

Integer and index work (edge lists, spanning-forest edge sets) must match
bit for bit; friction blocks and weights too (both sides evaluate eq. (1)
with the same round-to-nearest operations).  Floating-point results are
compared element-wise against the oracle on the same seeded inputs, with
the tolerances stated in each test.
"""
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


def cases():
    return [
        small_cube(1000, seed=1000),
        small_cube(3000, seed=1001),
        workloads.ball(n=4000, seed=2000, gamma0=1e-3),
        workloads.hex_sheet(nx=70, ny=50, seed=3000),
    ]


# ---------------------------------------------------------------- graph (a1)
@pytest.mark.parametrize("k", range(4))
def test_collision_graph_bit_exact(ctx, k):
    c = cases()[k]
    g = ctx.collision_graph(dev_tensor(c.pos), dev_tensor(c.radii))
    got = g.edges().cpu().numpy()
    want = oracle.contacts(c.pos, c.radii)
    assert got.shape == want.shape
    np.testing.assert_array_equal(got, want)


def test_collision_graph_tiny_and_empty(ctx):
    for pos, radii in [
        (np.zeros((1, 3)), np.array([0.5])),
        (np.array([[0.0, 0, 0], [0.9, 0, 0]]), np.array([0.5, 0.5])),
        (np.array([[0.0, 0, 0], [3.0, 0, 0], [9.0, 0, 0]]), np.array([0.5, 0.5, 0.5])),
        (np.array([[0.0, 0, 0], [1.0, 0, 0]]), np.array([0.5, 0.5])),    # touching: d == R_i + R_j
    ]:
        g = ctx.collision_graph(dev_tensor(pos), dev_tensor(radii))
        np.testing.assert_array_equal(g.edges().cpu().numpy(), oracle.contacts(pos, radii))


def test_collision_graph_crowded_cells(ctx):
    """Cells with more contacts than the single search keeps per cell (24):
    a large sphere ringed by 60 small ones (its contacts all have larger
    indices), also with the large sphere last; the second search path must
    give the same edge list as the oracle."""
    rng = np.random.default_rng(7)
    d = rng.standard_normal((60, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    ring = 3.3 * d
    for big_first, pos, radii in [
        (True, np.vstack([[0.0, 0, 0], ring]), np.concatenate([[3.0], np.full(60, 0.45)])),
        (False, np.vstack([ring, [0.0, 0, 0]]), np.concatenate([np.full(60, 0.45), [3.0]])),
    ]:
        g = ctx.collision_graph(dev_tensor(pos), dev_tensor(radii))
        want = oracle.contacts(pos, radii)
        upper = np.bincount(want[:, 0], minlength=61)
        assert (upper.max() > 24) == big_first
        np.testing.assert_array_equal(g.edges().cpu().numpy(), want)


def test_collision_graph_rejects_bad_input(ctx):
    pos = dev_tensor(np.zeros((3, 3)))
    with pytest.raises(sgp.SgpError) as e:
        ctx.collision_graph(pos, dev_tensor(np.array([0.5, -0.1, 0.5])))
    assert e.value.code == sgp.ERR_INVALID_ARG
    bad = np.zeros((3, 3))
    bad[1, 1] = np.nan
    with pytest.raises(sgp.SgpError):
        ctx.collision_graph(dev_tensor(bad), dev_tensor(np.full(3, 0.5)))


# ------------------------------------------------------- blocks, weights (a2)
@pytest.mark.parametrize("k", range(4))
def test_friction_blocks_bit_exact(ctx, k):
    c = cases()[k]
    s = GpuSystem(ctx, c, tree=False)
    o = oracle_system(c)
    np.testing.assert_array_equal(s.ij.cpu().numpy(), o.ij)
    np.testing.assert_array_equal(s.gp.cpu().numpy(), o.g_par)
    np.testing.assert_array_equal(s.gq.cpu().numpy(), o.g_perp)
    blocks, w = s.M.edge_blocks()
    np.testing.assert_array_equal(blocks.cpu().numpy(), o.blocks)
    np.testing.assert_array_equal(w.cpu().numpy(), o.w)


def test_degenerate_centres_rejected(ctx):
    pos = np.array([[0.0, 0, 0], [0.0, 0, 0], [3.0, 0, 0]])
    g = ctx.collision_graph(dev_tensor(pos), dev_tensor(np.full(3, 0.5)))
    one = dev_tensor(np.ones(1))
    with pytest.raises(sgp.SgpError) as e:
        ctx.friction_assemble(g, dev_tensor(pos), one, one, 1e-2)
    assert e.value.code == sgp.ERR_DEGENERATE
    pos2 = dev_tensor(np.array([[0.0, 0, 0], [0.9, 0, 0]]))
    g2 = ctx.collision_graph(pos2, dev_tensor(np.full(2, 0.5)))
    with pytest.raises(sgp.SgpError) as e:
        ctx.friction_assemble(g2, pos2, dev_tensor(np.array([0.0])), one, 1e-2)
    assert e.value.code == sgp.ERR_INVALID_ARG


# ------------------------------------------------------------- product (a6)
@pytest.mark.parametrize("k", range(4))
def test_spmv_matches_oracle(ctx, k):
    c = cases()[k]
    s = GpuSystem(ctx, c, tree=False)
    o = oracle_system(c)
    v = np.random.default_rng(k).standard_normal((c.n, 3))
    got = ctx.spmv(s.M, dev_tensor(v)).cpu().numpy()
    want = oracle.matvec(c.n, o.ij, o.blocks, c.gamma0, v)
    scale = np.abs(want).max()
    assert np.max(np.abs(got - want)) <= 1e-13 * scale
    # rigid translations: only the substrate term survives, exactly
    t = np.tile([0.3, -1.7, 2.25], (c.n, 1))
    np.testing.assert_array_equal(ctx.spmv(s.M, dev_tensor(t)).cpu().numpy(), c.gamma0 * t)


# ------------------------------------------------------ spanning forest (a3)
@pytest.mark.parametrize("k", range(4))
def test_spanning_forest_bit_exact(ctx, k):
    c = cases()[k]
    s = GpuSystem(ctx, c)
    o = oracle_system(c)
    f = oracle.prim_msf(c.n, o.ij, o.w)
    got = s.T.edge_ids().cpu().numpy()
    np.testing.assert_array_equal(got, np.sort(f.tree_edges))
    ne, ncomp, _ = s.T.info()
    assert ne == len(f.tree_edges) and ncomp == c.n - ne


def test_spanning_forest_with_all_weights_tied(ctx):
    """Constant coefficients: every weight ties, the edge index decides."""
    c = small_cube(800, seed=5, lo=2.0, hi=2.0)
    s = GpuSystem(ctx, c)
    o = oracle_system(c)
    assert np.all(o.w == o.w[0])
    f = oracle.prim_msf(c.n, o.ij, o.w)
    np.testing.assert_array_equal(s.T.edge_ids().cpu().numpy(), np.sort(f.tree_edges))


# ---------------------------------------------------- tree factor/solve (a4, a5, a7)
EPS = np.finfo(np.float64).eps


def _tree_check(ctx, c, seed=0, precision=sgp.PREC_F64):
    """Forward error of the GPU tree solve against the oracle's, and the
    tolerance the arithmetic allows: both are backward stable solves of
    P x = b in different elimination orders, so they may differ by about
    eps * kappa(P); kappa(P) <= (gamma0 + 2 max_i sum_j |Upsilon_ij|) / gamma0
    (Gershgorin; lambda_min(P) >= gamma0 by Lemma 2.4).  The backward error
    |P x - b| / (|P| |x|) must be at rounding level regardless of kappa."""
    s = GpuSystem(ctx, c, precision=precision)
    o = oracle_system(c)
    f = oracle.prim_msf(c.n, o.ij, o.w)
    fac = oracle.tree_ldlt(f, o.blocks, c.gamma0)
    b = np.random.default_rng(seed).standard_normal((c.n, 3))
    got = ctx.tree_apply(s.Fac, dev_tensor(b)).cpu().numpy()
    want = oracle.tree_solve(fac, b)
    te = np.sort(f.tree_edges)
    norms = np.abs(o.blocks[te]).sum(axis=2).max(axis=1)
    rowsum = np.zeros(c.n)
    np.add.at(rowsum, o.ij[te, 0], norms)
    np.add.at(rowsum, o.ij[te, 1], norms)
    pnorm = c.gamma0 + 2 * rowsum.max()
    kappa = pnorm / c.gamma0
    Px = oracle.matvec(c.n, o.ij[te], o.blocks[te], c.gamma0, got)
    back = np.linalg.norm(Px - b) / (pnorm * np.linalg.norm(got))
    assert back <= 1e-14, back
    return rel_err(got, want), 64 * EPS * kappa, s


@pytest.mark.parametrize("k", range(4))
def test_tree_solve_matches_oracle(ctx, k):
    err, tol, s = _tree_check(ctx, cases()[k], k)
    assert err <= tol, (err, tol)
    rounds, levels = s.Fac.info()
    assert rounds <= 4 * np.log2(s.n) + 8


@pytest.mark.parametrize("k", [1, 2])
def test_tree_solve_fp64_apply_of_mixed_factor(ctx, k):
    """A MIXED factor sizes its shared-memory tail for FP32 vectors; an FP64
    apply of it (the public call) must still be the FP64 solve."""
    err, tol, _ = _tree_check(ctx, cases()[k], k, precision=sgp.PREC_MIXED)
    assert err <= tol, (err, tol)


def test_tree_solve_mid_size_ball(ctx):
    """60,000 cells: many level kernels before the tail, in both precisions."""
    c = workloads.ball(n=60000, seed=2001, gamma0=1e-3)
    for prec in (sgp.PREC_F64, sgp.PREC_MIXED):
        s = GpuSystem(ctx, c, precision=prec)
        b = np.random.default_rng(3).standard_normal((c.n, 3))
        x = ctx.tree_apply(s.Fac, dev_tensor(b)).cpu().numpy()
        te = s.T.edge_ids().cpu().numpy()
        ij = s.ij.cpu().numpy()[te]
        blocks = s.M.edge_blocks()[0].cpu().numpy()[te]
        Px = oracle.matvec(c.n, ij, blocks, c.gamma0, x)
        norms = np.abs(blocks).sum(axis=2).max(axis=1)
        rowsum = np.zeros(c.n)
        np.add.at(rowsum, ij[:, 0], norms)
        np.add.at(rowsum, ij[:, 1], norms)
        pnorm = c.gamma0 + 2 * rowsum.max()
        back = np.linalg.norm(Px - b) / (pnorm * np.linalg.norm(x))
        assert back <= 1e-14, (prec, back)


def test_tree_solve_long_chain(ctx):
    """A chain of 20000 cells: depth 20000, contraction must still take
    O(log n) rounds."""
    n = 20000
    pos = np.zeros((n, 3))
    pos[:, 0] = 0.9 * np.arange(n)
    pos[:, 1] = 0.02 * np.sin(0.1 * np.arange(n))
    cells = workloads.Cells("chain", pos, np.full(n, 0.5), 9, 0.1, 10.0, 1e-3)
    err, tol, s = _tree_check(ctx, cells)
    assert err <= tol, (err, tol)
    rounds, _ = s.Fac.info()
    assert rounds <= 60, rounds


def test_tree_solve_star(ctx):
    """A star: one centre touching 12 cells, plus isolated cells."""
    d = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                  [1, 1, 0], [-1, -1, 0], [1, 0, 1], [0, -1, -1], [-1, 1, 0], [0, 1, -1]], float)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pos = np.vstack([[0, 0, 0], 0.95 * d, [[50, 0, 0], [60, 0, 0]]])
    radii = np.concatenate([[0.5], np.full(12, 0.5), [0.5, 0.5]])
    cells = workloads.Cells("star", pos, radii, 3, 0.1, 10.0, 1e-2)
    err, tol, _ = _tree_check(ctx, cells)
    assert err <= tol, (err, tol)


# ------------------------------------------------------------------ PCG (a8)
def test_pcg_same_iterations_as_oracle(ctx):
    c = small_cube(1000, seed=1000)
    s = GpuSystem(ctx, c)
    o = oracle_system(c)
    F = c.forces()
    f = oracle.prim_msf(c.n, o.ij, o.w)
    fac = oracle.tree_ldlt(f, o.blocks, c.gamma0)
    for k in (1, 5, 30):
        v, info = ctx.pcg_solve(s.M, s.Fac, dev_tensor(F), tol=1e-300, maxit=k, raise_on_error=False)
        assert info.iterations == k and info.status == sgp.ERR_NO_CONVERGENCE
        r = oracle.pcg(c.n, o.ij, o.blocks, c.gamma0, F, oracle.PRECOND_TREE, fac, fixed_iters=k)
        assert rel_err(v.cpu().numpy(), r.x) <= 1e-9


@pytest.mark.parametrize("precond", [sgp.PRECOND_TREE, sgp.PRECOND_BLOCK_JACOBI, sgp.PRECOND_NONE])
def test_pcg_solution_matches_oracle(ctx, precond):
    c = small_cube(1000, seed=1000)
    s = GpuSystem(ctx, c)
    o = oracle_system(c)
    F = c.forces()
    omap = {sgp.PRECOND_TREE: oracle.PRECOND_TREE, sgp.PRECOND_BLOCK_JACOBI: oracle.PRECOND_JACOBI,
            sgp.PRECOND_NONE: oracle.PRECOND_NONE}[precond]
    # iteration counts at the cube workload's tolerance agree within 2
    v, info = ctx.pcg_solve(s.M, s.Fac, dev_tensor(F), tol=1e-10, precond=precond)
    r, _ = oracle.solve_system(o, F, tol=1e-10, precond=omap)
    assert abs(info.iterations - r.iters) <= 2, (info.iterations, r.iters)
    assert info.true_rel_residual <= 2e-10
    xt = oracle.matvec(c.n, o.ij, o.blocks, c.gamma0, v.cpu().numpy())
    assert np.linalg.norm(F - xt) / np.linalg.norm(F) <= 2e-10
    # solutions agree to 1e-9 when both are converged tightly
    v2, _ = ctx.pcg_solve(s.M, s.Fac, dev_tensor(F), tol=1e-13, precond=precond)
    r2, _ = oracle.solve_system(o, F, tol=1e-13, precond=omap)
    assert rel_err(v2.cpu().numpy(), r2.x) <= 1e-9


def test_pcg_initial_guess_and_zero_rhs(ctx):
    c = small_cube(1000, seed=1002)
    s = GpuSystem(ctx, c)
    F = dev_tensor(c.forces())
    v, info = ctx.pcg_solve(s.M, s.Fac, torch.zeros_like(F), tol=1e-8)
    assert info.iterations == 0 and not v.any()
    v1, info1 = ctx.pcg_solve(s.M, s.Fac, F, tol=1e-12)
    v2, info2 = ctx.pcg_solve(s.M, s.Fac, F, v1.clone(), tol=1e-10, x0_given=True)
    assert info2.iterations == 0
    v3 = v1 + 1e-3 * torch.randn_like(v1)
    v4, info4 = ctx.pcg_solve(s.M, s.Fac, F, v3, tol=1e-12, x0_given=True)
    assert info4.true_rel_residual <= 2e-12
    assert rel_err(v4.cpu().numpy(), v1.cpu().numpy()) <= 1e-9


def test_pcg_bitwise_reproducible(ctx):
    c = workloads.ball(n=6000, seed=2001, gamma0=1e-3)
    s = GpuSystem(ctx, c)
    F = dev_tensor(c.forces())
    v1, i1 = ctx.pcg_solve(s.M, s.Fac, F, tol=1e-8)
    s2 = GpuSystem(ctx, c)
    v2, i2 = ctx.pcg_solve(s2.M, s2.Fac, F, tol=1e-8)
    assert i1.iterations == i2.iterations
    assert torch.equal(v1, v2)


def test_pcg_isolated_cells(ctx):
    pos = np.array([[0.0, 0, 0], [5.0, 0, 0], [5.9, 0, 0], [20.0, 0, 0]])
    cells = workloads.Cells("iso", pos, np.full(4, 0.5), 5, 0.1, 10.0, 0.5)
    s = GpuSystem(ctx, cells)
    F = cells.forces()
    v, info = ctx.pcg_solve(s.M, s.Fac, dev_tensor(F), tol=1e-13)
    o = oracle_system(cells)
    r, _ = oracle.solve_system(o, F, tol=1e-13)
    assert rel_err(v.cpu().numpy(), r.x) <= 1e-12


# ------------------------------------------------------- mixed precision (a10)
def test_mixed_precision_error_vs_fp64_oracle(ctx):
    c = workloads.hex_sheet(nx=80, ny=80, seed=3000)
    s = GpuSystem(ctx, c, precision=sgp.PREC_MIXED)
    o = oracle_system(c)
    F = c.forces()
    v, info = ctx.pcg_solve(s.M, s.Fac, dev_tensor(F), tol=1e-10, precision=sgp.PREC_MIXED)
    assert info.status == 0 and info.true_rel_residual <= 1e-10
    ref, _ = oracle.solve_system(o, F, tol=1e-13)
    assert rel_err(v.cpu().numpy(), ref.x) <= 1e-8
    assert info.outer_iterations >= 2
