"""Batched solves (many independent configurations in one solve) against
the oracle solving each instance on its own.

The instances are balls centred at the same point, so they overlap in
space: the batched collision graph must still never join two instances.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2410_04512_gb300 as sgp
import workloads
from gpu_common import dev_tensor, rel_err

pytestmark = pytest.mark.gpu

SEED = 4000


@pytest.fixture(scope="module")
def ctx(cuda_device):
    return sgp.Context(0)


def make_batch(sizes, seed0=SEED):
    cells = [workloads.batch_instance(int(n), s, seed0=seed0) if n > 0 else None for s, n in enumerate(sizes)]
    off = workloads.sphere_offsets(np.asarray(sizes, dtype=np.int64))
    pos = np.concatenate([c.pos for c in cells if c is not None] or [np.zeros((0, 3))])
    radii = np.concatenate([c.radii for c in cells if c is not None] or [np.zeros(0)])
    return cells, off, np.ascontiguousarray(pos), np.ascontiguousarray(radii)


def batch_gammas(ij, lo=0.1, hi=10.0):
    t = workloads.gamma_table(lo, hi)
    return workloads.pair_gamma_np(SEED, ij[:, 0], ij[:, 1], t, t)


class GpuBatch:
    def __init__(self, ctx, sizes, precision=sgp.PREC_F64):
        self.cells, self.off, pos, radii = make_batch(sizes)
        self.pos, self.radii = dev_tensor(pos), dev_tensor(radii)
        self.g = ctx.collision_graph_batched(self.off, self.pos, self.radii)
        self.ij = self.g.edges()
        t = dev_tensor(workloads.gamma_table(0.1, 10.0))
        gp, gq = workloads.pair_gamma_torch(SEED, self.ij, t, t)
        self.M = ctx.friction_assemble(self.g, self.pos, gp.contiguous(), gq.contiguous(), 1e-2, precision)
        self.T = ctx.max_spanning_tree(self.M)
        self.Fh = ctx.tree_factor(self.M, self.T)
        n = int(self.off[-1])
        self.F = np.random.default_rng(5).standard_normal((n, 3))


def oracle_instance(b, s):
    lo, hi = int(b.off[s]), int(b.off[s + 1])
    c = b.cells[s]
    ij = oracle.contacts(c.pos, c.radii)
    gp, gq = batch_gammas(ij + lo)
    blocks, w = oracle.friction_blocks(ij, c.pos, gp, gq)
    return oracle.System(hi - lo, ij, gp, gq, blocks, w, 1e-2)


SIZES = [300, 1200, 0, 1, 2500, 700, 4000, 950, 2, 1800]


def test_batched_graph_bit_exact_and_separate(ctx):
    b = GpuBatch(ctx, SIZES)
    want = []
    for s, c in enumerate(b.cells):
        if c is not None:
            want.append(oracle.contacts(c.pos, c.radii) + int(b.off[s]))
    want = np.concatenate(want)
    np.testing.assert_array_equal(b.ij.cpu().numpy(), want)
    # the same cells as one configuration do touch across instances
    g1 = ctx.collision_graph(b.pos, b.radii)
    assert g1.m > b.g.m


@pytest.mark.parametrize("precond", [sgp.PRECOND_TREE, sgp.PRECOND_BLOCK_JACOBI])
def test_batched_fp64_matches_oracle_per_instance(ctx, precond):
    b = GpuBatch(ctx, SIZES)
    v, infos = ctx.pcg_solve_batched(b.M, b.Fh, b.off, dev_tensor(b.F), tol=1e-13, precond=precond)
    x = v.cpu().numpy()
    omap = {sgp.PRECOND_TREE: oracle.PRECOND_TREE, sgp.PRECOND_BLOCK_JACOBI: oracle.PRECOND_JACOBI}[precond]
    for s in range(len(SIZES)):
        lo, hi = int(b.off[s]), int(b.off[s + 1])
        if hi == lo:
            assert infos[s].iterations == 0
            continue
        o = oracle_instance(b, s)
        ref, _ = oracle.solve_system(o, b.F[lo:hi], tol=1e-13, precond=omap)
        assert rel_err(x[lo:hi], ref.x) <= 1e-9, s
        assert infos[s].true_rel_residual <= 2e-13
    # iteration counts at 1e-8 agree with the oracle's, instance by instance
    v2, infos2 = ctx.pcg_solve_batched(b.M, b.Fh, b.off, dev_tensor(b.F), tol=1e-8, precond=precond)
    for s in range(len(SIZES)):
        lo, hi = int(b.off[s]), int(b.off[s + 1])
        if hi - lo < 2:
            continue
        o = oracle_instance(b, s)
        ref, _ = oracle.solve_system(o, b.F[lo:hi], tol=1e-8, precond=omap)
        assert abs(infos2[s].iterations - ref.iters) <= 2, (s, infos2[s].iterations, ref.iters)


def test_batched_mixed_precision_error(ctx):
    b = GpuBatch(ctx, SIZES, precision=sgp.PREC_MIXED)
    v, infos = ctx.pcg_solve_batched(b.M, b.Fh, b.off, dev_tensor(b.F), tol=1e-10, precision=sgp.PREC_MIXED)
    x = v.cpu().numpy()
    for s in range(len(SIZES)):
        lo, hi = int(b.off[s]), int(b.off[s + 1])
        if hi == lo:
            continue
        assert infos[s].status == 0 and infos[s].true_rel_residual <= 1e-10
        o = oracle_instance(b, s)
        ref, _ = oracle.solve_system(o, b.F[lo:hi], tol=1e-13)
        assert rel_err(x[lo:hi], ref.x) <= 1e-8, s


def test_batched_matches_single_solves(ctx):
    """The batch gives each instance what a solve of that instance alone gives."""
    b = GpuBatch(ctx, [1500, 2200, 900])
    v, infos = ctx.pcg_solve_batched(b.M, b.Fh, b.off, dev_tensor(b.F), tol=1e-10)
    for s in range(3):
        lo, hi = int(b.off[s]), int(b.off[s + 1])
        c = b.cells[s]
        pos = dev_tensor(c.pos)
        g = ctx.collision_graph(pos, dev_tensor(c.radii))
        ij = g.edges().to(torch.int64) + lo
        t = dev_tensor(workloads.gamma_table(0.1, 10.0))
        gp, gq = workloads.pair_gamma_torch(SEED, ij, t, t)
        M = ctx.friction_assemble(g, pos, gp.contiguous(), gq.contiguous(), 1e-2)
        Fh = ctx.tree_factor(M, ctx.max_spanning_tree(M))
        v1, i1 = ctx.pcg_solve(M, Fh, dev_tensor(b.F[lo:hi]), tol=1e-10)
        assert abs(i1.iterations - infos[s].iterations) <= 1
        assert rel_err(v[lo:hi].cpu().numpy(), v1.cpu().numpy()) <= 1e-8


def test_batched_rejects_edges_between_instances(ctx):
    cells, off, pos, radii = make_batch([800, 900])
    pos_d, radii_d = dev_tensor(pos), dev_tensor(radii)
    g = ctx.collision_graph(pos_d, radii_d)         # not batched: instances touch
    ij = g.edges()
    t = dev_tensor(workloads.gamma_table(0.1, 10.0))
    gp, gq = workloads.pair_gamma_torch(SEED, ij, t, t)
    M = ctx.friction_assemble(g, pos_d, gp.contiguous(), gq.contiguous(), 1e-2)
    with pytest.raises(sgp.SgpError) as e:
        ctx.pcg_solve_batched(M, None, off, dev_tensor(np.ones((int(off[-1]), 3))), precond=sgp.PRECOND_NONE)
    assert e.value.code == sgp.ERR_INVALID_ARG


def test_batched_rejects_a_cell_order_that_mixes_instances(ctx):
    """Two instances far apart (no edge between them) assembled on a graph of
    the whole union: the graph's grid-cell order interleaves them, which the
    batched solver cannot use, so it must refuse rather than mix them; the
    same union solved as one system is fine."""
    cells, off, pos, radii = make_batch([700, 900])
    pos = pos.copy()
    lo = int(off[1])
    pos[lo:, 2] += 1000.0     # far away along the grid's fastest axis: their cells interleave
    pos_d, radii_d = dev_tensor(pos), dev_tensor(radii)
    g = ctx.collision_graph(pos_d, radii_d)
    ij = g.edges()
    assert not ((ij[:, 0] < lo) & (ij[:, 1] >= lo)).any()
    t = dev_tensor(workloads.gamma_table(0.1, 10.0))
    gp, gq = workloads.pair_gamma_torch(SEED, ij, t, t)
    M = ctx.friction_assemble(g, pos_d, gp.contiguous(), gq.contiguous(), 1e-2)
    F = dev_tensor(np.ones((int(off[-1]), 3)))
    with pytest.raises(sgp.SgpError) as e:
        ctx.pcg_solve_batched(M, None, off, F, precond=sgp.PRECOND_NONE)
    assert e.value.code == sgp.ERR_INVALID_ARG
    v, info = ctx.pcg_solve(M, None, F, tol=1e-10, precond=sgp.PRECOND_NONE)
    assert info.status == 0 and info.true_rel_residual <= 1e-10
