"""Parity at the full sizes the bench times, in its launch configuration
(the autotuner's choice).  The oracle recomputes everything it can at full
size from the same seeded inputs: the complete contact set (k-d tree
candidates decided by the C scan's exact FP64 test), the friction blocks,
Prim's spanning forest and the tree factor.  Solutions are checked by the
true residual from the oracle's own product and, on the spheroid, against
the oracle's own PCG solve.  Batches are checked on sampled instances."""
import numpy as np
import pytest
import torch

import oracle
import paper_2410_04512_gb300 as sgp
import workloads
from gpu_common import dev_tensor, rel_err
from oracle import mpnn

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def ctx(cuda_device):
    return sgp.Context(0)


class Full:
    """One workload built by the GPU path (through the C ABI) and by the
    oracle, from the same positions, radii and coefficient law."""

    def __init__(self, ctx, c, prec):
        self.c = c
        self.pos, self.radii = dev_tensor(c.pos), dev_tensor(c.radii)
        self.g = ctx.collision_graph(self.pos, self.radii)
        self.ij = self.g.edges()
        tp, tq = c.tables()
        gp, gq = workloads.pair_gamma_torch(c.seed, self.ij, dev_tensor(tp), dev_tensor(tq))
        self.M = ctx.friction_assemble(self.g, self.pos, gp.contiguous(), gq.contiguous(), c.gamma0, prec)
        self.T = ctx.max_spanning_tree(self.M)
        self.Fh = ctx.tree_factor(self.M, self.T)
        # oracle side
        self.o_ij = oracle.contacts_kdtree(c.pos, c.radii)
        self.o = oracle.build_system(c.pos, c.radii, c.gammas_np, c.gamma0, ij=self.o_ij)
        self.mv = lambda x: oracle.matvec(c.n, self.o.ij, self.o.blocks, c.gamma0, x)


def _check_structure(ctx, s):
    """Graph, blocks and spanning forest bit for bit at full size."""
    np.testing.assert_array_equal(s.ij.cpu().numpy(), s.o_ij)
    blocks, w = s.M.edge_blocks()
    np.testing.assert_array_equal(blocks.cpu().numpy(), s.o.blocks)
    np.testing.assert_array_equal(w.cpu().numpy(), s.o.w)
    f = oracle.prim_msf(s.c.n, s.o.ij, s.o.w)
    np.testing.assert_array_equal(s.T.edge_ids().cpu().numpy(), np.sort(f.tree_edges))
    return f


def _true_residual(s, F, v):
    return np.linalg.norm(F - s.mv(v)) / np.linalg.norm(F)


# ------------------------------------------------------------ 1e6 spheroid
@pytest.fixture(scope="module")
def spheroid(ctx):
    import bench
    c = workloads.ball(n=1_000_000, seed=bench.replica_seed(0), gamma0=1e-3)
    s = Full(ctx, c, sgp.PREC_MIXED)
    s.F = c.forces()
    s.tuning = ctx.autotune(s.M, s.T, s.Fh, dev_tensor(s.F), precision=sgp.PREC_MIXED, iterations=10)
    return s


def test_spheroid_structure_bit_exact(ctx, spheroid):
    _check_structure(ctx, spheroid)


def test_spheroid_tree_solve(ctx, spheroid):
    s = spheroid
    f = oracle.prim_msf(s.c.n, s.o.ij, s.o.w)
    fac = oracle.tree_ldlt(f, s.o.blocks, s.c.gamma0)
    b = np.random.default_rng(11).standard_normal((s.c.n, 3))
    got = ctx.tree_apply(s.Fh, dev_tensor(b)).cpu().numpy()
    want = oracle.tree_solve(fac, b)
    te = np.sort(f.tree_edges)
    Px = oracle.matvec(s.c.n, s.o.ij[te], s.o.blocks[te], s.c.gamma0, got)
    norms = np.abs(s.o.blocks[te]).sum(axis=2).max(axis=1)
    rowsum = np.zeros(s.c.n)
    np.add.at(rowsum, s.o.ij[te, 0], norms)
    np.add.at(rowsum, s.o.ij[te, 1], norms)
    pnorm = s.c.gamma0 + 2 * rowsum.max()
    assert np.linalg.norm(Px - b) / (pnorm * np.linalg.norm(got)) <= 1e-14
    assert rel_err(got, want) <= 64 * EPS * pnorm / s.c.gamma0


def test_spheroid_solutions_match_the_oracle(ctx, spheroid):
    """The chosen form (mixed, autotuned) at the bench tolerance reaches it by
    the oracle's own product; solved tightly, both forms agree with the
    oracle's FP64 solve (1e-8 mixed, 1e-9 FP64)."""
    s = spheroid
    Fd = dev_tensor(s.F)
    v, info = ctx.pcg_solve(s.M, s.Fh, Fd, tol=1e-8, precision=sgp.PREC_MIXED)
    assert info.status == 0
    assert _true_residual(s, s.F, v.cpu().numpy()) <= 1.0e-8 * (1 + 1e-6)
    ref, _ = oracle.solve_system(s.o, s.F, tol=1e-12)
    vm, _ = ctx.pcg_solve(s.M, s.Fh, Fd, tol=1e-12, precision=sgp.PREC_MIXED)
    assert rel_err(vm.cpu().numpy(), ref.x) <= 1e-8
    vf, _ = ctx.pcg_solve(s.M, s.Fh, Fd, tol=1e-12, precision=sgp.PREC_F64)
    assert rel_err(vf.cpu().numpy(), ref.x) <= 1e-9


# ------------------------------------------------------------ 4e6 hex sheet
def test_hex_sheet_full_size(ctx):
    c = workloads.hex_sheet(nx=2000, ny=2000, seed=3000)
    s = Full(ctx, c, sgp.PREC_MIXED)
    _check_structure(ctx, s)
    F = c.forces()
    ctx.autotune(s.M, s.T, s.Fh, dev_tensor(F), precision=sgp.PREC_MIXED, iterations=10)
    v, info = ctx.pcg_solve(s.M, s.Fh, dev_tensor(F), tol=1e-10, precision=sgp.PREC_MIXED)
    assert info.status == 0
    assert _true_residual(s, F, v.cpu().numpy()) <= 1e-10 * (1 + 1e-6)


# ------------------------------------------------------------ 512-instance batch
def test_batch512_sampled_instances(ctx):
    sizes = workloads.batch_sizes(512, seed=4000)
    off = workloads.sphere_offsets(sizes)
    cells = [workloads.batch_instance(int(n), k) for k, n in enumerate(sizes)]
    pos = dev_tensor(np.concatenate([c.pos for c in cells]))
    radii = dev_tensor(np.concatenate([c.radii for c in cells]))
    g = ctx.collision_graph_batched(off, pos, radii)
    ij = g.edges()
    tab = dev_tensor(workloads.gamma_table(0.1, 10.0))
    gp, gq = workloads.pair_gamma_torch(4000, ij, tab, tab)
    M = ctx.friction_assemble(g, pos, gp.contiguous(), gq.contiguous(), 1e-2, sgp.PREC_MIXED)
    T = ctx.max_spanning_tree(M)
    Fh = ctx.tree_factor(M, T)
    n = int(off[-1])
    F = np.random.Generator(np.random.PCG64([4000, 7919])).standard_normal((n, 3))
    ctx.autotune(M, T, Fh, dev_tensor(F), offsets=off, precision=sgp.PREC_MIXED, iterations=5)
    v, infos = ctx.pcg_solve_batched(M, Fh, off, dev_tensor(F), tol=1e-8, precision=sgp.PREC_MIXED)
    assert all(i.status == 0 for i in infos)
    v = v.cpu().numpy()
    ij = ij.cpu().numpy()
    # the largest, the smallest and a spread of instances in between
    order = np.argsort(sizes)
    pick = np.unique(np.concatenate([order[:3], order[-3:], order[::64]]))
    tab_np = workloads.gamma_table(0.1, 10.0)
    for k in pick:
        lo, hi = int(off[k]), int(off[k + 1])
        c = cells[k]
        o_ij = oracle.contacts_kdtree(c.pos, c.radii)
        mine = ij[(ij[:, 0] >= lo) & (ij[:, 0] < hi)] - lo
        np.testing.assert_array_equal(mine, o_ij)
        gpn, gqn = workloads.pair_gamma_np(4000, o_ij[:, 0] + lo, o_ij[:, 1] + lo, tab_np, tab_np)
        blocks, _ = oracle.friction_blocks(o_ij, c.pos, gpn, gqn)
        r = F[lo:hi] - oracle.matvec(hi - lo, o_ij, blocks, 1e-2, v[lo:hi])
        assert np.linalg.norm(r) <= 1e-8 * (1 + 1e-6) * np.linalg.norm(F[lo:hi]), k


# ------------------------------------------------------------ 2e5 warm-start spheroid
def test_warm_start_network_full_size(ctx):
    c = workloads.spheroid_200k()
    s = Full(ctx, c, sgp.PREC_MIXED)
    F = workloads.spring_forces_np(c.pos, c.radii, s.o.ij) + workloads.active_noise(c.seed, 1, c.n)
    params = workloads.mpnn_init(5000)
    params[-3:] = (0.2, 0.7, 0.1)
    params[-3 - 3 * mpnn.H:-3] *= 30
    net = ctx.mpnn_create(params)
    v0 = ctx.mpnn_forward(net, s.M, s.Fh, dev_tensor(F), None).cpu().numpy()
    f = oracle.prim_msf(c.n, s.o.ij, s.o.w)
    fac = oracle.tree_ldlt(f, s.o.blocks, c.gamma0)
    Dinv = oracle.block_jacobi(c.n, s.o.ij, s.o.blocks, c.gamma0)
    basis = np.stack([np.einsum("nij,nj->ni", Dinv, F), oracle.tree_solve(fac, F), np.zeros_like(F)])
    ptr, nbr = mpnn.adjacency(c.n, s.o.ij)
    want = mpnn.forward(params.astype(np.float64), basis, ptr, nbr)
    assert np.abs(v0 - want).max() <= 2e-4 * np.abs(want).max()
