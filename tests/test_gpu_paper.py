"""The paper's experiment geometries (Section 5: noisy hexagonal close
packing, rejection-sampled spheroid, dumbbell; equal cells, Hertz contact
areas) through the C ABI against the oracle: contact graphs, blocks and
spanning forests bit for bit, and PCG with every preconditioner."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2410_04512_gb300 as sgp
import workloads
from gpu_common import GpuSystem, dev_tensor, oracle_system, rel_err

pytestmark = pytest.mark.gpu

CASES = {
    "hex": lambda: workloads.paper_hex(n=3000, seed=6001),
    "hex_high_kappa": lambda: workloads.paper_hex(n=3000, seed=6002, gamma_med=3.0e3),
    "random": lambda: workloads.paper_random(n=3000, seed=7001),
    "dumbbell": lambda: workloads.paper_dumbbell(n=3000, seed=8001),
}


@pytest.fixture(scope="module")
def ctx(cuda_device):
    return sgp.Context(0)


@pytest.mark.parametrize("name", sorted(CASES))
def test_graph_blocks_and_forest_bit_exact(ctx, name):
    c = CASES[name]()
    s = GpuSystem(ctx, c)
    o = oracle_system(c)
    np.testing.assert_array_equal(s.ij.cpu().numpy(), o.ij)
    np.testing.assert_array_equal(s.gp.cpu().numpy(), o.g_par)
    np.testing.assert_array_equal(s.gq.cpu().numpy(), o.g_perp)
    blocks, w = s.M.edge_blocks()
    np.testing.assert_array_equal(blocks.cpu().numpy(), o.blocks)
    np.testing.assert_array_equal(w.cpu().numpy(), o.w)
    f = oracle.prim_msf(c.n, o.ij, o.w)
    np.testing.assert_array_equal(s.T.edge_ids().cpu().numpy(), np.sort(f.tree_edges))


@pytest.mark.parametrize("name", sorted(CASES))
def test_known_solution_recovered(ctx, name):
    """F = Gamma x* for a known x* (the paper's protocol): every
    preconditioner recovers x*, in the number of iterations the oracle's PCG
    takes on the same system."""
    c = CASES[name]()
    s = GpuSystem(ctx, c)
    o = oracle_system(c)
    xs = np.random.default_rng(5).standard_normal((c.n, 3))
    F = oracle.matvec(c.n, o.ij, o.blocks, c.gamma0, xs)
    fac = oracle.tree_ldlt(oracle.prim_msf(c.n, o.ij, o.w), o.blocks, c.gamma0)
    dj = oracle.block_jacobi(c.n, o.ij, o.blocks, c.gamma0)
    for pc, opc in ((sgp.PRECOND_TREE, oracle.PRECOND_TREE), (sgp.PRECOND_BLOCK_JACOBI, oracle.PRECOND_JACOBI),
                    (sgp.PRECOND_NONE, oracle.PRECOND_NONE)):
        v, info = ctx.pcg_solve(s.M, s.Fac, dev_tensor(F), tol=1e-12, precond=pc)
        assert info.status == 0
        assert rel_err(v.cpu().numpy(), xs) <= 1e-6, (name, pc)
        r = oracle.pcg(c.n, o.ij, o.blocks, c.gamma0, F, opc, fac, jacobi_dinv=dj, tol=1e-12)
        # the same recurrence; rounding (summation order) moves the count a little
        assert abs(r.iters - info.iterations) <= max(3, 0.02 * r.iters), (name, pc, r.iters, info.iterations)
    # error-bound stopping at the paper's 1e-5 meets it in the Gamma norm
    v, info = ctx.pcg_solve(s.M, s.Fac, dev_tensor(F), tol=1e-5, stop=sgp.STOP_ERROR)
    e = xs - v.cpu().numpy()
    rel = np.sqrt(np.sum(e * oracle.matvec(c.n, o.ij, o.blocks, c.gamma0, e)) /
                  np.sum(v.cpu().numpy() * oracle.matvec(c.n, o.ij, o.blocks, c.gamma0, v.cpu().numpy())))
    assert rel <= 1e-5 * (1 + 1e-6)
