"""The augmented spanning-forest preconditioner and the nested flexible CG
(Sections 3.1, 3.3 and 5) through the C ABI against the oracle: pieces and
augmented edges bit for bit, the product with P', flexible-CG iterates at
equal outer and inner iteration counts, and whole solves."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import oracle.augmented as oaug
import paper_2410_04512_gb300 as sgp
import workloads
from gpu_common import GpuSystem, dev_tensor, oracle_system, rel_err, small_cube

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda_device):
    return sgp.Context(0)


def _chain(n=20000):
    pos = np.zeros((n, 3))
    pos[:, 0] = 0.9 * np.arange(n)
    pos[:, 1] = 0.02 * np.sin(0.1 * np.arange(n))
    return workloads.Cells("chain", pos, np.full(n, 0.5), 9, 0.1, 10.0, 1e-3)


def _forest():
    rng = np.random.default_rng(5)
    pos = np.concatenate([rng.uniform(0, 400, size=(300, 3)), rng.uniform(0, 6, size=(200, 3)) + 500.0])
    return workloads.Cells("forest", pos, np.full(pos.shape[0], 0.5), 8, 0.1, 10.0, 1e-2)


CASES = {
    "cube1k": lambda: small_cube(1000, seed=1000),
    "ball60k": lambda: workloads.ball(n=60000, seed=2001, gamma0=1e-3),
    "chain20k": _chain,
    "hex": lambda: workloads.hex_sheet(nx=120, ny=90, seed=3000),
    "forest": _forest,
}
_cache = {}


def _oracle(name):
    """Oracle system and forest of a case (k-d tree contacts above 5000
    cells: pinned to the brute-force scan in the oracle's own tests)."""
    if name not in _cache:
        c = CASES[name]()
        ij = oracle.contacts_kdtree(c.pos, c.radii) if c.n > 5000 else None
        o = oracle_system(c, ij=ij)
        f = oracle.prim_msf(c.n, o.ij, o.w)
        _cache[name] = (c, o, f)
    return _cache[name]


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("t", [1, 2, 0, 37, -1])
def test_pieces_and_edges_match_oracle(ctx, name, t):
    c, o, f = _oracle(name)
    t = c.n if t == -1 else t
    s = GpuSystem(ctx, c)
    assert np.array_equal(s.ij.cpu().numpy(), o.ij)
    assert np.array_equal(s.T.edge_ids().cpu().numpy(), np.sort(f.tree_edges))
    A = ctx.augment_tree(s.M, s.T, t)
    info = A.info()
    want = oaug.build(c.n, o.ij, o.w, f.tree_edges, t)
    assert info["t"] == want.t
    assert info["piece_cap"] == -(-c.n // want.t)
    assert info["pieces"] == want.npieces
    assert np.array_equal(A.pieces(c.n).cpu().numpy(), want.piece)
    assert np.array_equal(A.edges().cpu().numpy(), want.edges)
    assert info["edges"] == want.edges.shape[0] and info["added"] == want.added
    if t == c.n:
        assert info["edges"] == o.ij.shape[0]


@pytest.mark.parametrize("name", ["cube1k", "hex", "forest"])
def test_product_with_P_prime(ctx, name):
    c, o, f = _oracle(name)
    s = GpuSystem(ctx, c)
    A = ctx.augment_tree(s.M, s.T, 0)
    e = A.edges().cpu().numpy()
    P = A.matrix(c.n)
    v = np.random.default_rng(7).standard_normal((c.n, 3))
    got = ctx.spmv(P, dev_tensor(v)).cpu().numpy()
    want = oracle.matvec(c.n, o.ij[e], o.blocks[e], c.gamma0, v)
    assert rel_err(got, want) <= 1e-13
    # every cell its own piece: P' is Gamma, slot for slot, bit for bit
    Aall = ctx.augment_tree(s.M, s.T, c.n)
    Pall = Aall.matrix(c.n)
    vd = dev_tensor(v)
    assert torch.equal(ctx.spmv(Pall, vd), ctx.spmv(s.M, vd))


@pytest.mark.parametrize("k,j", [(1, 1), (4, 3), (15, 2)])
def test_fcg_iterates_at_equal_counts(ctx, k, j):
    """k outer steps with exactly j inner iterations each, against the
    oracle's flexible CG with the same counts: to 1e-9."""
    c = small_cube(3000, seed=1004)
    s = GpuSystem(ctx, c)
    o = oracle_system(c)
    f = oracle.prim_msf(c.n, o.ij, o.w)
    fac = oracle.tree_ldlt(f, o.blocks, c.gamma0)
    want_aug = oaug.build(c.n, o.ij, o.w, f.tree_edges, 0)
    A = ctx.augment_tree(s.M, s.T, 0)
    F = c.forces()
    v, info = ctx.fcg_solve(s.M, A, s.Fac, dev_tensor(F), tol=1e-300, maxit=k, inner_tol=1e-300, inner_maxit=j,
                            raise_on_error=False)
    assert info.status == sgp.ERR_NO_CONVERGENCE
    assert info.outer_iterations == k and info.iterations == k * j
    r = oaug.fcg(c.n, o.ij, o.blocks, c.gamma0, F, want_aug, fac, fixed_iters=k, inner_fixed=j)
    assert r.iters == k and r.inner_iters == k * j
    assert rel_err(v.cpu().numpy(), r.x) <= 1e-9


@pytest.mark.parametrize("name,tol", [("cube1k", 1e-10), ("ball60k", 1e-8), ("hex", 1e-8)])
def test_fcg_solves_to_tolerance(ctx, name, tol):
    c, o, f = _oracle(name)
    s = GpuSystem(ctx, c)
    A = ctx.augment_tree(s.M, s.T, 0)
    F = c.forces()
    v, info = ctx.fcg_solve(s.M, A, s.Fac, dev_tensor(F), tol=tol, inner_tol=0.1)
    assert info.status == 0 and info.rel_residual <= tol
    assert info.iterations >= info.outer_iterations
    # accuracy parity: the oracle's FP64 residual of the GPU solution
    x = v.cpu().numpy()
    res = np.linalg.norm(F - oracle.matvec(c.n, o.ij, o.blocks, c.gamma0, x)) / np.linalg.norm(F)
    assert res <= 1.05 * tol
    assert abs(res - info.true_rel_residual) <= 1e-3 * res + 1e-15
    # the oracle's own flexible CG at the same delta takes about as many steps
    fac = oracle.tree_ldlt(f, o.blocks, c.gamma0)
    want = oaug.fcg(c.n, o.ij, o.blocks, c.gamma0, F, oaug.build(c.n, o.ij, o.w, f.tree_edges, 0), fac,
                    tol=tol, inner_tol=0.1)
    assert abs(info.outer_iterations - want.iters) <= max(3, want.iters // 20)


def test_one_piece_per_tree_is_plain_pcg(ctx):
    """t = 1: T' = T, the inner PCG is exact after one iteration, and the
    flexible iteration is the plain tree-preconditioned PCG."""
    c = small_cube(3000, seed=1005)
    s = GpuSystem(ctx, c)
    A = ctx.augment_tree(s.M, s.T, 1)
    assert A.info()["added"] == 0
    F = dev_tensor(c.forces())
    v, info = ctx.fcg_solve(s.M, A, s.Fac, F, tol=1e-10, inner_tol=1e-12)
    assert info.iterations == info.outer_iterations
    vp, ip = ctx.pcg_solve(s.M, s.Fac, F, tol=1e-10)
    assert abs(info.outer_iterations - ip.iterations) <= 2
    assert rel_err(v.cpu().numpy(), vp.cpu().numpy()) <= 1e-7


def test_edge_cases_and_errors(ctx):
    c = _forest()
    s = GpuSystem(ctx, c)
    A = ctx.augment_tree(s.M, s.T, 3)
    F0 = torch.zeros((c.n, 3), dtype=torch.float64, device="cuda")
    v, info = ctx.fcg_solve(s.M, A, s.Fac, F0)
    assert info.outer_iterations == 0 and info.iterations == 0 and not v.any()
    F = dev_tensor(c.forces())
    v, info = ctx.fcg_solve(s.M, A, s.Fac, F, tol=1e-10)
    assert info.status == 0 and info.true_rel_residual <= 1.05e-10
    with pytest.raises(sgp.SgpError):
        ctx.augment_tree(s.M, s.T, -2)
    with pytest.raises(sgp.SgpError):
        ctx.fcg_solve(s.M, A, s.Fac, F, inner_tol=1.0)
    other = GpuSystem(ctx, small_cube(500, seed=9))
    with pytest.raises(sgp.SgpError):
        ctx.fcg_solve(other.M, A, other.Fac, dev_tensor(np.zeros((500, 3))))
    # warm start: x0 given and already a solution
    v2, info2 = ctx.fcg_solve(s.M, A, s.Fac, F, v=v.clone(), x0_given=True, tol=1e-8)
    assert info2.outer_iterations == 0


def test_fcg_bitwise_reproducible(ctx):
    c = workloads.ball(n=30000, seed=2004, gamma0=1e-3)
    F = dev_tensor(c.forces())
    out = []
    for _ in range(2):
        s = GpuSystem(ctx, c)
        A = ctx.augment_tree(s.M, s.T, 0)
        v, info = ctx.fcg_solve(s.M, A, s.Fac, F, tol=1e-8)
        out.append((v, info.outer_iterations, info.iterations))
    assert out[0][1:] == out[1][1:]
    assert torch.equal(out[0][0], out[1][0])
