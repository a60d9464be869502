"""Pins of the CPU oracle to facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, a dense LAPACK computation, brute force on tiny inputs, an
independent algorithm (Kruskal, exhaustive enumeration), or a bound the
paper proves.  Chosen so that a dropped term, a wrong sign, a wrong index or
a transposed operand in the oracle fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import workloads

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def small_cells(n=120, seed=11, side=None, gamma_lo=0.1, gamma_hi=10.0, gamma0=1e-2):
    if side is None:
        side = (n / 1.4253) ** (1.0 / 3.0)
    return workloads.cube(n=n, side=side, seed=seed, gamma_lo=gamma_lo, gamma_hi=gamma_hi,
                          gamma0=gamma0)


def system_of(cells):
    return oracle.build_system(cells.pos, cells.radii, cells.gammas_np, cells.gamma0)


# ---------------------------------------------------------------------------
# Lemma 2.1: Upsilon is SPD with eigenvalue g_par on span(u) and g_perp twice
# on its complement; |Upsilon| = g_max; the tree weight is min(g_par, g_perp).
# ---------------------------------------------------------------------------
def test_block_eigenstructure_lemma_2_1():
    c = small_cells(200, seed=3)
    s = system_of(c)
    assert s.ij.shape[0] > 100
    u = c.pos[s.ij[:, 1]] - c.pos[s.ij[:, 0]]
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    for e in range(s.ij.shape[0]):
        B = s.blocks[e]
        assert np.array_equal(B, B.T)
        # eigenvector u with eigenvalue g_par
        np.testing.assert_allclose(B @ u[e], s.g_par[e] * u[e], rtol=1e-13, atol=1e-13 * s.g_par[e])
        lam = np.linalg.eigvalsh(B)
        want = np.sort([s.g_par[e], s.g_perp[e], s.g_perp[e]])
        np.testing.assert_allclose(lam, want, rtol=1e-12)
        assert s.w[e] == min(s.g_par[e], s.g_perp[e])
        np.testing.assert_allclose(np.linalg.norm(B, 2), max(s.g_par[e], s.g_perp[e]), rtol=1e-12)


# ---------------------------------------------------------------------------
# Two cells (closed form of eq. (2)): x1 = 0, x2 = (s, 0, 0), s < R1 + R2.
# u = e_x, Upsilon = diag(g_par, g_perp, g_perp).  Per axis k with
# g = (g_par, g_perp, g_perp)_k the sum mode has eigenvalue gamma0 and the
# difference mode gamma0 + 2g:
#   v1 = ((F1+F2)/gamma0 + (F1-F2)/(gamma0+2g)) / 2,
#   v2 = ((F1+F2)/gamma0 - (F1-F2)/(gamma0+2g)) / 2.
# The spanning tree is the graph itself, so P = Gamma and PCG converges in
# one iteration.
# ---------------------------------------------------------------------------
def _read_golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    vals = {}
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = line.split("=", 1)
            vals[k.strip()] = np.array([float(t) for t in v.split()])
    return vals


def test_two_cell_closed_form():
    g = _read_golden("two_cell.txt")
    pos = g["pos"].reshape(2, 3)
    radii = g["radii"]
    gp, gq, g0 = float(g["gamma_par"][0]), float(g["gamma_perp"][0]), float(g["gamma0"][0])
    F = g["F"].reshape(2, 3)
    ij = oracle.contacts(pos, radii)
    assert ij.tolist() == [[0, 1]]
    blocks, w = oracle.friction_blocks(ij, pos, [gp], [gq])
    np.testing.assert_array_equal(blocks[0], np.diag([gp, gq, gq]))
    assert w[0] == min(gp, gq)
    gk = np.array([gp, gq, gq])
    v1 = 0.5 * ((F[0] + F[1]) / g0 + (F[0] - F[1]) / (g0 + 2 * gk))
    v2 = 0.5 * ((F[0] + F[1]) / g0 - (F[0] - F[1]) / (g0 + 2 * gk))
    want = np.stack([v1, v2])
    np.testing.assert_allclose(want, g["v"].reshape(2, 3), rtol=1e-12)
    sysm = oracle.System(2, ij, np.array([gp]), np.array([gq]), blocks, w, g0)
    res, fac = oracle.solve_system(sysm, F, tol=1e-14)
    assert res.iters == 1
    np.testing.assert_allclose(res.x, want, rtol=1e-12)
    # the tree solve alone is the exact inverse here (P = Gamma)
    np.testing.assert_allclose(oracle.tree_solve(fac, F), want, rtol=1e-12)


def test_two_cell_rotated_normal():
    """The same pair along a general direction: Upsilon u = g_par u and
    Upsilon w = g_perp w for w orthogonal to u."""
    pos = np.array([[0.1, -0.2, 0.3], [0.5, 0.2, 0.7]])
    radii = np.array([0.5, 0.5])
    ij = oracle.contacts(pos, radii)
    B, w = oracle.friction_blocks(ij, pos, [2.0], [7.0])
    u = (pos[1] - pos[0]) / np.linalg.norm(pos[1] - pos[0])
    a = np.cross(u, [1.0, 0.0, 0.0])
    a /= np.linalg.norm(a)
    b = np.cross(u, a)
    np.testing.assert_allclose(B[0] @ u, 2.0 * u, atol=1e-14)
    np.testing.assert_allclose(B[0] @ a, 7.0 * a, atol=1e-14)
    np.testing.assert_allclose(B[0] @ b, 7.0 * b, atol=1e-14)


# ---------------------------------------------------------------------------
# Collision graph: brute force against a k-d tree candidate search
# ---------------------------------------------------------------------------
def test_contacts_against_kdtree():
    from scipy.spatial import cKDTree
    c = small_cells(600, seed=5)
    ij = oracle.contacts(c.pos, c.radii)
    assert np.all(ij[:, 0] < ij[:, 1])
    key = ij[:, 0].astype(np.int64) * c.n + ij[:, 1]
    assert np.all(np.diff(key) > 0), "sorted by (i, j), no duplicates"
    cand = cKDTree(c.pos).query_pairs(2 * c.radii.max() + 1e-9, output_type="ndarray")
    d = np.linalg.norm(c.pos[cand[:, 1]] - c.pos[cand[:, 0]], axis=1)
    rr = c.radii[cand[:, 0]] + c.radii[cand[:, 1]]
    assert np.min(np.abs(d - rr)) > 1e-12, "no pair sits on the contact boundary"
    want = np.sort(cand[d < rr], axis=1)
    want = want[np.lexsort((want[:, 1], want[:, 0]))]
    np.testing.assert_array_equal(ij, want)
    # sampled rows agree with the full scan
    rows = np.array([0, 7, 100, 599])
    sub = oracle.contacts_of_rows(c.pos, c.radii, rows)
    np.testing.assert_array_equal(sub, ij[np.isin(ij[:, 0], rows)])


@pytest.mark.parametrize("kind", ["cube", "ball", "sheet"])
def test_kdtree_contacts_equal_the_brute_force_scan(kind):
    c = {"cube": lambda: small_cells(900, seed=8),
         "ball": lambda: workloads.ball(n=1500, seed=9),
         "sheet": lambda: workloads.hex_sheet(nx=40, ny=30, seed=10)}[kind]()
    np.testing.assert_array_equal(oracle.contacts_kdtree(c.pos, c.radii), oracle.contacts(c.pos, c.radii))
    # pairs exactly at the contact distance stay out on both sides
    pos = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [2.25, 0.0, 0.0]])
    radii = np.array([0.5, 0.5, 0.9])
    np.testing.assert_array_equal(oracle.contacts_kdtree(pos, radii), oracle.contacts(pos, radii))
    assert oracle.contacts(pos, radii).tolist() == [[1, 2]]


def test_degenerate_coincident_centres():
    pos = np.array([[1.0, 1.0, 1.0], [1.0, 1.0, 1.0]])
    ij = oracle.contacts(pos, np.array([0.5, 0.5]))
    with pytest.raises(oracle.OracleError) as e:
        oracle.friction_blocks(ij, pos, [1.0], [1.0])
    assert e.value.code == oracle.ERR_DEGENERATE


# ---------------------------------------------------------------------------
# Gamma: the block Laplacian (Definition, Section 2) equals the App. B.2
# matrix-free product; symmetric positive definite with lambda_min >= gamma0
# (Lemma 2.4); the Laplacian part annihilates rigid translations exactly.
# ---------------------------------------------------------------------------
def test_matvec_equals_dense_block_laplacian():
    c = small_cells(150, seed=7)
    s = system_of(c)
    G = oracle.dense_laplacian(s.n, s.ij, s.blocks, s.gamma0)
    rng = np.random.default_rng(0)
    for _ in range(3):
        v = rng.standard_normal((s.n, 3))
        np.testing.assert_allclose(oracle.matvec(s.n, s.ij, s.blocks, s.gamma0, v).ravel(),
                                   G @ v.ravel(), rtol=1e-12, atol=1e-12)


def test_gamma_spd_lemma_2_4():
    c = small_cells(150, seed=8)
    s = system_of(c)
    G = oracle.dense_laplacian(s.n, s.ij, s.blocks, s.gamma0)
    assert np.array_equal(G, G.T)
    lam = np.linalg.eigvalsh(G)
    assert lam[0] > 0
    assert lam[0] >= s.gamma0 * (1 - 1e-9)
    # without the substrate term the Laplacian is only semidefinite
    L0 = oracle.dense_laplacian(s.n, s.ij, s.blocks, 0.0)
    assert np.linalg.eigvalsh(L0)[0] > -1e-10 * np.abs(L0).max()


def test_translation_annihilated_exactly():
    c = small_cells(300, seed=9)
    s = system_of(c)
    t = np.array([0.37, -1.25, 2.5])
    v = np.tile(t, (s.n, 1))
    x = oracle.matvec(s.n, s.ij, s.blocks, s.gamma0, v)
    np.testing.assert_array_equal(x, s.gamma0 * v)


# ---------------------------------------------------------------------------
# Maximum spanning forest: Prim against Kruskal (strict order w desc, id
# asc) and against exhaustive enumeration of all spanning forests.
# ---------------------------------------------------------------------------
def kruskal(n, ij, w):
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    order = sorted(range(len(w)), key=lambda e: (-w[e], e))
    out = []
    for e in order:
        a, b = find(int(ij[e][0])), find(int(ij[e][1]))
        if a != b:
            parent[a] = b
            out.append(e)
    return sorted(out)


def n_components(n, edges):
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            a = parent[a]
        return a
    comps = n
    for a, b in edges:
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[ra] = rb
            comps -= 1
    return comps


def test_prim_equals_kruskal_with_ties():
    rng = np.random.default_rng(1)
    for trial in range(40):
        n = int(rng.integers(1, 60))
        m = int(rng.integers(0, 3 * n + 1))
        pairs = set()
        for _ in range(m):
            a, b = rng.integers(0, max(n, 1), size=2)
            if a != b:
                pairs.add((min(a, b), max(a, b)))
        ij = np.array(sorted(pairs), dtype=np.int32).reshape(-1, 2)
        w = rng.integers(1, 4, size=ij.shape[0]).astype(np.float64)   # many ties
        f = oracle.prim_msf(n, ij, w)
        assert sorted(f.tree_edges.tolist()) == kruskal(n, ij, w)
        assert len(f.tree_edges) == n - n_components(n, [tuple(p) for p in ij])


def test_prim_maximum_by_exhaustive_enumeration():
    rng = np.random.default_rng(2)
    for trial in range(25):
        n = int(rng.integers(2, 8))
        all_pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
        keep = rng.random(len(all_pairs)) < 0.6
        pairs = [p for p, k in zip(all_pairs, keep) if k]
        if not pairs:
            continue
        ij = np.array(pairs, dtype=np.int32)
        w = rng.random(len(pairs)) + 0.1
        c = n_components(n, pairs)
        best, best_set = -1.0, None
        for sub in itertools.combinations(range(len(pairs)), n - c):
            es = [pairs[e] for e in sub]
            if n_components(n, es) != c:
                continue
            tot = float(np.sum(w[list(sub)]))
            if tot > best:
                best, best_set = tot, sorted(sub)
        f = oracle.prim_msf(n, ij, w)
        assert sorted(f.tree_edges.tolist()) == best_set
        # Prim's parent pointers describe the same forest
        pe = sorted(int(e) for e in f.parent_edge if e >= 0)
        assert pe == best_set
        pos_in_order = np.empty(n, dtype=np.int64)
        pos_in_order[f.order] = np.arange(n)
        for v in range(n):
            if f.parent[v] >= 0:
                assert pos_in_order[f.parent[v]] < pos_in_order[v], "parents inserted first"


# ---------------------------------------------------------------------------
# Tree factor and solve (Algorithm 2, Appendix B.1): exact inverse of the
# tree preconditioner P (dense LAPACK), zero fill (Theorem, Section 3.3),
# L D L^T = P.
# ---------------------------------------------------------------------------
def tree_dense(s, forest):
    te = np.sort(forest.tree_edges)
    return oracle.dense_laplacian(s.n, s.ij[te], s.blocks[te], s.gamma0)


def test_tree_solve_against_dense_lapack():
    for seed, n in ((21, 40), (22, 150), (23, 200)):
        c = small_cells(n, seed=seed)
        s = system_of(c)
        forest = oracle.prim_msf(s.n, s.ij, s.w)
        fac = oracle.tree_ldlt(forest, s.blocks, s.gamma0)
        P = tree_dense(s, forest)
        b = np.random.default_rng(seed).standard_normal((s.n, 3))
        x = oracle.tree_solve(fac, b)
        want = sla.solve(P, b.ravel(), assume_a="pos")
        np.testing.assert_allclose(x.ravel(), want, rtol=1e-11, atol=1e-11 * np.abs(want).max())
        np.testing.assert_allclose(P @ x.ravel(), b.ravel(), rtol=1e-10, atol=1e-10)


def test_tree_ldlt_reconstructs_P_with_zero_fill():
    c = small_cells(60, seed=31)
    s = system_of(c)
    forest = oracle.prim_msf(s.n, s.ij, s.w)
    fac = oracle.tree_ldlt(forest, s.blocks, s.gamma0)
    n = s.n
    elim = forest.order[::-1]          # elimination order: children first
    pos = np.empty(n, dtype=np.int64)
    pos[elim] = np.arange(n)
    Lm = np.eye(3 * n)
    Dm = np.zeros((3 * n, 3 * n))
    nnz = 0
    for v in range(n):
        k = pos[v]
        Dm[3 * k:3 * k + 3, 3 * k:3 * k + 3] = fac.D[v]
        if forest.parent[v] >= 0:
            p = pos[forest.parent[v]]
            assert p > k, "parent eliminated after child"
            Lm[3 * p:3 * p + 3, 3 * k:3 * k + 3] = fac.L[v]
            nnz += 1
    assert nnz == len(forest.tree_edges), "L has exactly one off-diagonal block per tree edge"
    perm = np.concatenate([[3 * v, 3 * v + 1, 3 * v + 2] for v in elim])
    P = tree_dense(s, forest)[np.ix_(perm, perm)]
    np.testing.assert_allclose(Lm @ Dm @ Lm.T, P, rtol=1e-11, atol=1e-11 * np.abs(P).max())
    for v in range(n):
        np.testing.assert_allclose(fac.D[v] @ fac.Dinv[v], np.eye(3), atol=1e-9)


# ---------------------------------------------------------------------------
# PCG (Section 1.1): against dense solves; the preconditioned spectrum lies
# in [1, kappa m (n-1)] (Theorems of Section 4, kappa from the end of
# Section 4); the Gamma-norm error obeys the CG bound with kappa(P^-1 Gamma).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precond", [oracle.PRECOND_TREE, oracle.PRECOND_JACOBI, oracle.PRECOND_NONE])
def test_pcg_against_dense_solve(precond):
    c = small_cells(180, seed=41)
    s = system_of(c)
    F = c.forces()
    G = oracle.dense_laplacian(s.n, s.ij, s.blocks, s.gamma0)
    want = sla.solve(G, F.ravel(), assume_a="pos")
    res, _ = oracle.solve_system(s, F, tol=1e-13, precond=precond)
    assert res.status == oracle.OK
    np.testing.assert_allclose(res.x.ravel(), want, rtol=1e-9, atol=1e-9 * np.abs(want).max())
    # recursive residual agrees with the true residual
    rt = np.linalg.norm(F.ravel() - G @ res.x.ravel()) / np.linalg.norm(F)
    assert rt < 1e-12


def test_preconditioned_spectrum_bounds():
    c = small_cells(120, seed=51)
    s = system_of(c)
    forest = oracle.prim_msf(s.n, s.ij, s.w)
    G = oracle.dense_laplacian(s.n, s.ij, s.blocks, s.gamma0)
    P = tree_dense(s, forest)
    lam = sla.eigh(G, P, eigvals_only=True)
    assert lam[0] >= 1 - 1e-10
    kappa = float(np.max(np.maximum(s.g_par, s.g_perp) / np.minimum(s.g_par, s.g_perp)))
    m = s.ij.shape[0]
    assert lam[-1] <= kappa * m * (s.n - 1)
    # any spanning subgraph, e.g. the MINIMUM spanning forest, also has
    # lambda_min >= 1 (Theorem, Section 4): take the tree of reversed weights
    f2 = oracle.prim_msf(s.n, s.ij, 1.0 / s.w)
    P2 = tree_dense(s, f2)
    assert sla.eigh(G, P2, eigvals_only=True)[0] >= 1 - 1e-10


def test_pcg_error_follows_cg_bound():
    c = small_cells(120, seed=61)
    s = system_of(c)
    F = c.forces()
    forest = oracle.prim_msf(s.n, s.ij, s.w)
    fac = oracle.tree_ldlt(forest, s.blocks, s.gamma0)
    G = oracle.dense_laplacian(s.n, s.ij, s.blocks, s.gamma0)
    P = tree_dense(s, forest)
    lam = sla.eigh(G, P, eigvals_only=True)
    kap = lam[-1] / lam[0]
    xs = sla.solve(G, F.ravel(), assume_a="pos")

    def enorm(x):
        e = x.ravel() - xs
        return math.sqrt(e @ G @ e)
    e0 = enorm(np.zeros_like(F))
    rho = (math.sqrt(kap) - 1) / (math.sqrt(kap) + 1)
    errs = []
    for k in (1, 2, 4, 8, 16):
        r = oracle.pcg(s.n, s.ij, s.blocks, s.gamma0, F, oracle.PRECOND_TREE, fac, fixed_iters=k)
        assert r.iters == k
        ek = enorm(r.x)
        errs.append(ek)
        assert ek <= 2 * rho ** k * e0 * (1 + 1e-8)
    assert all(b < a for a, b in zip(errs, errs[1:])), "Gamma-norm error decreases monotonically"


def test_tree_graph_converges_in_one_iteration():
    """If the collision graph is itself a tree, P = Gamma."""
    n = 30
    pos = np.zeros((n, 3))
    pos[:, 0] = 0.9 * np.arange(n)
    pos[:, 1] = 0.05 * np.sin(np.arange(n))
    radii = np.full(n, 0.5)
    cells = workloads.Cells("chain", pos, radii, 77, 0.1, 10.0, 1e-2)
    s = system_of(cells)
    assert s.ij.shape[0] == n - 1
    res, _ = oracle.solve_system(s, cells.forces(), tol=1e-12)
    assert res.iters == 1


def test_zero_rhs_and_isolated_cells():
    pos = np.array([[0.0, 0, 0], [5.0, 0, 0], [5.9, 0, 0], [20.0, 0, 0]])
    radii = np.full(4, 0.5)
    cells = workloads.Cells("iso", pos, radii, 5, 0.1, 10.0, 0.5)
    s = system_of(cells)
    assert s.ij.tolist() == [[1, 2]]
    res, _ = oracle.solve_system(s, np.zeros((4, 3)), tol=1e-10)
    assert res.iters == 0 and not res.x.any()
    F = cells.forces()
    res, fac = oracle.solve_system(s, F, tol=1e-13)
    G = oracle.dense_laplacian(4, s.ij, s.blocks, s.gamma0)
    np.testing.assert_allclose(res.x.ravel(), sla.solve(G, F.ravel()), rtol=1e-10)
    # isolated cells: x = F / gamma0
    np.testing.assert_allclose(res.x[0], F[0] / 0.5, rtol=1e-14)
    np.testing.assert_allclose(res.x[3], F[3] / 0.5, rtol=1e-14)


def test_pcg_reports_non_convergence():
    c = small_cells(150, seed=71)
    s = system_of(c)
    res, _ = oracle.solve_system(s, c.forces(), tol=1e-14, precond=oracle.PRECOND_NONE, maxit=3)
    assert res.status == oracle.ERR_NO_CONVERGENCE and res.iters == 3


def test_mst_beats_jacobi_and_identity_iterations():
    """Section 5 reports fewer iterations for the MST preconditioner than for
    block Jacobi or none; on the cube law the ordering must hold."""
    c = small_cells(1000, seed=1000, side=8.886)
    s = system_of(c)
    F = c.forces()
    its = {}
    for p in (oracle.PRECOND_TREE, oracle.PRECOND_JACOBI, oracle.PRECOND_NONE):
        r, _ = oracle.solve_system(s, F, tol=1e-8, precond=p)
        assert r.status == oracle.OK
        its[p] = r.iters
    assert its[oracle.PRECOND_TREE] < its[oracle.PRECOND_JACOBI] <= its[oracle.PRECOND_NONE]


def test_all_cores_baseline_solves_the_same_system():
    """The all-cores CPU baseline (row-wise product and vector operations on
    OpenMP threads, the oracle's sequential tree solve) is the same PCG: on a
    1000-cell cube it takes the oracle's iterations and reaches its solution
    to rounding, and after a fixed number of steps it reports them."""
    c = workloads.cube(n=1000, side=8.886, seed=1000)
    o = oracle.build_system(c.pos, c.radii, c.gammas_np, c.gamma0)
    F = c.forces()
    f = oracle.prim_msf(c.n, o.ij, o.w)
    fac = oracle.tree_ldlt(f, o.blocks, c.gamma0)
    r1 = oracle.pcg(c.n, o.ij, o.blocks, c.gamma0, F, oracle.PRECOND_TREE, fac, tol=1e-10)
    r2 = oracle.pcg_parallel(c.n, o.ij, o.blocks, c.gamma0, F, fac, tol=1e-10)
    assert abs(r1.iters - r2.iters) <= 1
    assert np.linalg.norm(r1.x - r2.x) <= 1e-9 * np.linalg.norm(r1.x)
    r3 = oracle.pcg_parallel(c.n, o.ij, o.blocks, c.gamma0, F, fac, tol=1e-300, maxit=7)
    assert r3.iters == 7 and r3.status == oracle.ERR_NO_CONVERGENCE
    assert oracle.parallel_threads() >= 1
