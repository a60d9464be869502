"""Pins of the oracle's augmented spanning-tree preconditioner and flexible CG
(Sections 3.1, 3.3, 4 and 5) to things other than the oracle itself:
networkx's depth-first search, breadth-first connectivity, brute force over
all edges, dense eigenvalues (Loewner order, the Section 4 bound) and
scipy's preconditioned conjugate gradients."""

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import oracle
import oracle.augmented as aug
import workloads

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def cells_cube(n=150, seed=21, gamma0=1e-2):
    return workloads.cube(n=n, side=(n / 1.4253) ** (1.0 / 3.0), seed=seed, gamma0=gamma0)


def cells_chain(n=60):
    pos = np.zeros((n, 3))
    pos[:, 0] = 0.9 * np.arange(n)
    pos[:, 1] = 0.05 * np.sin(0.7 * np.arange(n))
    return workloads.Cells("chain", pos, np.full(n, 0.5), 9, 0.1, 10.0, 1e-2)


def cells_forest(seed=5):
    rng = np.random.default_rng(seed)
    pos = np.concatenate([rng.uniform(0, 40, size=(40, 3)), rng.uniform(0, 3.5, size=(60, 3)) + 60.0])
    return workloads.Cells("forest", pos, np.full(pos.shape[0], 0.5), 8, 0.1, 10.0, 1e-2)


def system(c):
    s = oracle.build_system(c.pos, c.radii, c.gammas_np, c.gamma0)
    f = oracle.prim_msf(s.n, s.ij, s.w)
    return s, f


CASES = {"cube": cells_cube, "chain": cells_chain, "forest": cells_forest}


@pytest.mark.parametrize("name", sorted(CASES))
def test_preorder_is_networkx_dfs_with_sorted_children(name):
    nx = pytest.importorskip("networkx")
    s, f = system(CASES[name]())
    pre, parent = aug.forest_preorder(s.n, s.ij, f.tree_edges)
    G = nx.Graph()
    G.add_nodes_from(range(s.n))
    te = f.tree_edges
    # insert each cell's tree neighbours in ascending order: networkx then
    # walks children in that order
    nb = [[] for _ in range(s.n)]
    for e in te:
        a, b = (int(x) for x in s.ij[e])
        nb[a].append(b)
        nb[b].append(a)
    for v in range(s.n):
        for u in sorted(nb[v]):
            G.add_edge(v, u)
    want = []
    seen = set()
    for root in range(s.n):
        if root in seen:
            continue
        comp = list(nx.dfs_preorder_nodes(G, source=root))
        seen.update(comp)
        want.extend(comp)
    assert np.array_equal(np.argsort(pre), np.array(want))
    # parent = the tree neighbour visited before v
    for v in range(s.n):
        if parent[v] >= 0:
            assert parent[v] in nb[v] and pre[parent[v]] < pre[v]
        else:
            assert all(pre[u] > pre[v] for u in nb[v]) and v == min(nx.node_connected_component(G, v))


def _pieces_valid(s, f, piece, t):
    n = s.n
    smax = -(-n // t)
    pre, parent = aug.forest_preorder(s.n, s.ij, f.tree_edges)
    npieces = int(piece.max()) + 1
    assert npieces >= min(t, n)
    # every piece lies in one preorder block, has at most s cells, and is
    # connected through tree edges inside it (breadth-first search)
    adj = [[] for _ in range(n)]
    for e in f.tree_edges:
        a, b = (int(x) for x in s.ij[e])
        adj[a].append(b)
        adj[b].append(a)
    for k in range(npieces):
        cells = np.nonzero(piece == k)[0]
        assert 1 <= cells.shape[0] <= smax
        assert np.unique(pre[cells] // smax).shape[0] == 1
        seen = {int(cells[0])}
        todo = [int(cells[0])]
        while todo:
            v = todo.pop()
            for u in adj[v]:
                if piece[u] == k and u not in seen:
                    seen.add(u)
                    todo.append(u)
        assert len(seen) == cells.shape[0]
    # maximal: a tree edge inside one block joins the same piece
    for e in f.tree_edges:
        a, b = (int(x) for x in s.ij[e])
        if pre[a] // smax == pre[b] // smax:
            assert piece[a] == piece[b]
    # numbered in preorder of their top cell
    tops = [int(np.min(pre[piece == k])) for k in range(npieces)]
    assert tops == sorted(tops)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("t", [1, 2, 3, 7, 1000])
def test_partition_is_valid(name, t):
    s, f = system(CASES[name]())
    piece = aug.tree_partition(s.n, s.ij, f.tree_edges, t)
    _pieces_valid(s, f, piece, t)
    if t == 1:
        # one piece per tree of the forest
        assert int(piece.max()) + 1 == s.n - f.tree_edges.shape[0]


def test_default_piece_count():
    assert aug.default_pieces(1_000_000) == 32
    assert aug.default_pieces(1) == 1 and aug.default_pieces(0) == 1


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("t", [2, 5, 1000])
def test_added_edges_by_brute_force(name, t):
    s, f = system(CASES[name]())
    piece = aug.tree_partition(s.n, s.ij, f.tree_edges, t)
    got = aug.augment(s.n, s.ij, s.w, f.tree_edges, piece)
    best = {}
    for e in range(s.ij.shape[0]):
        a, b = int(piece[s.ij[e, 0]]), int(piece[s.ij[e, 1]])
        if a == b:
            continue
        key = (min(a, b), max(a, b))
        if key not in best or s.w[e] > s.w[best[key]]:   # strictly heavier; ties keep the smaller index
            best[key] = e
    want = sorted(set(int(e) for e in f.tree_edges) | set(best.values()))
    assert got.tolist() == want
    if t >= s.n:
        # every cell its own piece: every edge is the only one of its pair
        assert got.tolist() == list(range(s.ij.shape[0]))


def _dense_P(s, edges):
    return oracle.dense_laplacian(s.n, s.ij[edges], s.blocks[edges], s.gamma0)


@pytest.mark.parametrize("t", [2, 4, 8])
def test_loewner_order_and_section_4_bound(t):
    """P <= P' <= Gamma (P' adds edge Laplacians to P, Gamma adds the rest),
    so 1 <= lambda(Gamma, P') <= lambda_max(Gamma, P); and the Section 4
    theorem: lambda_max(L_G, L_T') <= 2 kappa d^3 n^2 / t^2, which with the
    common gamma0 I gives lambda_max(Gamma, P') <= max(1, that)."""
    c = cells_cube(120, seed=31)
    s, f = system(c)
    A = aug.build(s.n, s.ij, s.w, f.tree_edges, t)
    assert A.added > 0
    G = oracle.dense_laplacian(s.n, s.ij, s.blocks, s.gamma0)
    P = _dense_P(s, np.sort(f.tree_edges))
    Pa = _dense_P(s, A.edges)
    tol = 1e-10 * np.abs(G).max()
    assert np.linalg.eigvalsh(Pa - P).min() >= -tol
    assert np.linalg.eigvalsh(G - Pa).min() >= -tol
    lam_a = sla.eigh(G, Pa, eigvals_only=True)
    lam_p = sla.eigh(G, P, eigvals_only=True)
    assert lam_a[0] >= 1 - 1e-9
    assert lam_a[-1] <= lam_p[-1] * (1 + 1e-9)
    kappa = float(np.max(np.maximum(s.g_par, s.g_perp) / np.minimum(s.g_par, s.g_perp)))
    deg = np.bincount(s.ij.ravel(), minlength=s.n).max()
    bound = 2 * kappa * deg ** 3 * s.n ** 2 / t ** 2
    assert lam_a[-1] <= max(1.0, bound)
    # more pieces, more support: with every cell its own piece P' = Gamma
    Aall = aug.build(s.n, s.ij, s.w, f.tree_edges, s.n)
    assert np.allclose(_dense_P(s, Aall.edges), G, rtol=0, atol=tol)


def test_flexible_cg_with_exact_inner_solves_is_pcg_with_P_prime():
    """With z = P'^-1 r exactly, flexible CG is preconditioned CG with P'
    (its beta equals the Fletcher-Reeves one when the preconditioner is
    fixed): iterates at k = 1, 3, 10 against scipy's cg with M = P'^-1."""
    c = cells_cube(150, seed=41)
    s, f = system(c)
    A = aug.build(s.n, s.ij, s.w, f.tree_edges, 4)
    fac = oracle.tree_ldlt(f, s.blocks, s.gamma0)
    F = c.forces()
    G = oracle.dense_laplacian(s.n, s.ij, s.blocks, s.gamma0)
    Pa = _dense_P(s, A.edges)
    cho = sla.cho_factor(Pa)
    exact = lambda r: sla.cho_solve(cho, r.ravel()).reshape(-1, 3)
    Minv = spla.LinearOperator(G.shape, matvec=lambda v: sla.cho_solve(cho, v))
    for k in (1, 3, 10):
        res = aug.fcg(s.n, s.ij, s.blocks, s.gamma0, F, A, fac, fixed_iters=k, inner_solve=exact)
        assert res.iters == k
        want, _ = spla.cg(G, F.ravel(), x0=np.zeros(3 * s.n), rtol=1e-300, atol=0.0, maxiter=k, M=Minv)
        np.testing.assert_allclose(res.x.ravel(), want, rtol=0, atol=1e-9 * np.abs(want).max())


@pytest.mark.parametrize("inner_tol", [0.1, 1e-3])
def test_nested_solve_reaches_the_dense_solution(inner_tol):
    c = cells_cube(200, seed=43)
    s, f = system(c)
    A = aug.build(s.n, s.ij, s.w, f.tree_edges)
    fac = oracle.tree_ldlt(f, s.blocks, s.gamma0)
    F = c.forces()
    G = oracle.dense_laplacian(s.n, s.ij, s.blocks, s.gamma0)
    want = np.linalg.solve(G, F.ravel())
    res = aug.fcg(s.n, s.ij, s.blocks, s.gamma0, F, A, fac, tol=1e-10, inner_tol=inner_tol)
    assert res.status == oracle.OK and res.relres <= 1e-10
    assert res.inner_iters >= res.iters
    true = np.linalg.norm(F.ravel() - G @ res.x.ravel()) / np.linalg.norm(F)
    assert true <= 1e-9
    kappa = np.linalg.cond(G)
    np.testing.assert_allclose(res.x.ravel(), want, rtol=0, atol=10 * kappa * 1e-10 * np.abs(want).max())


def test_fcg_edge_cases():
    c = cells_forest()
    s, f = system(c)
    A = aug.build(s.n, s.ij, s.w, f.tree_edges, 3)
    fac = oracle.tree_ldlt(f, s.blocks, s.gamma0)
    z = aug.fcg(s.n, s.ij, s.blocks, s.gamma0, np.zeros((s.n, 3)), A, fac)
    assert z.iters == 0 and not z.x.any()
    # t = 1: T' = T, so the inner PCG converges in one iteration (P' = P)
    A1 = aug.build(s.n, s.ij, s.w, f.tree_edges, 1)
    assert A1.added == 0
    F = c.forces()
    r = aug.fcg(s.n, s.ij, s.blocks, s.gamma0, F, A1, fac, tol=1e-10, inner_tol=1e-12)
    assert r.inner_iters == r.iters
    with pytest.raises(oracle.OracleError):
        aug.tree_partition(s.n, s.ij, f.tree_edges, 0)
