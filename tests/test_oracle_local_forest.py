"""Pins of the oracle's partitioned spanning-forest preconditioner
(Section 6): the leaves of a uniform spatial grid, the union of the
leaves' maximum spanning forests, and the preconditioner it gives."""
from fractions import Fraction

import networkx as nx
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import oracle.local_forest as lf
import workloads


def test_leaf_labels_exact():
    """floor(x / h) re-derived in exact rational arithmetic from the FP64
    values (the FP64 quotient is correctly rounded, so it can only differ
    from the exact one when the exact quotient is within half an ulp of an
    integer; the positions here are chosen away from that), and the
    packing of the low 10 bits."""
    rng = np.random.default_rng(3)
    pos = rng.uniform(-3000.0, 3000.0, size=(500, 3))
    h = 2.75
    got = lf.grid_leaves(pos, h)
    for i in range(pos.shape[0]):
        k = []
        for c in range(3):
            q = Fraction(pos[i, c]) / Fraction(h)
            fl = q.numerator // q.denominator
            assert abs(float(q - fl) - 0.5) < 0.5 - 1e-9      # not at a leaf boundary
            k.append(fl % 1024)
        assert got[i] == k[0] | (k[1] << 10) | (k[2] << 20)
    # a leaf boundary: x = h exactly is in leaf 1, just below is in leaf 0
    lab = lf.grid_leaves(np.array([[2.75, 0, 0], [np.nextafter(2.75, 0), 0, 0], [-1e-300, 0, 0]]), h)
    assert list(lab) == [1, 0, 1023]
    with pytest.raises(ValueError):
        lf.grid_leaves(pos, 0.0)


def _system(n=1500, seed=91, gamma0=1e-2):
    c = workloads.cube(n=n, side=(n / 1.4253) ** (1.0 / 3.0), seed=seed, gamma0=gamma0)
    return c, oracle.build_system(c.pos, c.radii, c.gammas_np, c.gamma0)


def _kruskal_per_leaf(n, ij, w, leaf):
    """Maximum spanning forests leaf by leaf, by networkx's Kruskal on the
    leaf's own subgraph; the strict order (weight descending, then index
    ascending) enters as distinct integer keys."""
    order = np.lexsort((np.arange(ij.shape[0]), -np.asarray(w)))
    key = np.empty(ij.shape[0], dtype=np.int64)
    key[order] = ij.shape[0] - np.arange(ij.shape[0])     # larger key = earlier in the order
    out = []
    for L in np.unique(leaf):
        cells = np.nonzero(leaf == L)[0]
        G = nx.Graph()
        G.add_nodes_from(cells.tolist())
        for e in range(ij.shape[0]):
            a, b = ij[e]
            if leaf[a] == L and leaf[b] == L:
                G.add_edge(int(a), int(b), key=int(key[e]), e=e)
        T = nx.maximum_spanning_tree(G, weight="key", algorithm="kruskal")
        out += [d["e"] for _, _, d in T.edges(data=True)]
    return np.sort(np.array(out, dtype=np.int64))


@pytest.mark.parametrize("h", [2.0, 3.5, 1e6])
def test_union_of_leaf_forests(h):
    c, s = _system()
    leaf = lf.grid_leaves(c.pos, h)
    f = lf.local_msf(s.n, s.ij, s.w, leaf)
    te = np.sort(f.tree_edges)
    # no edge crosses leaves
    assert np.all(leaf[s.ij[te, 0]] == leaf[s.ij[te, 1]])
    # Kruskal leaf by leaf gives the same edges
    np.testing.assert_array_equal(te, _kruskal_per_leaf(s.n, s.ij, s.w, leaf))
    # n - (components of the leaves' subgraphs) edges
    keep = lf.local_edges(s.ij, leaf)
    G = nx.Graph()
    G.add_nodes_from(range(s.n))
    G.add_edges_from(s.ij[keep].tolist())
    assert te.shape[0] == s.n - nx.number_connected_components(G)
    if h == 1e6:
        # one leaf: the global forest
        np.testing.assert_array_equal(te, np.sort(oracle.prim_msf(s.n, s.ij, s.w).tree_edges))


def test_preconditioner_block_diagonal_and_bounded_below():
    """P_loc = gamma0 I + L(forest) has no block between leaves, and
    lambda_min(Gamma, P_loc) >= 1 (the forest is a subgraph, Section 4):
    checked by a dense generalized eigensolve.  The tree solve with its
    factor equals a dense solve with P_loc."""
    c, s = _system(n=400, seed=93)
    leaf = lf.grid_leaves(c.pos, 2.5)
    assert np.unique(leaf).shape[0] >= 4
    f = lf.local_msf(s.n, s.ij, s.w, leaf)
    te = np.sort(f.tree_edges)
    P = oracle.dense_laplacian(s.n, s.ij[te], s.blocks[te], s.gamma0)
    cross = leaf[:, None] != leaf[None, :]
    assert not np.any(P.reshape(s.n, 3, s.n, 3).transpose(0, 2, 1, 3)[cross])
    G = oracle.dense_laplacian(s.n, s.ij, s.blocks, s.gamma0)
    lam = sla.eigh(G, P, eigvals_only=True)
    assert lam[0] >= 1 - 1e-9
    fac = oracle.tree_ldlt(f, s.blocks, s.gamma0)
    b = np.random.default_rng(4).standard_normal((s.n, 3))
    np.testing.assert_allclose(oracle.tree_solve(fac, b).ravel(), np.linalg.solve(P, b.ravel()),
                               rtol=0, atol=1e-9 * np.abs(np.linalg.solve(P, b.ravel())).max())
    # PCG with P_loc reaches the solution
    F = c.forces()
    r = oracle.pcg(s.n, s.ij, s.blocks, s.gamma0, F, oracle.PRECOND_TREE, fac, tol=1e-10)
    assert r.status == oracle.OK
    x = np.linalg.solve(G, F.ravel())
    assert np.linalg.norm(r.x.ravel() - x) <= 1e-7 * np.linalg.norm(x)


def test_edge_cases():
    c, s = _system(n=200, seed=95)
    # every cell its own leaf: no edges, the preconditioner is gamma0 I
    leaf = np.arange(s.n, dtype=np.int32)
    f = lf.local_msf(s.n, s.ij, s.w, leaf)
    assert f.tree_edges.shape[0] == 0
    fac = oracle.tree_ldlt(f, s.blocks, s.gamma0)
    b = np.random.default_rng(6).standard_normal((s.n, 3))
    np.testing.assert_allclose(oracle.tree_solve(fac, b), b / s.gamma0, rtol=1e-15)
    # no contacts at all
    f0 = lf.local_msf(5, np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(5, np.int32))
    assert f0.tree_edges.shape[0] == 0
