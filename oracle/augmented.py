"""CPU oracle of the augmented spanning-tree preconditioner and the nested
(flexible) conjugate gradients that apply it (FP64).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``, the
smoke check and the benchmark's CPU leg may import it; it shares no code with
the CUDA library.

What it computes (arXiv 2410.04512):
  * Section 3.1, Vaidya's second preconditioner: the spanning forest is cut
    into disjoint subtrees ("pieces") of at most ceil(n/t) cells, and for
    every pair of pieces that the collision graph connects, the heaviest
    edge between them is added back.  P' = gamma0 I + block Laplacian of the
    augmented forest T'.  t defaults to round(n^(1/4)) (the optimum the
    section quotes).
  * Section 3.3 (last paragraphs): P' has fill, so systems in P' are solved
    by an inner conjugate-gradient run preconditioned by the plain forest
    factor, to a relative residual delta (Section 5: delta = 0.1).
  * Section 5: the outer iteration is flexible CG, because an inner
    iteration stopped at a tolerance is not a fixed linear operator.  The
    variant here keeps one previous direction (Notay's FCG with truncation
    parameter 1): z_k = B_k(r_k), p_k = z_k - (z_k^T q_{k-1} / p_{k-1}^T q_{k-1}) p_{k-1},
    q_k = Gamma p_k, alpha_k = p_k^T r_k / p_k^T q_k.

Readings where the paper is silent (also listed in the design notes):
  * Partition rule.  The paper names the TreePartition procedure of Chen and
    Toledo without stating it.  Here: every tree is rooted at its smallest
    cell id; a depth-first preorder visits children in ascending id order and
    the trees one after another in ascending order of their roots, numbering
    all n cells 0..n-1; with s = ceil(n/t), a piece is a maximal set of cells
    that the tree connects and whose preorder numbers fall in the same block
    [k s, (k+1) s).  Pieces are therefore connected subtrees of at most s
    cells, at least t of them; they are numbered in preorder of their top
    cell.
  * Heaviest edge: the same strict order as the spanning forest (weight
    descending, then edge index ascending), so each pair's choice is unique.
    The added edge may already be a tree edge; T' is the union, as a sorted
    list of edge indices.

Pins (tests/test_oracle_augmented.py): the preorder against networkx's
depth-first search, piece connectivity and maximality by breadth-first
search, the added edges by brute force over all edges, the Loewner order
P <= P' <= Gamma and the Section 4 bound on lambda_max(Gamma, P') by dense
eigenvalues, and the flexible iteration with exact inner solves against
scipy's conjugate gradients preconditioned by P'^-1.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import (ERR_NO_CONVERGENCE, ERR_NOT_SPD, OK, PRECOND_TREE, OracleError, TreeFactor, _f64, _i32, matvec,
               pcg)


def default_pieces(n: int) -> int:
    """t = round(n^(1/4)), at least 1 (Section 3.1)."""
    return max(1, int(round(n ** 0.25)))


def forest_preorder(n: int, ij, tree_edges) -> tuple[np.ndarray, np.ndarray]:
    """Depth-first preorder of the spanning forest under the reading above:
    returns (pre, parent), pre[v] the preorder number of cell v, parent[v]
    its parent (-1 at each tree's smallest cell)."""
    ij = _i32(ij)
    te = np.asarray(tree_edges, dtype=np.int64)
    adj = [[] for _ in range(n)]
    for e in te:
        a, b = int(ij[e, 0]), int(ij[e, 1])
        adj[a].append(b)
        adj[b].append(a)
    for lst in adj:
        lst.sort()
    pre = np.full(n, -1, dtype=np.int64)
    parent = np.full(n, -1, dtype=np.int64)
    k = 0
    for root in range(n):          # the first unvisited cell is its tree's smallest
        if pre[root] >= 0:
            continue
        stack = [root]
        while stack:
            v = stack.pop()
            pre[v] = k
            k += 1
            kids = [u for u in adj[v] if u != parent[v]]
            for u in kids:
                parent[u] = v
            stack.extend(reversed(kids))   # smallest child on top
    return pre, parent


def tree_partition(n: int, ij, tree_edges, t: int) -> np.ndarray:
    """Piece label of every cell (Section 3.1, reading above); int32."""
    if t < 1:
        raise OracleError(1, "tree_partition: t must be >= 1")
    if n == 0:
        return np.zeros(0, dtype=np.int32)
    s = -(-n // t)
    pre, parent = forest_preorder(n, ij, tree_edges)
    order = np.argsort(pre)                      # cells in preorder
    top = np.empty(n, dtype=np.int64)
    label = np.empty(n, dtype=np.int64)
    npieces = 0
    for v in order:                              # a parent comes before its children
        p = parent[v]
        if p < 0 or pre[p] // s != pre[v] // s:
            top[v] = v
            label[v] = npieces
            npieces += 1
        else:
            top[v] = top[p]
            label[v] = label[p]
    return label.astype(np.int32)


def augment(n: int, ij, w, tree_edges, piece) -> np.ndarray:
    """Edge indices of T' = tree edges plus, for every pair of pieces joined
    by some edge, the heaviest such edge (w descending, index ascending);
    sorted ascending, int32."""
    ij, w = _i32(ij), _f64(w)
    piece = np.asarray(piece, dtype=np.int64)
    m = ij.shape[0]
    pa, pb = piece[ij[:, 0]], piece[ij[:, 1]]
    inter = np.nonzero(pa != pb)[0]
    lo, hi = np.minimum(pa[inter], pb[inter]), np.maximum(pa[inter], pb[inter])
    # group by (lo, hi); inside a group the first in (w desc, index asc)
    srt = np.lexsort((inter, -w[inter], hi, lo))
    lo_s, hi_s = lo[srt], hi[srt]
    first = np.ones(srt.shape[0], dtype=bool)
    first[1:] = (lo_s[1:] != lo_s[:-1]) | (hi_s[1:] != hi_s[:-1])
    chosen = inter[srt[first]]
    keep = np.zeros(m, dtype=bool)
    keep[np.asarray(tree_edges, dtype=np.int64)] = True
    keep[chosen] = True
    return np.nonzero(keep)[0].astype(np.int32)


@dataclass
class Augmented:
    t: int
    piece: np.ndarray      # (n,) piece label
    npieces: int
    edges: np.ndarray      # edge indices of T', ascending
    added: int             # edges of T' that are not tree edges


def build(n: int, ij, w, tree_edges, t: int = 0) -> Augmented:
    t = t if t > 0 else default_pieces(n)
    piece = tree_partition(n, ij, tree_edges, t)
    edges = augment(n, ij, w, tree_edges, piece)
    added = int(edges.shape[0] - np.asarray(tree_edges).shape[0])
    return Augmented(t, piece, int(piece.max()) + 1 if n else 0, edges, added)


@dataclass
class FcgResult:
    x: np.ndarray
    iters: int              # outer (flexible) iterations
    inner_iters: int        # inner PCG iterations, all outer steps together
    relres: float           # recursive |r|/|F|
    status: int


def fcg(n: int, ij, blocks, gamma0: float, F, aug: Augmented, factor: TreeFactor, tol: float = 1e-8,
        inner_tol: float = 0.1, inner_maxit: int = 1000, maxit: int = 100000, fixed_iters: int = 0,
        inner_fixed: int = 0, x0=None, inner_solve=None) -> FcgResult:
    """Flexible CG on Gamma x = F with z = P'^-1 r applied by an inner PCG on
    P' (the forest factor as its preconditioner, from z = 0, to relative
    residual inner_tol or inner_maxit iterations; inner_fixed > 0 runs
    exactly that many).  fixed_iters > 0 runs exactly that many outer
    iterations.  inner_solve(r) -> z replaces the inner PCG (tests)."""
    ij, blocks, F = _i32(ij), _f64(blocks), _f64(F)
    aij, ablk = ij[aug.edges], blocks[aug.edges]
    x = np.zeros((n, 3)) if x0 is None else _f64(x0).copy()
    inner_total = 0

    def B(r):
        nonlocal inner_total
        if inner_solve is not None:
            return inner_solve(r)
        res = pcg(n, aij, ablk, gamma0, r, PRECOND_TREE, factor, tol=inner_tol,
                  maxit=inner_maxit if not inner_fixed else inner_fixed, fixed_iters=inner_fixed)
        inner_total += res.iters
        return res.x

    def dot(a, b):
        return float(np.dot(a.ravel(), b.ravel()))

    FF = dot(F, F)
    if FF == 0.0:
        return FcgResult(np.zeros((n, 3)), 0, 0, 0.0, OK)
    r = F - matvec(n, ij, blocks, gamma0, x) if x0 is not None else F.copy()
    rr = dot(r, r)
    stop2 = tol * tol * FF
    it = 0
    status = OK
    p = q = None
    pq = 0.0
    while fixed_iters > 0 or rr > stop2:
        if fixed_iters > 0 and it >= fixed_iters:
            break
        if fixed_iters == 0 and it >= maxit:
            status = ERR_NO_CONVERGENCE
            break
        z = B(r)
        if p is None:
            p = z.copy()
        else:
            beta = -dot(z, q) / pq
            p = z + beta * p
        q = matvec(n, ij, blocks, gamma0, p)
        pq = dot(p, q)
        if not pq > 0.0:
            status = ERR_NOT_SPD
            break
        alpha = dot(p, r) / pq
        x = x + alpha * p
        r = r - alpha * q
        rr = dot(r, r)
        it += 1
    return FcgResult(x, it, inner_total, float(np.sqrt(rr / FF)), status)
