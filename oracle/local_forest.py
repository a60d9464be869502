"""CPU oracle of the partitioned ("local") spanning-forest preconditioner
(FP64).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``, the
smoke check and the benchmark's CPU leg may import it; it shares no code with
the CUDA library.

What it computes (arXiv 2410.04512, Section 6, the proposed hierarchical
preconditioner): the cells are split into spatial leaves of a few hundred
cells; each leaf keeps the maximum spanning forest of its own interaction
subgraph (the contacts whose two cells lie in the leaf); contacts between
leaves are dropped from the preconditioner.  P_loc = gamma0 I + the block
Laplacian of the union of the leaves' forests, block diagonal over the
leaves, so its leaves are solved independently.

Readings where the paper is silent (also listed in the design notes):
  * Leaves.  The paper names octrees, Z-order or Hilbert grids with 300-1000
    cells per leaf.  Here: the leaves of a uniform grid of side h (the
    octree's leaves at one depth); cell i lies in the leaf
    (floor(x_i/h), floor(y_i/h), floor(z_i/h)), labelled by the low 10 bits
    of each coordinate, label = kx | ky << 10 | kz << 20 (kx = floor(x/h) mod
    1024).  Labels repeat only for leaves 1024 h apart along an axis, which
    no contact joins; such leaves share a label and are then treated as one,
    which leaves the preconditioner block diagonal.  h is the caller's.
  * The forest of a leaf is the maximum spanning forest of its subgraph
    under the same strict order as the global forest (weight descending,
    then edge index ascending), so the union is unique.

Pins (tests/test_oracle_local_forest.py): the labels against an integer
re-derivation from exact rational positions, the union against Kruskal run
leaf by leaf on networkx graphs, the edge count n - (components of the
leaves' subgraphs), the absence of cross-leaf edges, P_loc block diagonal
over the leaves and lambda_min(Gamma, P_loc) >= 1 (a subgraph's Laplacian,
Section 4) by a dense generalized eigensolve.
"""
from __future__ import annotations

import numpy as np

from . import Forest, _f64, _i32, prim_msf

LEAF_BITS = 10
LEAF_MASK = (1 << LEAF_BITS) - 1


def grid_leaves(pos, h: float) -> np.ndarray:
    """Leaf label of every cell: the uniform grid of side h, coordinates
    floor(x / h) (FP64 division, correctly rounded), low 10 bits of each
    packed x | y << 10 | z << 20.  (n,) int32."""
    pos = _f64(pos)
    if not (h > 0.0) or not np.isfinite(h):
        raise ValueError("grid_leaves: h must be a positive finite number")
    k = np.floor(pos / h).astype(np.int64)
    lab = (k[:, 0] & LEAF_MASK) | ((k[:, 1] & LEAF_MASK) << LEAF_BITS) | ((k[:, 2] & LEAF_MASK) << (2 * LEAF_BITS))
    return lab.astype(np.int32)


def local_edges(ij, leaf) -> np.ndarray:
    """Indices (ascending) of the contacts whose two cells share a leaf."""
    ij, leaf = _i32(ij), np.asarray(leaf)
    if ij.shape[0] == 0:
        return np.zeros(0, dtype=np.int64)
    return np.nonzero(leaf[ij[:, 0]] == leaf[ij[:, 1]])[0]


def local_msf(n: int, ij, w, leaf) -> Forest:
    """The union of the leaves' maximum spanning forests: Prim's forest of
    the graph that keeps only the contacts inside a leaf (that graph is the
    disjoint union of the leaves' subgraphs, so its maximum spanning forest
    is the union of theirs).  Edge ids are those of the full contact list."""
    ij, w = _i32(ij), _f64(w)
    keep = local_edges(ij, leaf)
    f = prim_msf(n, ij[keep], w[keep])
    pe = np.full(f.parent_edge.shape, -1, dtype=np.int32)
    has = f.parent_edge >= 0
    pe[has] = keep[f.parent_edge[has]]
    return Forest(tree_edges=keep[f.tree_edges].astype(np.int32), order=f.order, parent=f.parent,
                  parent_edge=pe)
