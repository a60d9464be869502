"""Shared helpers of the GPU parity tests: run the CUDA path through the
C ABI (via the thin binding) and the oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np
import torch

import oracle
import paper_2410_04512_gb300 as sgp
import workloads


def dev_tensor(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def small_cube(n=1000, seed=1000, side=None, gamma0=1e-2, lo=0.1, hi=10.0):
    if side is None:
        side = 8.886 * (n / 1000.0) ** (1.0 / 3.0)
    return workloads.cube(n=n, side=side, seed=seed, gamma0=gamma0, gamma_lo=lo, gamma_hi=hi)


class GpuSystem:
    """Graph, friction matrix (and optionally tree and factor) on the GPU."""

    def __init__(self, ctx: sgp.Context, cells: workloads.Cells, precision=sgp.PREC_F64,
                 tree=True):
        self.ctx, self.cells = ctx, cells
        self.pos = dev_tensor(cells.pos)
        self.radii = dev_tensor(cells.radii)
        self.graph = ctx.collision_graph(self.pos, self.radii)
        self.ij = self.graph.edges()
        self.gp, self.gq = cells.gammas_torch(self.ij, self.pos, self.radii)
        self.M = ctx.friction_assemble(self.graph, self.pos, self.gp.contiguous(), self.gq.contiguous(),
                                       cells.gamma0, precision)
        self.T = self.Fac = None
        if tree:
            self.T = ctx.max_spanning_tree(self.M)
            self.Fac = ctx.tree_factor(self.M, self.T)

    @property
    def n(self):
        return self.cells.n


def oracle_system(cells: workloads.Cells, ij=None):
    return oracle.build_system(cells.pos, cells.radii, cells.gammas_np, cells.gamma0, ij=ij)


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
