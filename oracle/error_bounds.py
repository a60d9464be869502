"""CPU oracle of PCG stopped on a Gauss-Radau upper bound of the Gamma-norm
error (FP64).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``, the
smoke check and the benchmark's CPU leg may import it; it shares no code with
the CUDA library.

The paper monitors CG with Gauss-Radau error estimators (Section 5, citing
Meurant and Tichy) and proves lambda_min(Gamma, P) >= 1 for the spanning-
forest preconditioner (Section 4).  That bound is exactly the prescribed
lower eigenvalue estimate mu that a Gauss-Radau upper bound needs, so the
solver can stop on a guaranteed (in exact arithmetic) bound of the error
instead of on the residual.

With PCG's step lengths alpha_j and rho_j = r_j^T z_j (z = H r), the error of
iterate k satisfies (Hestenes-Stiefel; the Krylov relations of CG)
    |x - x_k|_Gamma^2 = sum_{j >= k} alpha_j rho_j,
    |x_k - x_0|_Gamma^2 = sum_{j < k} alpha_j rho_j,
and, for any 0 < mu <= lambda_min(H Gamma), the Gauss-Radau quadrature rule
with a node fixed at mu gives the upper bound (Meurant and Tichy's form of it)
    |x - x_k|_Gamma^2 <= phi_k rho_k,
    phi_0 = 1/mu,   phi_{k+1} = (phi_k - alpha_k) / (mu (phi_k - alpha_k) + beta_{k+1}),
with beta_{k+1} = rho_{k+1}/rho_k.  The delayed lower bound is the partial
sum sum_{j=k}^{k+d-1} alpha_j rho_j.

Stopping rule (error mode): after z_{k+1} and rho_{k+1}, stop when
    phi_{k+1} rho_{k+1} <= tol^2 sum_{j <= k} alpha_j rho_j,
i.e. the bound on |x - x_{k+1}|_Gamma relative to |x_{k+1} - x_0|_Gamma (the
solution's norm from a zero start) is at most tol.  mu: 1 for the tree
preconditioner (Section 4), gamma0 for none (Lemma 2.4: lambda_min(Gamma) >=
gamma0).

Pins (tests/test_oracle_error_bounds.py): the bound against the true error
of a dense solve at every k, the recursion against the Gauss-Radau rule
computed from the Lanczos matrix of the CG coefficients (Golub's
modification of the last diagonal entry), the norm identity, and the
guarantee at the stopped iterate.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import (ERR_NO_CONVERGENCE, ERR_NOT_SPD, OK, PRECOND_JACOBI, PRECOND_NONE, PRECOND_TREE, OracleError,
               TreeFactor, _f64, _i32, matvec, tree_solve)

STOP_RESIDUAL, STOP_ERROR = 0, 1


def default_mu(precond: int, gamma0: float) -> float:
    if precond == PRECOND_TREE:
        return 1.0          # Section 4: lambda_min(Gamma, P) >= 1
    if precond == PRECOND_NONE:
        return gamma0       # Lemma 2.4
    raise OracleError(1, "default_mu: block Jacobi has no bound in the paper; pass mu")


@dataclass
class GrResult:
    x: np.ndarray
    iters: int
    relres: float
    status: int
    alpha: list = field(default_factory=list)   # alpha_j, j = 0..iters-1
    rho: list = field(default_factory=list)     # rho_j, j = 0..(last computed)
    upper: list = field(default_factory=list)   # phi_j rho_j for every computed rho_j
    gsum: list = field(default_factory=list)    # sum_{i<j} alpha_i rho_i for the same j
    err_bound: float = 0.0                      # sqrt(upper / gsum) at the last computed rho


def pcg_gauss_radau(n: int, ij, blocks, gamma0: float, F, precond=PRECOND_TREE, factor: TreeFactor | None = None,
                    jacobi_dinv=None, mu: float = 0.0, tol: float = 1e-8, stop: int = STOP_ERROR,
                    maxit: int = 100000, fixed_iters: int = 0, x0=None) -> GrResult:
    """Section 1.1 PCG on Gamma x = F with the Gauss-Radau bound tracked at
    every step and (stop = STOP_ERROR) used as the stopping test."""
    ij, blocks, F = _i32(ij), _f64(blocks), _f64(F)
    mu = mu if mu > 0 else default_mu(precond, gamma0)

    def H(r):
        if precond == PRECOND_TREE:
            return tree_solve(factor, r)
        if precond == PRECOND_JACOBI:
            return np.einsum("nab,nb->na", _f64(jacobi_dinv), r)
        return r.copy()

    def dot(a, b):
        return float(np.dot(a.ravel(), b.ravel()))

    x = np.zeros((n, 3)) if x0 is None else _f64(x0).copy()
    res = GrResult(x, 0, 0.0, OK)
    FF = dot(F, F)
    if FF == 0.0:
        res.x = np.zeros((n, 3))
        return res
    r = F - matvec(n, ij, blocks, gamma0, x) if x0 is not None else F.copy()
    rr = dot(r, r)
    stop2 = tol * tol * FF
    if stop == STOP_RESIDUAL and fixed_iters <= 0 and rr <= stop2:
        res.relres = float(np.sqrt(rr / FF))
        return res
    z = H(r)
    p = z.copy()
    rho = dot(r, z)
    phi = 1.0 / mu
    gsum = 0.0
    res.rho.append(rho)
    res.upper.append(phi * rho)
    res.gsum.append(0.0)
    k = 0
    status = OK
    while True:
        q = matvec(n, ij, blocks, gamma0, p)
        pq = dot(p, q)
        if not pq > 0.0:
            status = ERR_NOT_SPD
            break
        alpha = rho / pq
        x = x + alpha * p
        r = r - alpha * q
        k += 1
        res.alpha.append(alpha)
        rr = dot(r, r)
        if fixed_iters > 0:
            if k >= fixed_iters:
                break
        else:
            if stop == STOP_RESIDUAL and rr <= stop2:
                break
            if k >= maxit:
                status = ERR_NO_CONVERGENCE
                break
        z = H(r)
        rho2 = dot(r, z)
        if not rho2 > 0.0:
            if rho2 == 0.0 and stop == STOP_ERROR:
                break          # exact solution
            status = ERR_NOT_SPD
            break
        beta = rho2 / rho
        gsum += alpha * rho
        d = phi - alpha
        phi = d / (mu * d + beta)
        rho = rho2
        res.rho.append(rho)
        res.upper.append(phi * rho)
        res.gsum.append(gsum)
        if stop == STOP_ERROR and fixed_iters <= 0 and phi * rho <= tol * tol * gsum:
            break
        p = z + beta * p
    res.x, res.iters, res.status = x, k, status
    res.relres = float(np.sqrt(rr / FF))
    if res.gsum[-1] > 0:
        res.err_bound = float(np.sqrt(max(res.upper[-1], 0.0) / res.gsum[-1]))
    return res


def lower_bound(res: GrResult, k: int, delay: int) -> float:
    """Hestenes-Stiefel lower bound of |x - x_k|_Gamma^2 with delay d:
    sum_{j=k}^{k+d-1} alpha_j rho_j (needs k + d <= len(alpha))."""
    return float(sum(res.alpha[j] * res.rho[j] for j in range(k, k + delay)))
