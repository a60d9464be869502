"""Pins of the oracle's Gauss-Radau error bound and error-based stopping
(Sections 4 and 5) to a dense solve, to the Gauss-Radau quadrature rule
built from the Lanczos matrix of the CG coefficients, and to the norm
identities of CG."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import oracle.error_bounds as eb
import workloads

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def cells(n=150, seed=71, gamma0=1e-2):
    return workloads.cube(n=n, side=(n / 1.4253) ** (1.0 / 3.0), seed=seed, gamma0=gamma0)


def setup(n=150, seed=71, gamma0=1e-2):
    c = cells(n, seed, gamma0)
    s = oracle.build_system(c.pos, c.radii, c.gammas_np, c.gamma0)
    f = oracle.prim_msf(s.n, s.ij, s.w)
    fac = oracle.tree_ldlt(f, s.blocks, s.gamma0)
    G = oracle.dense_laplacian(s.n, s.ij, s.blocks, s.gamma0)
    return c, s, f, fac, G


def _anorm2(G, e):
    e = e.ravel()
    return float(e @ G @ e)


def _lanczos(res, k):
    """Jacobi matrix T_k of the CG coefficients (Lanczos for H Gamma)."""
    a, rho = res.alpha, res.rho
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / a[j] + (rho[j] / rho[j - 1] / a[j - 1] if j > 0 else 0.0)
        if j > 0:
            T[j, j - 1] = T[j - 1, j] = -np.sqrt(rho[j] / rho[j - 1]) / a[j - 1]
    return T


def test_bounds_bracket_the_true_error_at_every_step():
    c, s, f, fac, G = setup()
    F = c.forces()
    x = np.linalg.solve(G, F.ravel()).reshape(-1, 3)
    P = oracle.dense_laplacian(s.n, s.ij[np.sort(f.tree_edges)], s.blocks[np.sort(f.tree_edges)], s.gamma0)
    lam_min = sla.eigh(G, P, eigvals_only=True)[0]
    assert lam_min >= 1 - 1e-10            # Section 4: mu = 1 is admissible
    K = 40
    for mu in (1.0, lam_min * (1 - 1e-9)):
        res = eb.pcg_gauss_radau(s.n, s.ij, s.blocks, s.gamma0, F, oracle.PRECOND_TREE, fac, mu=mu,
                                 fixed_iters=K)
        # the iterates after k steps, from separate fixed-count runs
        for k in (0, 1, 2, 5, 10, 20, 30):
            xk = eb.pcg_gauss_radau(s.n, s.ij, s.blocks, s.gamma0, F, oracle.PRECOND_TREE, fac, mu=mu,
                                    fixed_iters=k).x if k else np.zeros_like(F)
            true = _anorm2(G, x - xk)
            assert res.upper[k] >= true * (1 - 1e-8), (mu, k)
            assert eb.lower_bound(res, k, 5) <= true * (1 + 1e-8)
            # |x_k|_Gamma^2 = sum_{j<k} alpha_j rho_j from a zero start (exact
            # arithmetic; rounding moves it by about eps kappa |x|^2)
            assert abs(_anorm2(G, xk) - res.gsum[k]) <= 1e-6 * _anorm2(G, x)


def test_recursion_equals_gauss_radau_rule_from_the_lanczos_matrix():
    """phi_k rho_k = rho_0 [(T~_{k+1}^-1)_11 - (T_k^-1)_11], T~ the Jacobi
    matrix with its last diagonal entry chosen so that mu is an eigenvalue
    (Golub), for k = 1..15; and rho_0 (T_k^-1)_11 = sum_{j<k} alpha_j rho_j."""
    c, s, f, fac, G = setup(n=120, seed=73)
    F = c.forces()
    mu = 1.0
    res = eb.pcg_gauss_radau(s.n, s.ij, s.blocks, s.gamma0, F, oracle.PRECOND_TREE, fac, mu=mu, fixed_iters=20)
    rho0 = res.rho[0]
    for k in range(1, 16):
        Tk = _lanczos(res, k)
        gauss = rho0 * np.linalg.inv(Tk)[0, 0]
        assert abs(gauss - res.gsum[k]) <= 1e-10 * gauss
        eta = np.sqrt(res.rho[k] / res.rho[k - 1]) / res.alpha[k - 1]
        ek = np.zeros(k)
        ek[-1] = 1.0
        d = np.linalg.solve(Tk - mu * np.eye(k), ek)
        omega = mu + eta ** 2 * d[-1]
        Tt = np.zeros((k + 1, k + 1))
        Tt[:k, :k] = Tk
        Tt[k, k - 1] = Tt[k - 1, k] = -eta
        Tt[k, k] = omega
        assert np.min(np.abs(np.linalg.eigvalsh(Tt) - mu)) <= 1e-8 * mu
        radau = rho0 * np.linalg.inv(Tt)[0, 0]
        np.testing.assert_allclose(res.upper[k], radau - gauss, rtol=1e-7, atol=1e-12 * gauss)


@pytest.mark.parametrize("tol", [1e-3, 1e-5, 1e-8])
def test_error_stopping_guarantees_the_tolerance(tol):
    c, s, f, fac, G = setup(n=200, seed=75)
    F = c.forces()
    x = np.linalg.solve(G, F.ravel()).reshape(-1, 3)
    res = eb.pcg_gauss_radau(s.n, s.ij, s.blocks, s.gamma0, F, oracle.PRECOND_TREE, fac, tol=tol)
    assert res.status == oracle.OK
    rel = np.sqrt(_anorm2(G, x - res.x) / _anorm2(G, res.x))
    assert rel <= tol
    assert res.err_bound <= tol and rel <= res.err_bound * (1 + 1e-6)
    # one step earlier the bound was still above the tolerance
    assert res.upper[-2] > tol * tol * res.gsum[-2]
    # the C oracle's PCG at the same count runs the same recurrence: the
    # iterates differ by rounding, amplified to a fraction of the error left
    same = oracle.pcg(s.n, s.ij, s.blocks, s.gamma0, F, oracle.PRECOND_TREE, fac, fixed_iters=res.iters)
    np.testing.assert_allclose(res.x, same.x, rtol=0, atol=tol * np.abs(same.x).max())


def test_identity_preconditioner_with_gamma0():
    c, s, f, fac, G = setup(n=100, seed=77, gamma0=0.5)
    F = c.forces()
    x = np.linalg.solve(G, F.ravel()).reshape(-1, 3)
    assert np.linalg.eigvalsh(G)[0] >= s.gamma0 * (1 - 1e-12)   # Lemma 2.4
    res = eb.pcg_gauss_radau(s.n, s.ij, s.blocks, s.gamma0, F, oracle.PRECOND_NONE, tol=1e-6)
    assert res.status == oracle.OK
    rel = np.sqrt(_anorm2(G, x - res.x) / _anorm2(G, res.x))
    assert rel <= 1e-6 and rel <= res.err_bound * (1 + 1e-6)


def test_edge_cases():
    c, s, f, fac, G = setup(n=80, seed=79)
    z = eb.pcg_gauss_radau(s.n, s.ij, s.blocks, s.gamma0, np.zeros((s.n, 3)), oracle.PRECOND_TREE, fac)
    assert z.iters == 0 and not z.x.any()
    with pytest.raises(oracle.OracleError):
        eb.default_mu(oracle.PRECOND_JACOBI, s.gamma0)
    # a wrong mu above lambda_min breaks the guarantee: the bound undershoots
    F = c.forces()
    x = np.linalg.solve(G, F.ravel()).reshape(-1, 3)
    res = eb.pcg_gauss_radau(s.n, s.ij, s.blocks, s.gamma0, F, oracle.PRECOND_TREE, fac, mu=1e6, fixed_iters=3)
    assert res.upper[0] < _anorm2(G, x)
