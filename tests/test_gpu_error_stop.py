"""PCG stopped on the Gauss-Radau bound of the Gamma-norm error (Sections 4
and 5) through the C ABI, against the oracle: iteration counts, the bound,
and the guarantee |v* - v|_Gamma <= tol |v|_Gamma at the returned iterate."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import oracle.error_bounds as eb
import paper_2410_04512_gb300 as sgp
import workloads
from gpu_common import GpuSystem, dev_tensor, oracle_system, small_cube

pytestmark = pytest.mark.gpu


def _ctx(bin_cap=0):
    c = sgp.Context(0)
    c.set_tuning(bin_cap=bin_cap)
    return c


def _gnorm(c, o, e):
    return float(np.sqrt(np.sum(e * oracle.matvec(c.n, o.ij, o.blocks, c.gamma0, e))))


def _reference(c, o, fac):
    F = c.forces()
    return F, oracle.pcg(c.n, o.ij, o.blocks, c.gamma0, F, oracle.PRECOND_TREE, fac, tol=1e-14).x


@pytest.fixture(scope="module")
def cube3k():
    c = small_cube(3000, seed=1006)
    o = oracle_system(c)
    f = oracle.prim_msf(c.n, o.ij, o.w)
    fac = oracle.tree_ldlt(f, o.blocks, c.gamma0)
    F, xs = _reference(c, o, fac)
    return c, o, fac, F, xs


@pytest.mark.parametrize("tol", [1e-4, 1e-6, 1e-9])
@pytest.mark.parametrize("bin_cap", [-1, 1024])
def test_error_stop_matches_oracle(cuda_device, cube3k, tol, bin_cap):
    c, o, fac, F, xs = cube3k
    cx = _ctx(bin_cap)
    s = GpuSystem(cx, c)
    assert (s.Fac.layout()["fp64"] == 1) == (bin_cap > 0)
    v, info = cx.pcg_solve(s.M, s.Fac, dev_tensor(F), tol=tol, stop=sgp.STOP_ERROR)
    want = eb.pcg_gauss_radau(c.n, o.ij, o.blocks, c.gamma0, F, oracle.PRECOND_TREE, fac, tol=tol)
    assert info.status == 0 and want.status == 0
    assert abs(info.iterations - want.iters) <= 1
    x = v.cpu().numpy()
    rel = _gnorm(c, o, xs - x) / _gnorm(c, o, x)
    assert rel <= tol * (1 + 1e-6)
    assert info.err_bound <= tol and rel <= info.err_bound * (1 + 1e-6)
    if info.iterations == want.iters:
        # the same recursion on scalars that differ by rounding (summation
        # order); rho_k carries a relative error of about eps kappa / |r_k|,
        # so the two bounds drift apart as the residual falls
        assert abs(info.err_bound - want.err_bound) <= 0.1 * want.err_bound


def test_residual_mode_reports_a_valid_bound(cuda_device, cube3k):
    c, o, fac, F, xs = cube3k
    cx = _ctx()
    s = GpuSystem(cx, c)
    v, info = cx.pcg_solve(s.M, s.Fac, dev_tensor(F), tol=1e-6)
    x = v.cpu().numpy()
    rel = _gnorm(c, o, xs - x) / _gnorm(c, o, x)
    assert 0 < info.err_bound and rel <= info.err_bound * (1 + 1e-6)


def test_no_preconditioner_uses_gamma0(cuda_device):
    c = small_cube(1500, seed=1007, gamma0=0.3)
    o = oracle_system(c)
    cx = _ctx()
    s = GpuSystem(cx, c, tree=False)
    F = c.forces()
    v, info = cx.pcg_solve(s.M, None, dev_tensor(F), tol=1e-6, precond=sgp.PRECOND_NONE, stop=sgp.STOP_ERROR)
    want = eb.pcg_gauss_radau(c.n, o.ij, o.blocks, c.gamma0, F, oracle.PRECOND_NONE, tol=1e-6)
    assert abs(info.iterations - want.iters) <= 1
    xs = oracle.pcg(c.n, o.ij, o.blocks, c.gamma0, F, oracle.PRECOND_NONE, tol=1e-14).x
    x = v.cpu().numpy()
    assert _gnorm(c, o, xs - x) / _gnorm(c, o, x) <= 1e-6 * (1 + 1e-6)


def test_block_jacobi_needs_mu(cuda_device):
    c = small_cube(1000, seed=1008)
    o = oracle_system(c)
    cx = _ctx()
    s = GpuSystem(cx, c, tree=False)
    F = c.forces()
    with pytest.raises(sgp.SgpError):
        cx.pcg_solve(s.M, None, dev_tensor(F), precond=sgp.PRECOND_BLOCK_JACOBI, stop=sgp.STOP_ERROR)
    # any mu below lambda_min(D^-1 Gamma) keeps the guarantee; gamma0 / max
    # lambda_max(D_ii) is one (D <= lambda_max(D) I)
    dj = oracle.block_jacobi(c.n, o.ij, o.blocks, c.gamma0)
    mu = c.gamma0 * min(np.linalg.eigvalsh(d)[0] for d in dj)
    v, info = cx.pcg_solve(s.M, None, dev_tensor(F), tol=1e-6, precond=sgp.PRECOND_BLOCK_JACOBI,
                           stop=sgp.STOP_ERROR, mu=mu)
    xs = oracle.pcg(c.n, o.ij, o.blocks, c.gamma0, F, oracle.PRECOND_JACOBI, jacobi_dinv=dj, tol=1e-14).x
    x = v.cpu().numpy()
    assert _gnorm(c, o, xs - x) / _gnorm(c, o, x) <= 1e-6 * (1 + 1e-6)
    want = eb.pcg_gauss_radau(c.n, o.ij, o.blocks, c.gamma0, F, oracle.PRECOND_JACOBI, jacobi_dinv=dj, mu=mu,
                              tol=1e-6)
    assert abs(info.iterations - want.iters) <= 1


def test_invalid_combinations(cuda_device):
    c = small_cube(800, seed=1009)
    cx = _ctx()
    s = GpuSystem(cx, c, precision=sgp.PREC_MIXED)
    F = dev_tensor(c.forces())
    with pytest.raises(sgp.SgpError):
        cx.pcg_solve(s.M, s.Fac, F, precision=sgp.PREC_MIXED, stop=sgp.STOP_ERROR)
    with pytest.raises(sgp.SgpError):
        cx.pcg_solve(s.M, s.Fac, F, stop=2)
    with pytest.raises(sgp.SgpError):
        cx.pcg_solve(s.M, s.Fac, F, stop=sgp.STOP_ERROR, mu=float("nan"))
    # a zero right-hand side stops at once in error mode too
    v, info = cx.pcg_solve(s.M, s.Fac, F * 0, stop=sgp.STOP_ERROR)
    assert info.iterations == 0 and not v.any()
