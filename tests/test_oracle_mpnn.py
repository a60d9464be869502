"""Pins of the warm-start network's CPU oracle: gradients against central
finite differences, rotation and permutation equivariance, BF16 rounding
against hand-worked values, and the untrained network's output."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import mpnn


def small_problem(n=60, seed=3):
    c = workloads.cube(n=n, side=(n / 1.4253) ** (1 / 3), seed=seed)
    s = oracle.build_system(c.pos, c.radii, c.gammas_np, c.gamma0)
    rng = np.random.default_rng(seed)
    basis = rng.standard_normal((3, n, 3))
    ptr, nbr = mpnn.adjacency(n, s.ij)
    return c, s, basis, ptr, nbr


def test_parameter_count_and_layout():
    p = workloads.mpnn_init(1)
    assert p.dtype == np.float32 and p.size == mpnn.N_PARAMS
    assert mpnn.N_PARAMS == 64 * 8 + 64 + 3 * (64 * 128 + 64) + 3 * 64 + 3
    assert np.array_equal(mpnn.pack(mpnn.unpack(p.astype(np.float64))), p.astype(np.float64))


def test_bf16_rounding_hand_values():
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, 1.0 + 2.0 ** -7 + 2.0 ** -8, -2.5,
                     0.0, 1.0 + 2.0 ** -9], dtype=np.float32)
    # ties go to the even neighbour; 1 + 2^-7 is odd in the last BF16 bit
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -7, 1.0 + 2.0 ** -6, -2.5, 0.0, 1.0])
    np.testing.assert_array_equal(mpnn.bf16_round(vals), want)


def test_gradient_against_finite_differences():
    c, s, basis, ptr, nbr = small_problem()
    rng = np.random.default_rng(0)
    params = workloads.mpnn_init(7).astype(np.float64)
    params[-3:] = rng.standard_normal(3)          # non-trivial output head
    target = rng.standard_normal((c.n, 3))
    L, g = mpnn.backward(params, basis, ptr, nbr, target, round_bf16=False)
    assert np.isclose(L, mpnn.loss(mpnn.forward(params, basis, ptr, nbr, round_bf16=False), target))
    idx = rng.choice(params.size, size=60, replace=False)
    idx = np.concatenate([idx, np.arange(params.size - 10, params.size)])
    eps = 1e-6
    for k in idx:
        pp, pm = params.copy(), params.copy()
        pp[k] += eps
        pm[k] -= eps
        fd = (mpnn.loss(mpnn.forward(pp, basis, ptr, nbr, round_bf16=False), target) -
              mpnn.loss(mpnn.forward(pm, basis, ptr, nbr, round_bf16=False), target)) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_rotation_equivariance():
    c, s, basis, ptr, nbr = small_problem()
    params = workloads.mpnn_init(3).astype(np.float64)
    params[-3:] = [0.3, 0.9, -0.2]
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    R = R @ np.array([[1, 0, 0], [0, np.cos(1.1), -np.sin(1.1)], [0, np.sin(1.1), np.cos(1.1)]])
    v = mpnn.forward(params, basis, ptr, nbr)
    vr = mpnn.forward(params, basis @ R.T, ptr, nbr)
    np.testing.assert_allclose(vr, v @ R.T, rtol=1e-10, atol=1e-12)


def test_permutation_equivariance():
    c, s, basis, ptr, nbr = small_problem()
    params = workloads.mpnn_init(4).astype(np.float64)
    params[-3:] = [0.5, 0.5, 0.1]
    perm = np.random.default_rng(1).permutation(c.n)
    inv = np.argsort(perm)
    ij2 = np.sort(inv[s.ij], axis=1)
    ptr2, nbr2 = mpnn.adjacency(c.n, ij2)
    v = mpnn.forward(params, basis, ptr, nbr)
    v2 = mpnn.forward(params, basis[:, perm], ptr2, nbr2)
    np.testing.assert_allclose(v2, v[perm], rtol=1e-10, atol=1e-12)


def test_untrained_network_returns_the_tree_solve():
    c, s, basis, ptr, nbr = small_problem()
    params = workloads.mpnn_init(5).astype(np.float64)
    params[-3 - 3 * 64:-3] = 0.0                   # W_out = 0
    v = mpnn.forward(params, basis, ptr, nbr)
    np.testing.assert_array_equal(v, basis[1])
