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


def test_output_head_selects_the_tree_solve():
    c, s, basis, ptr, nbr = small_problem()
    params = workloads.mpnn_init(5).astype(np.float64)
    params[-3 - 3 * 64:-3] = 0.0                   # W_out = 0
    params[-3:] = (0.0, 1.0, 0.0)                  # b_out picks b1 = P^-1 F
    v = mpnn.forward(params, basis, ptr, nbr)
    np.testing.assert_array_equal(v, basis[1])


def test_adam_first_step_is_a_signed_step():
    # bias correction makes the first update lr * g / (|g| + eps): a step of
    # length lr against the sign of every gradient entry well above eps
    g = np.array([3.0, -2e-3, 0.0, 1e-12, -7.5])
    p, m, v = mpnn.adam_step(np.ones(5), g, np.zeros(5), np.zeros(5), 1, 0.01)
    np.testing.assert_allclose(p[[0, 1, 4]], [0.99, 1.01, 1.01], rtol=0, atol=1e-7)
    assert p[2] == 1.0 and abs(p[3] - 1.0) < 1e-5
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_adam_constant_gradient_keeps_unit_steps():
    # with a constant gradient both bias-corrected moments are exact, so every
    # step has length lr
    p, m, v = np.zeros(2), np.zeros(2), np.zeros(2)
    g = np.array([0.5, -4.0])
    for t in range(1, 6):
        p, m, v = mpnn.adam_step(p, g, m, v, t, 0.1)
    np.testing.assert_allclose(p, [-0.5, 0.5], rtol=1e-6)


def test_energy_loss_gradient_against_finite_differences():
    c, s, basis, ptr, nbr = small_problem()
    mv = lambda x: oracle.matvec(c.n, s.ij, s.blocks, s.gamma0, x)
    rng = np.random.default_rng(2)
    params = workloads.mpnn_init(8).astype(np.float64)
    params[-3:] = rng.standard_normal(3)
    target = rng.standard_normal((c.n, 3))
    L, g = mpnn.backward(params, basis, ptr, nbr, target, round_bf16=False, matvec=mv)
    v0 = mpnn.forward(params, basis, ptr, nbr, round_bf16=False)
    # the energy loss is the Gamma-norm error: check it against the dense matrix
    G = oracle.dense_laplacian(c.n, s.ij, s.blocks, s.gamma0)
    e, t = (v0 - target).ravel(), target.ravel()
    assert np.isclose(L, e @ G @ e / (t @ G @ t), rtol=1e-12)
    idx = np.concatenate([rng.choice(params.size, size=40, replace=False), np.arange(params.size - 6, params.size)])
    eps = 1e-6
    for k in idx:
        pp, pm = params.copy(), params.copy()
        pp[k] += eps
        pm[k] -= eps
        fd = (mpnn.loss(mpnn.forward(pp, basis, ptr, nbr, round_bf16=False), target, mv) -
              mpnn.loss(mpnn.forward(pm, basis, ptr, nbr, round_bf16=False), target, mv)) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_minimal_residual_scaling_never_increases_the_residual():
    c, s, basis, ptr, nbr = small_problem()
    mv = lambda x: oracle.matvec(c.n, s.ij, s.blocks, s.gamma0, x)
    rng = np.random.default_rng(4)
    F = rng.standard_normal((c.n, 3))
    for scale in (1e-3, 1.0, 1e3):
        v = scale * rng.standard_normal((c.n, 3))
        w = mpnn.mr_scale(v, F, mv)
        assert np.linalg.norm(F - mv(w)) <= np.linalg.norm(F) * (1 + 1e-12)
        # the step is the 1-D least-squares minimiser: the residual is
        # orthogonal to Gamma v
        assert abs(np.sum((F - mv(w)) * mv(v))) <= 1e-9 * np.linalg.norm(F) * np.linalg.norm(mv(v))
    # the exact solution is left unchanged
    x = np.linalg.solve(oracle.dense_laplacian(c.n, s.ij, s.blocks, s.gamma0), F.ravel()).reshape(-1, 3)
    np.testing.assert_allclose(mpnn.mr_scale(x, F, mv), x, rtol=1e-9, atol=1e-12)


def test_relu_ambiguity_and_mask_flips():
    c, s, basis, ptr, nbr = small_problem()
    params = workloads.mpnn_init(9).astype(np.float64)
    target = np.random.default_rng(5).standard_normal((c.n, 3))
    # a huge band marks every unit whose bound is nonzero ...
    _, C0 = mpnn.forward(params, basis, ptr, nbr, cache=True)
    nz = sum(int(np.sum(np.abs(C0["hs"][l]).sum(axis=1) + np.abs(C0["aggs"][l]).sum(axis=1) > 0)) for l in range(3))
    assert len(mpnn.relu_ambiguous(params, basis, ptr, nbr, rel=2.0)) == (c.n + nz) * mpnn.H
    # ... a zero band none
    assert mpnn.relu_ambiguous(params, basis, ptr, nbr, rel=0.0) == []
    # flipping an inactive unit of the last layer adds exactly that unit's
    # contribution dh * input to its weight-gradient row
    _, C = mpnn.forward(params, basis, ptr, nbr, cache=True)
    i, k = map(int, np.argwhere(C["zs"][3] <= 0)[0])
    _, g0 = mpnn.backward(params, basis, ptr, nbr, target)
    _, g1 = mpnn.backward(params, basis, ptr, nbr, target, flips=[(3, i, k)])
    d = mpnn.unpack(g1 - g0)
    nrm = np.sum(target ** 2)
    dv = 2.0 * (mpnn.forward(params, basis, ptr, nbr) - target) / nrm
    dh = np.einsum("d,kd->k", dv[i], basis[:, i]) @ C["p"]["W_out"]
    u = np.concatenate([C["hs"][2][i], C["aggs"][2][i]])
    np.testing.assert_allclose(d["W2"][k], dh[k] * u, rtol=1e-10, atol=1e-14)
    assert np.isclose(d["c2"][k], dh[k])
    rows = np.delete(np.arange(mpnn.H), k)
    assert np.all(d["W2"][rows] == 0.0)
