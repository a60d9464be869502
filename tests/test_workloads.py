"""Input generators of the time-stepping workload: the spring forces'
torch twin against the numpy definition, a hand-worked two-cell value and
momentum balance."""
import numpy as np
import torch

import oracle
import workloads


def test_two_cell_spring_force():
    pos = np.array([[0.0, 0.0, 0.0], [0.6, 0.8, 0.0]])  # distance 1
    radii = np.array([0.55, 0.65])                       # overlap 0.2
    F = workloads.spring_forces_np(pos, radii, np.array([[0, 1]]), k=2.0)
    np.testing.assert_allclose(F, [[-0.24, -0.32, 0.0], [0.24, 0.32, 0.0]], rtol=1e-14)


def test_spring_forces_torch_twin_and_momentum_balance():
    c = workloads.ball(n=800, seed=11)
    ij = oracle.contacts(c.pos, c.radii)
    F = workloads.spring_forces_np(c.pos, c.radii, ij)
    Ft = workloads.spring_forces_torch(torch.from_numpy(c.pos), torch.from_numpy(c.radii),
                                       torch.from_numpy(ij.astype(np.int32))).numpy()
    np.testing.assert_allclose(Ft, F, rtol=1e-12, atol=1e-14)
    assert np.abs(F.sum(axis=0)).max() <= 1e-12 * np.abs(F).sum()
    # cells without contacts feel no spring force
    deg = np.bincount(ij.ravel(), minlength=c.n)
    assert np.all(F[deg == 0] == 0.0)
    # the same draw for the same step, a fresh one for the next
    a = workloads.active_noise(1, 3, 50)
    assert np.array_equal(a, workloads.active_noise(1, 3, 50))
    assert not np.array_equal(a, workloads.active_noise(1, 4, 50))
    assert abs(a.std() - 0.1) < 0.03
