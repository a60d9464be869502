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


# ---------------------------------------------------------------------------
# The paper's experiment geometries (Section 5) and the Hertz contact law
# ---------------------------------------------------------------------------
def _golden(name):
    out = {}
    with open(__file__.replace("test_workloads.py", "golden/" + name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def test_hertz_two_cell_golden():
    g = _golden("hertz_two_cell.txt")
    pos = np.array([[0.0, 0.0, 0.0], [g["distance"], 0.0, 0.0]])
    radii = np.full(2, workloads.PAPER_R)
    gp, gq = workloads.hertz_gamma_np(pos, radii, np.array([[0, 1]]), workloads.PAPER_G_PAR,
                                      workloads.PAPER_G_PERP)
    np.testing.assert_allclose(gp, [g["g_par"]], rtol=1e-15)
    np.testing.assert_allclose(gq, [g["g_perp"]], rtol=1e-15)


def test_hertz_torch_twin_is_bit_identical():
    c = workloads.paper_random(n=2000, seed=17)
    ij = oracle.contacts(c.pos, c.radii)
    gp, gq = c.gammas_np(ij)
    tp, tq = c.gammas_torch(torch.from_numpy(ij.astype(np.int32)), torch.from_numpy(c.pos),
                            torch.from_numpy(c.radii))
    assert np.array_equal(gp, tp.numpy()) and np.array_equal(gq, tq.numpy())
    assert np.all(gp > 0)
    np.testing.assert_allclose(gq / gp, workloads.PAPER_G_PERP / workloads.PAPER_G_PAR, rtol=1e-15)


def test_hexagonal_close_packing_has_twelve_neighbours():
    c = workloads.paper_hex(n=3000, noise=0.0)
    sp = 2 * workloads.PAPER_R
    from scipy.spatial import cKDTree
    t = cKDTree(c.pos)
    d, _ = t.query(c.pos, k=13)
    assert np.allclose(d[:, 1].min(), sp) and d[:, 1].min() >= sp - 1e-12
    # cells well inside the cluster have 12 neighbours at the spacing
    centre = c.pos.mean(axis=0)
    inner = np.linalg.norm(c.pos - centre, axis=1) < 0.5 * np.linalg.norm(c.pos - centre, axis=1).max()
    counts = np.array([len(x) - 1 for x in t.query_ball_point(c.pos[inner], sp + 1e-9)])
    assert np.all(counts == 12)
    # ABAB stacking: the second shell at sqrt(2) spacing has 6 members
    # (face-centred ABC stacking has 6 as well, but HCP also has 2 at sqrt(8/3))
    counts83 = np.array([len(x) for x in t.query_ball_point(c.pos[inner], sp * np.sqrt(8 / 3) + 1e-9)]) - \
        np.array([len(x) for x in t.query_ball_point(c.pos[inner], sp * np.sqrt(8 / 3) - 1e-9)])
    assert np.all(counts83 == 2)
    noisy = workloads.paper_hex(n=3000, noise=0.3)
    dev = noisy.pos - c.pos
    assert abs(dev.std() - 0.3 * workloads.PAPER_R) < 0.01
    # the noise makes a lattice bond overlap when |(1 + a, b, c)| < 1, with
    # a, b, c ~ N(0, 2 (0.3 r)^2): a probability of 0.4145 (Monte Carlo, 1e6
    # samples); a few second-shell pairs (at sqrt(2) times the spacing) come
    # close enough too
    bonds = t.query_pairs(sp + 1e-9, output_type="ndarray")
    d = np.linalg.norm(noisy.pos[bonds[:, 0]] - noisy.pos[bonds[:, 1]], axis=1)
    assert abs((d < sp).mean() - 0.4145) < 0.02
    m = oracle.contacts(noisy.pos, noisy.radii).shape[0]
    assert (d < sp).sum() <= m <= 1.05 * (d < sp).sum()


def test_rejection_sampling_is_sequential_addition():
    """Batched rejection sampling equals the one-at-a-time rule: compare
    with a plain loop over the same candidate stream on a small case."""
    n, dmin = 400, 0.7
    a = 4.0
    inside = lambda c: np.sum(c * c, axis=1) <= a * a
    lo = np.array([-a, -a, -a])
    got = workloads._rejection_sample(np.random.Generator(np.random.PCG64([9, 9])), n, inside, lo, -lo, dmin,
                                      400 * n)
    # replay: the same generator, candidates in draw order, kept one by one
    g = np.random.Generator(np.random.PCG64([9, 9]))
    kept = []
    while len(kept) < n:
        m = max(4096, 4 * (n - len(kept)))
        cand = g.uniform(lo, -lo, size=(m, 3))
        cand = cand[inside(cand)]
        batch = []
        for x in cand:
            if all(np.sum((x - y) ** 2) >= dmin * dmin for y in kept + batch):
                batch.append(x)
        kept += batch[: n - len(kept)]
    assert np.array_equal(got, np.array(kept))
    from scipy.spatial import cKDTree
    d, _ = cKDTree(got).query(got, k=2)
    assert d[:, 1].min() >= dmin


def test_random_and_dumbbell_geometries():
    r = workloads.paper_random(n=3000, seed=19)
    a = r.meta["a"]
    x = r.pos
    assert np.all((x[:, 0] / a) ** 2 + (x[:, 1] / a) ** 2 + (x[:, 2] / (1.5 * a)) ** 2 <= 1.0 + 1e-12)
    d = workloads.paper_dumbbell(n=3000, seed=23)
    a, rb = d.meta["a"], d.meta["bridge_radius"]
    cx = 1.5 * a
    x = d.pos
    in_lobe = ((x[:, 0] - cx) ** 2 + x[:, 1] ** 2 + x[:, 2] ** 2 <= a * a) | \
              ((x[:, 0] + cx) ** 2 + x[:, 1] ** 2 + x[:, 2] ** 2 <= a * a)
    in_bridge = (np.abs(x[:, 0]) <= cx) & (x[:, 1] ** 2 + x[:, 2] ** 2 <= rb * rb)
    assert np.all(in_lobe | in_bridge)
    mid = np.abs(x[:, 0]) < 0.25 * a
    assert 0 < mid.sum() < 0.05 * d.n       # a thin bridge holds a few cells
    ij = oracle.contacts(d.pos, d.radii)
    assert np.any(np.abs(d.pos[ij[:, 0], 0]) < 0.25 * a)   # and they touch
