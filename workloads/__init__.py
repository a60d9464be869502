"""Seeded synthetic inputs for the support-graph PCG path.

This module is shared by the CPU oracle (``oracle/``), the tests and the
benchmark.  It draws positions, radii, forces and per-contact friction
coefficients and holds none of the method's arithmetic: no contact test, no
friction block, no spanning tree, no factorisation and no solve.

Input laws (the paper's cell model, Section 2 Steps 1-4 and eq. (1)):

* ``cube``   N cells, centres uniform in a cube of side L, radii U[0.45, 0.55].
* ``ball``   N cells, centres uniform in a ball (a spheroid of cells at a
             given packing fraction), radii U[0.45, 0.55].
* ``hex_sheet``  a monolayer: centres on a jittered hexagonal lattice in the
             z = 0 plane (jitter U[-j, j] on all three coordinates).
* ``batch``  many independent balls of log-uniform size.
* ``paper_hex``, ``paper_random``, ``paper_dumbbell``  the geometries of the
             paper's experiments (Section 5): equal cells r = 0.5 on a noisy
             hexagonal close packing, a rejection-sampled spheroid, and two
             lobes joined by a thin bridge; their coefficients follow the
             Hertz contact area (``hertz_gamma_np``) times the paper's
             gamma_par = 2e6 and gamma_perp = 8e7.

Per-contact friction coefficients gamma_par and gamma_perp (eq. (1)) are
drawn log-uniformly per unordered pair {i, j} by a counter-based generator:
SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) applied to a key built from (seed, i, j, stream).
The top 16 bits of the hash select one of 65536 equally spaced levels of
log(gamma); the level table is computed once on the host and handed to both
sides, so the coefficient of a pair is bit-identical on the CPU and on the
GPU.  ``pair_gamma_np`` (numpy, uint64) and ``pair_gamma_torch`` (torch,
int64 with wrap-around) implement the same integer arithmetic.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# SplitMix64 (published constants of the SplitMix64 finaliser)
# ---------------------------------------------------------------------------
_SM_INC = 0x9E3779B97F4A7C15
_SM_M1 = 0xBF58476D1CE4E5B9
_SM_M2 = 0x94D049BB133111EB
_MASK64 = (1 << 64) - 1
GAMMA_LEVELS_LOG2 = 16
GAMMA_LEVELS = 1 << GAMMA_LEVELS_LOG2


def splitmix64_np(x: np.ndarray) -> np.ndarray:
    """One SplitMix64 step on a uint64 array (wrap-around arithmetic)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(_SM_INC)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_SM_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_SM_M2)
        z = z ^ (z >> np.uint64(31))
    return z


def _s64(c: int) -> int:
    """Reinterpret an unsigned 64-bit constant as a signed int64."""
    c &= _MASK64
    return c - (1 << 64) if c >= (1 << 63) else c


def _lsr_torch(z, k: int):
    """Logical right shift of an int64 tensor (torch's >> is arithmetic)."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def splitmix64_torch(z):
    """Same SplitMix64 step on an int64 torch tensor (two's-complement wrap)."""
    z = z + _s64(_SM_INC)
    z = (z ^ _lsr_torch(z, 30)) * _s64(_SM_M1)
    z = (z ^ _lsr_torch(z, 27)) * _s64(_SM_M2)
    return z ^ _lsr_torch(z, 31)


def _stream_key(seed: int, stream: int) -> int:
    """Per-(seed, stream) 64-bit salt, computed with Python integers."""
    x = (int(seed) * 2 + int(stream)) & _MASK64
    return int(splitmix64_np(np.array([x], dtype=np.uint64))[0])


def gamma_table(lo: float, hi: float) -> np.ndarray:
    """Level table of a log-uniform law on [lo, hi]: level k sits at the
    midpoint of the k-th of GAMMA_LEVELS equal bins of log(gamma)."""
    k = np.arange(GAMMA_LEVELS, dtype=np.float64)
    return lo * np.exp((k + 0.5) / GAMMA_LEVELS * math.log(hi / lo))


def pair_gamma_np(seed: int, i: np.ndarray, j: np.ndarray, table_par: np.ndarray,
                  table_perp: np.ndarray):
    """(gamma_par, gamma_perp) for pairs (i, j); symmetric in i and j."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    a = np.minimum(i, j).astype(np.uint64)
    b = np.maximum(i, j).astype(np.uint64)
    key = (a << np.uint64(32)) | b
    out = []
    for s, tab in ((0, table_par), (1, table_perp)):
        h = splitmix64_np(key ^ np.uint64(_stream_key(seed, s)))
        lvl = (h >> np.uint64(64 - GAMMA_LEVELS_LOG2)).astype(np.int64)
        out.append(tab[lvl])
    return out[0], out[1]


def pair_gamma_torch(seed: int, ij, table_par, table_perp):
    """Torch twin of ``pair_gamma_np`` for an (m, 2) int32/int64 tensor of
    pairs; the tables are float64 tensors on the same device as ``ij``."""
    import torch
    ij = ij.to(torch.int64)
    a = torch.minimum(ij[:, 0], ij[:, 1])
    b = torch.maximum(ij[:, 0], ij[:, 1])
    key = (a << 32) | b
    out = []
    for s, tab in ((0, table_par), (1, table_perp)):
        h = splitmix64_torch(key ^ _s64(_stream_key(seed, s)))
        lvl = _lsr_torch(h, 64 - GAMMA_LEVELS_LOG2)
        out.append(tab[lvl])
    return out[0], out[1]


# ---------------------------------------------------------------------------
# Cell configurations
# ---------------------------------------------------------------------------
@dataclass
class Cells:
    """A synthetic cell configuration and the laws of its per-pair data."""
    name: str
    pos: np.ndarray              # (N, 3) float64, C-contiguous
    radii: np.ndarray            # (N,) float64
    seed: int
    gamma_lo: float
    gamma_hi: float
    gamma0: float
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    def tables(self):
        t = gamma_table(self.gamma_lo, self.gamma_hi)
        return t, t.copy()

    def gammas_np(self, ij: np.ndarray):
        tp, tq = self.tables()
        return pair_gamma_np(self.seed, ij[:, 0], ij[:, 1], tp, tq)

    def gammas_torch(self, ij, pos=None, radii=None):
        """The same coefficients for an (m, 2) torch tensor of pairs (on the
        pairs' device); pos and radii are the law's inputs where it has any."""
        import torch
        tp, tq = (torch.from_numpy(t).to(ij.device) for t in self.tables())
        return pair_gamma_torch(self.seed, ij, tp, tq)

    def forces(self, k: int = 0) -> np.ndarray:
        """F ~ N(0, 1) per component; ``k`` selects an independent draw."""
        rng = np.random.Generator(np.random.PCG64([self.seed, 7919, k]))
        return np.ascontiguousarray(rng.standard_normal((self.n, 3)))


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([seed, stream]))


def cube(n: int = 1000, side: float = 8.886, seed: int = 1000,
         r_lo: float = 0.45, r_hi: float = 0.55, gamma_lo: float = 0.1,
         gamma_hi: float = 10.0, gamma0: float = 1e-2) -> Cells:
    """Centres uniform in [0, side]^3.  side = 8.886 at N = 1000 gives a
    number density of 1.4253, i.e. a mean contact degree near 6 before
    boundary losses."""
    g = _rng(seed, 1)
    pos = np.ascontiguousarray(g.uniform(0.0, side, size=(n, 3)))
    radii = g.uniform(r_lo, r_hi, size=n)
    return Cells("cube", pos, radii, seed, gamma_lo, gamma_hi, gamma0,
                 {"side": side})


def ball_radius(n: int, packing: float = 0.6, mean_r3: float = 0.12625) -> float:
    """Ball radius that holds n cells at volume fraction ``packing``;
    mean_r3 = E[R^3] of the radius law (0.12625 for U[0.45, 0.55])."""
    return (n * mean_r3 / packing) ** (1.0 / 3.0)


def ball(n: int = 1_000_000, seed: int = 2000, radius: float | None = None,
         packing: float = 0.6, r_lo: float = 0.45, r_hi: float = 0.55,
         gamma_lo: float = 0.1, gamma_hi: float = 10.0,
         gamma0: float = 1e-3) -> Cells:
    """Centres uniform (Poisson) in a ball; the default radius gives the
    requested packing fraction for the radius law."""
    if radius is None:
        radius = ball_radius(n, packing)
    g = _rng(seed, 2)
    d = g.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius * np.cbrt(g.uniform(0.0, 1.0, size=n))
    pos = np.ascontiguousarray(d * r[:, None])
    radii = g.uniform(r_lo, r_hi, size=n)
    return Cells("ball", pos, radii, seed, gamma_lo, gamma_hi, gamma0,
                 {"radius": radius})


def hex_sheet(nx: int = 2000, ny: int = 2000, spacing: float = 0.9,
              jitter: float = 0.05, seed: int = 3000, r_lo: float = 0.48,
              r_hi: float = 0.52, gamma_lo: float = 0.01,
              gamma_hi: float = 100.0, gamma0: float = 1e-4) -> Cells:
    """A monolayer: a rhombic nx-by-ny patch of the hexagonal lattice with
    spacing ``spacing`` in the z = 0 plane, every coordinate jittered by
    U[-jitter, jitter]."""
    g = _rng(seed, 3)
    p, q = np.meshgrid(np.arange(nx, dtype=np.float64),
                       np.arange(ny, dtype=np.float64), indexing="xy")
    x = spacing * (p + 0.5 * q)
    y = spacing * (math.sqrt(3.0) / 2.0) * q
    pos = np.stack([x.ravel(), y.ravel(), np.zeros(nx * ny)], axis=1)
    pos = np.ascontiguousarray(pos + g.uniform(-jitter, jitter, size=pos.shape))
    radii = g.uniform(r_lo, r_hi, size=nx * ny)
    return Cells("hex_sheet", pos, radii, seed, gamma_lo, gamma_hi, gamma0,
                 {"nx": nx, "ny": ny, "spacing": spacing})


def batch_sizes(count: int = 512, lo: float = 1e3, hi: float = 1e5,
                seed: int = 4000) -> np.ndarray:
    """Instance sizes log-uniform in [lo, hi]."""
    g = _rng(seed, 4)
    return np.floor(np.exp(g.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)


def batch_instance(n: int, s: int, density: float = 1.4253, seed0: int = 4000,
                   gamma0: float = 1e-2) -> Cells:
    """Instance s of the batch: a ball at the cube workload's number density."""
    radius = (3.0 * n / (4.0 * math.pi * density)) ** (1.0 / 3.0)
    return ball(n, seed=seed0 + s, radius=radius, gamma0=gamma0)


def sphere_offsets(sizes: np.ndarray) -> np.ndarray:
    """Exclusive prefix sums of instance sizes (length count + 1)."""
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    return off


# ---------------------------------------------------------------------------
# Initial weights of the warm-start network (drawn here so that the GPU and
# the oracle start from the same values)
# ---------------------------------------------------------------------------
MPNN_H, MPNN_K, MPNN_DIN = 64, 3, 8


def mpnn_init(seed: int = 5000) -> np.ndarray:
    """FP32 master parameters, flat, in the order W_in (64x8), b_in, then for
    each of 3 layers W (64x128) and c (64), then W_out (3x64), b_out (3).
    Glorot-uniform matrices, zero biases, W_out scaled by 0.01: the
    untrained network returns a guess close to zero, so training starts
    from the solver's own default."""
    g = _rng(seed, 5)
    H, K, D = MPNN_H, MPNN_K, MPNN_DIN
    parts = []

    def glorot(o, i):
        a = math.sqrt(6.0 / (o + i))
        return g.uniform(-a, a, size=(o, i))

    parts += [glorot(H, D).ravel(), np.zeros(H)]
    for _ in range(3):
        parts += [glorot(H, 2 * H).ravel(), np.zeros(H)]
    parts += [0.01 * glorot(K, H).ravel(), np.zeros(K)]
    return np.concatenate(parts).astype(np.float32)


# ---------------------------------------------------------------------------
# Time stepping of the learned-warm-start workload: overlap springs plus
# active noise, positions advanced by x <- x + v dt
# ---------------------------------------------------------------------------
def spring_forces_np(pos: np.ndarray, radii: np.ndarray, ij: np.ndarray, k: float = 1.0) -> np.ndarray:
    """Repulsive overlap springs: each contact (i, j) pushes j away from i
    with k * (R_i + R_j - |r_j - r_i|) along u = (r_j - r_i) / |r_j - r_i|
    and i away from j by the opposite force."""
    ij = np.asarray(ij, dtype=np.int64)
    d = pos[ij[:, 1]] - pos[ij[:, 0]]
    dist = np.sqrt(np.sum(d * d, axis=1))
    ov = np.maximum(radii[ij[:, 0]] + radii[ij[:, 1]] - dist, 0.0)
    f = (k * ov / dist)[:, None] * d
    F = np.zeros_like(pos)
    np.add.at(F, ij[:, 0], -f)
    np.add.at(F, ij[:, 1], f)
    return F


def spring_forces_torch(pos, radii, ij, k: float = 1.0):
    """Torch twin of ``spring_forces_np`` with a fixed summation order per
    cell (contacts sorted by cell, summed along a padded table), so the same
    inputs give the same bits on every run."""
    import torch
    n = pos.shape[0]
    ij = ij.to(torch.int64)
    if ij.shape[0] == 0:
        return torch.zeros_like(pos)
    a, b = ij[:, 0], ij[:, 1]
    d = pos[b] - pos[a]
    dist = torch.sqrt(torch.sum(d * d, dim=1))
    ov = torch.clamp(radii[a] + radii[b] - dist, min=0.0)
    f = (k * ov / dist)[:, None] * d
    rows = torch.cat([a, b])
    vals = torch.cat([-f, f])
    order = torch.argsort(rows, stable=True)
    rows, vals = rows[order], vals[order]
    deg = torch.bincount(rows, minlength=n)
    start = torch.cumsum(deg, 0) - deg
    slot = torch.arange(rows.numel(), device=pos.device) - start[rows]
    tab = torch.zeros((n, int(deg.max().item()), 3), dtype=pos.dtype, device=pos.device)
    tab[rows, slot] = vals
    return tab.sum(dim=1)


def active_noise(seed: int, step: int, n: int, sigma: float = 0.1) -> np.ndarray:
    """Per-cell active force N(0, sigma^2) per component, drawn afresh at
    every time step."""
    rng = np.random.Generator(np.random.PCG64([seed, 7717, step]))
    return np.ascontiguousarray(sigma * rng.standard_normal((n, 3)))


def spheroid_200k(seed: int = 5000) -> Cells:
    """The learned-warm-start workload's spheroid: 200,000 cells in a ball at
    packing fraction 0.6 (radius 34.78), gamma in [0.1, 10], gamma0 = 1e-3."""
    return ball(n=200_000, seed=seed, gamma0=1e-3)


# ---------------------------------------------------------------------------
# The paper's own experiment geometries (Section 5, Experimental Setup):
# equal cells of radius r = 0.5, Hertz contact areas, gamma_par = 2e6,
# gamma_perp = 8e7 per unit area, cell-substrate friction gamma_med I
# ---------------------------------------------------------------------------
PAPER_R = 0.5
PAPER_G_PAR, PAPER_G_PERP = 2.0e6, 8.0e7


def hertz_gamma_np(pos: np.ndarray, radii: np.ndarray, ij: np.ndarray, g_par: float, g_perp: float):
    """Per-contact coefficients A_ij g_par and A_ij g_perp with the Hertz
    contact area A_ij = pi R* delta (contact radius sqrt(R* delta)), R* =
    R_i R_j / (R_i + R_j), delta = R_i + R_j - |r_j - r_i| the overlap.
    Every operation in a fixed order (the torch twin repeats it)."""
    ij = np.asarray(ij, dtype=np.int64)
    a, b = ij[:, 0], ij[:, 1]
    d0 = pos[b, 0] - pos[a, 0]
    d1 = pos[b, 1] - pos[a, 1]
    d2 = pos[b, 2] - pos[a, 2]
    dist = np.sqrt(d0 * d0 + d1 * d1 + d2 * d2)
    s = radii[a] + radii[b]
    area = (math.pi * ((radii[a] * radii[b]) / s)) * (s - dist)
    return area * g_par, area * g_perp


def hertz_gamma_torch(pos, radii, ij, g_par: float, g_perp: float):
    """``hertz_gamma_np`` for torch tensors: evaluated on the host and copied
    to the pairs' device, so both sides hold the same bits (the square root
    of torch's CPU kernels is not always the correctly rounded one)."""
    import torch
    gp, gq = hertz_gamma_np(pos.detach().cpu().numpy(), radii.detach().cpu().numpy(),
                            ij.detach().cpu().numpy(), g_par, g_perp)
    return torch.from_numpy(gp).to(ij.device), torch.from_numpy(gq).to(ij.device)


class HertzCells(Cells):
    """A configuration whose per-contact coefficients follow the Hertz law."""

    def gammas_np(self, ij: np.ndarray):
        return hertz_gamma_np(self.pos, self.radii, ij, self.meta["g_par"], self.meta["g_perp"])

    def gammas_torch(self, ij, pos, radii):
        return hertz_gamma_torch(pos, radii, ij, self.meta["g_par"], self.meta["g_perp"])


def _paper_cells(name, pos, seed, gamma_med, meta):
    n = pos.shape[0]
    meta = dict(meta, g_par=PAPER_G_PAR, g_perp=PAPER_G_PERP)
    return HertzCells(name, np.ascontiguousarray(pos), np.full(n, PAPER_R), seed, 0.0, 0.0, gamma_med, meta)


def _nearest_to_centre(pts: np.ndarray, n: int) -> np.ndarray:
    c = pts.mean(axis=0)
    d2 = np.sum((pts - c) ** 2, axis=1)
    order = np.lexsort((np.arange(pts.shape[0]), d2))   # distance, then index
    return pts[np.sort(order[:n])]


def paper_hex(n: int = 50_000, spacing: float = 2 * PAPER_R, noise: float = 0.3, seed: int = 6000,
              gamma_med: float = 3.0e4) -> HertzCells:
    """Hexagonal close packing (ABAB stacking of hexagonal layers, 12
    neighbours at distance ``spacing``, by default 2r: the spheres of the
    packing touch their 12 neighbours): the n lattice sites nearest the
    centre of a large block, each coordinate perturbed by N(0, (noise r)^2).
    The noise turns about half of the touching pairs into overlaps (contacts
    with a Hertz area) and separates the rest."""
    k = int(math.ceil((n * 1.6) ** (1.0 / 3.0))) + 2
    h = spacing * math.sqrt(2.0 / 3.0)
    p, q, l = np.meshgrid(np.arange(k, dtype=np.float64), np.arange(k, dtype=np.float64),
                          np.arange(k, dtype=np.float64), indexing="ij")
    odd = np.mod(l, 2.0)
    x = spacing * (p + 0.5 * q + 0.5 * odd)
    y = spacing * (math.sqrt(3.0) / 2.0) * (q + odd / 3.0)
    z = h * l
    pts = _nearest_to_centre(np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1), n)
    g = _rng(seed, 6)
    pts = pts + g.normal(0.0, noise * PAPER_R, size=pts.shape)
    return _paper_cells("paper_hex", pts, seed, gamma_med, {"spacing": spacing, "noise": noise})


def _rejection_sample(g: np.random.Generator, n: int, inside, lo: np.ndarray, hi: np.ndarray, dmin: float,
                      max_tries: int):
    """Random sequential addition: points drawn uniformly in the box [lo, hi]
    and, in draw order, kept when ``inside`` holds and no kept point lies
    closer than dmin.  Candidates are drawn in batches; a batch is checked
    against the kept points with a k-d tree and then against its own earlier
    members in draw order, which is the sequential rule."""
    from scipy.spatial import cKDTree
    kept = np.empty((0, 3))
    tree = None
    tries = 0
    while kept.shape[0] < n:
        if tries >= max_tries:
            raise RuntimeError("rejection sampling: the domain is too full")
        m = max(4096, 4 * (n - kept.shape[0]))
        cand = g.uniform(lo, hi, size=(m, 3))
        tries += m
        cand = cand[inside(cand)]
        if tree is not None and cand.shape[0]:
            d, _ = tree.query(cand, k=1, distance_upper_bound=dmin)
            cand = cand[~(d < dmin)]
        if cand.shape[0] == 0:
            continue
        pairs = cKDTree(cand).query_pairs(dmin, output_type="ndarray")
        first, second = np.minimum(pairs[:, 0], pairs[:, 1]), np.maximum(pairs[:, 0], pairs[:, 1])
        # in draw order: a candidate is kept unless an earlier kept candidate
        # conflicts with it; decided by rounds (undecided 0, kept 1, dead 2)
        state = np.zeros(cand.shape[0], dtype=np.int8)
        while (state == 0).any():
            hit = np.zeros(cand.shape[0], dtype=bool)
            np.logical_or.at(hit, second, state[first] == 1)
            state[(state == 0) & hit] = 2
            wait = np.zeros(cand.shape[0], dtype=bool)
            np.logical_or.at(wait, second, state[first] == 0)
            state[(state == 0) & ~wait] = 1
        take = np.nonzero(state == 1)[0][: n - kept.shape[0]]
        kept = np.concatenate([kept, cand[take]])
        tree = cKDTree(kept)
    return kept


def paper_random(n: int = 50_000, density: float = 1.6, dmin: float = 0.7, aspect: float = 1.5,
                 seed: int = 7000, gamma_med: float = 3.0e4) -> HertzCells:
    """Random packing in a spheroid (semi-axes a, a, aspect a, volume n /
    density) by rejection sampling with a minimum centre distance dmin < 2r
    (cells may overlap, so they touch, but not pile up)."""
    a = (3.0 * n / (4.0 * math.pi * aspect * density)) ** (1.0 / 3.0)
    inside = lambda c: (c[:, 0] / a) ** 2 + (c[:, 1] / a) ** 2 + (c[:, 2] / (aspect * a)) ** 2 <= 1.0
    g = _rng(seed, 7)
    lo = np.array([-a, -a, -aspect * a])
    pts = _rejection_sample(g, n, inside, lo, -lo, dmin, 400 * n)
    return _paper_cells("paper_random", pts, seed, gamma_med, {"a": a, "density": density, "dmin": dmin})


def paper_dumbbell(n: int = 50_000, density: float = 1.6, dmin: float = 0.7, bridge_radius: float = 1.5,
                   seed: int = 8000, gamma_med: float = 3.0e4) -> HertzCells:
    """Two equal spherical lobes joined by a thin cylindrical bridge (radius
    bridge_radius, length one lobe radius), all filled by the same rejection
    sampling: the graph has a bottleneck."""
    # volumes: 2 lobes of radius a and a bridge of length a
    f = lambda a: 2 * (4.0 / 3.0) * math.pi * a ** 3 + math.pi * bridge_radius ** 2 * a - n / density
    lo_a, hi_a = 1.0, 1000.0
    for _ in range(200):
        mid = 0.5 * (lo_a + hi_a)
        lo_a, hi_a = (mid, hi_a) if f(mid) < 0 else (lo_a, mid)
    a = 0.5 * (lo_a + hi_a)
    cx = a + 0.5 * a   # lobe centres at x = +-cx; the bridge spans |x| <= a / 2 plus the caps' overlap

    def inside(c):
        l1 = (c[:, 0] - cx) ** 2 + c[:, 1] ** 2 + c[:, 2] ** 2 <= a * a
        l2 = (c[:, 0] + cx) ** 2 + c[:, 1] ** 2 + c[:, 2] ** 2 <= a * a
        br = (np.abs(c[:, 0]) <= cx) & (c[:, 1] ** 2 + c[:, 2] ** 2 <= bridge_radius ** 2)
        return l1 | l2 | br

    g = _rng(seed, 8)
    lo = np.array([-cx - a, -a, -a])
    pts = _rejection_sample(g, n, inside, lo, -lo, dmin, 400 * n)
    return _paper_cells("paper_dumbbell", pts, seed, gamma_med,
                        {"a": a, "density": density, "dmin": dmin, "bridge_radius": bridge_radius})
