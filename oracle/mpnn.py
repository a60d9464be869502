"""CPU oracle of the learned warm start (a message-passing network that
predicts the PCG initial guess).  TEST INFRASTRUCTURE ONLY (see
oracle/__init__.py).  The paper has no learned component; this is the
definition the GPU kernels must reproduce.

Network (width H = 64, 3 message-passing layers, BF16 weights):
  basis (K = 3 vector fields per cell): b0 = D^-1 F (block-Jacobi solve),
        b1 = P^-1 F (spanning-forest solve), b2 = v_prev (zero if none)
  features x_i (8): |b0|, |b1|, |b2|, b0.b1, b0.b2, b1.b2 (all divided by
        the mean |b1| of the step, the products by its square), deg_i / 6, 1
  h0 = relu(W_in x + b_in)                                (8 -> 64)
  for l = 1..3:  a_i = mean_{j ~ i} h_j   (0 for an isolated cell)
                 h_l = relu(W_l [h; a] + c_l)             (128 -> 64)
  c = W_out h3 + b_out                                    (64 -> 3)
  v0_i = sum_k c_ik b_i^(k)
Every input is rotation invariant and every output vector a scalar
combination of equivariant fields, so rotating F (and the geometry) rotates
v0.  Two training losses against the converged solution v*:
  "l2":     L = |v0 - v*|^2 / |v*|^2
  "energy": L = (v0 - v*)^T Gamma (v0 - v*) / v*^T Gamma v*, the error norm
            that conjugate gradients minimises over its Krylov space.
Inference may rescale the prediction by the minimal-residual step
alpha = (Gamma v0)^T F / |Gamma v0|^2, after which |F - Gamma v0| <= |F|.
Weights enter in BF16 (round-to-nearest-even of the FP32 master values);
arithmetic here is FP64.
"""
from __future__ import annotations

import numpy as np

H = 64
K = 3
D_IN = 8
SHAPES = [("W_in", (H, D_IN)), ("b_in", (H,))]
for _l in range(3):
    SHAPES += [(f"W{_l}", (H, 2 * H)), (f"c{_l}", (H,))]
SHAPES += [("W_out", (K, H)), ("b_out", (K,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = flat[o:o + k].reshape(shp)
        o += k
    return out


def pack(params: dict) -> np.ndarray:
    return np.concatenate([np.asarray(params[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round FP32 values to BF16 (round to nearest, ties to even) and return
    them as FP64 (exact)."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def adjacency(n: int, ij: np.ndarray):
    """Neighbour lists (both directions) as CSR."""
    a = np.concatenate([ij[:, 0], ij[:, 1]]).astype(np.int64)
    b = np.concatenate([ij[:, 1], ij[:, 0]]).astype(np.int64)
    order = np.lexsort((b, a))
    a, b = a[order], b[order]
    ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(ptr, a + 1, 1)
    return np.cumsum(ptr), b


def features(basis: np.ndarray, deg: np.ndarray) -> np.ndarray:
    """basis: (K, n, 3); deg: (n,) -> x: (n, 8)."""
    b0, b1, b2 = basis
    s = np.mean(np.linalg.norm(b1, axis=1))
    s = s if s > 0 else 1.0
    n0, n1, n2 = (np.linalg.norm(b, axis=1) / s for b in (b0, b1, b2))
    d01 = np.sum(b0 * b1, axis=1) / s ** 2
    d02 = np.sum(b0 * b2, axis=1) / s ** 2
    d12 = np.sum(b1 * b2, axis=1) / s ** 2
    return np.stack([n0, n1, n2, d01, d02, d12, deg / 6.0, np.ones_like(n0)], axis=1)


def _mean_agg(ptr, nbr, h):
    n = ptr.shape[0] - 1
    deg = np.diff(ptr)
    s = np.zeros_like(h)
    rows = np.repeat(np.arange(n), deg)
    np.add.at(s, rows, h[nbr])
    return s / np.maximum(deg, 1)[:, None], deg


def forward(params_flat: np.ndarray, basis: np.ndarray, ptr, nbr, cache: bool = False,
            round_bf16: bool = True):
    """v0 (n, 3) from FP32 master parameters (rounded to BF16 here unless
    round_bf16 is False, which finite-difference checks use)."""
    p = unpack(bf16_round(params_flat) if round_bf16 else np.asarray(params_flat, dtype=np.float64))
    deg = np.diff(ptr).astype(np.float64)
    x = features(basis, deg)
    z0 = x @ p["W_in"].T + p["b_in"]
    h = np.maximum(z0, 0.0)
    hs, zs, aggs = [h], [z0], []
    for l in range(3):
        a, _ = _mean_agg(ptr, nbr, h)
        u = np.concatenate([h, a], axis=1)
        z = u @ p[f"W{l}"].T + p[f"c{l}"]
        h = np.maximum(z, 0.0)
        aggs.append(a)
        zs.append(z)
        hs.append(h)
    c = h @ p["W_out"].T + p["b_out"]
    v0 = np.einsum("nk,knd->nd", c, basis)
    if cache:
        return v0, dict(p=p, x=x, hs=hs, zs=zs, aggs=aggs, c=c)
    return v0


def loss(v0: np.ndarray, target: np.ndarray, matvec=None) -> float:
    """The "l2" loss, or the "energy" loss when ``matvec`` (v -> Gamma v)
    is given."""
    e = v0 - target
    if matvec is None:
        return float(np.sum(e * e) / np.sum(target * target))
    return float(np.sum(e * matvec(e)) / np.sum(target * matvec(target)))


def mr_scale(v0: np.ndarray, F: np.ndarray, matvec) -> np.ndarray:
    """alpha v0 with the minimal-residual step alpha = (G v0)^T F / |G v0|^2
    (v0 unchanged when G v0 = 0)."""
    g = matvec(v0)
    den = float(np.sum(g * g))
    return v0 * (float(np.sum(g * F)) / den) if den > 0 else v0


def relu_ambiguous(params_flat, basis, ptr, nbr, rel: float = 2e-5, round_bf16: bool = True):
    """ReLU decisions that rounding may take either way: (layer, cell, unit)
    triples (layer 0 is the input layer, 1..3 the message-passing layers)
    whose pre-activation z lies within ``rel`` times its bound
    |W| |input| + |bias| of zero.  An evaluation in lower precision may put
    such a z on the other side of zero; its gradient then differs from this
    one by flipping those entries of the ReLU mask."""
    v0, C = forward(params_flat, basis, ptr, nbr, cache=True, round_bf16=round_bf16)
    p = C["p"]
    out = []
    ins = [C["x"]] + [np.concatenate([C["hs"][l], C["aggs"][l]], axis=1) for l in range(3)]
    Ws = [(p["W_in"], p["b_in"])] + [(p[f"W{l}"], p[f"c{l}"]) for l in range(3)]
    for layer, (u, (W, b)) in enumerate(zip(ins, Ws)):
        bound = np.abs(u) @ np.abs(W).T + np.abs(b)
        # an all-zero input row and bias give z = 0 exactly in any precision
        cells, units = np.nonzero((np.abs(C["zs"][layer]) <= rel * bound) & (bound > 0))
        out += [(layer, int(i), int(k)) for i, k in zip(cells, units)]
    return out


def backward(params_flat, basis, ptr, nbr, target, round_bf16: bool = True, matvec=None, flips=()):
    """(loss, gradient w.r.t. the (BF16-rounded) parameters, flat) of the
    "l2" loss, or of the "energy" loss when ``matvec`` is given.  ``flips``
    lists (layer, cell, unit) entries of the ReLU masks to invert (see
    ``relu_ambiguous``)."""
    v0, C = forward(params_flat, basis, ptr, nbr, cache=True, round_bf16=round_bf16)
    masks = [z > 0 for z in C["zs"]]
    for layer, i, k in flips:
        masks[layer][i, k] = not masks[layer][i, k]
    p = C["p"]
    e = v0 - target
    if matvec is None:
        nrm = np.sum(target ** 2)
        L = float(np.sum(e * e) / nrm)
        dv = 2.0 * e / nrm
    else:
        Ge = matvec(e)
        nrm = np.sum(target * matvec(target))
        L = float(np.sum(e * Ge) / nrm)
        dv = 2.0 * Ge / nrm
    dc = np.einsum("nd,knd->nk", dv, basis)
    g = {}
    g["W_out"] = dc.T @ C["hs"][3]
    g["b_out"] = dc.sum(axis=0)
    dh = dc @ p["W_out"]
    n = ptr.shape[0] - 1
    deg = np.diff(ptr)
    rows = np.repeat(np.arange(n), deg)
    for l in (2, 1, 0):
        dz = dh * masks[l + 1]
        u = np.concatenate([C["hs"][l], C["aggs"][l]], axis=1)
        g[f"W{l}"] = dz.T @ u
        g[f"c{l}"] = dz.sum(axis=0)
        du = dz @ p[f"W{l}"]
        dh_self, da = du[:, :H], du[:, H:]
        # a_i = mean_j h_j  ->  dh_j += sum_{i ~ j} da_i / deg_i
        w = da / np.maximum(deg, 1)[:, None]
        dh_nb = np.zeros_like(dh_self)
        np.add.at(dh_nb, nbr, w[rows])
        dh = dh_self + dh_nb
    dz0 = dh * masks[0]
    g["W_in"] = dz0.T @ C["x"]
    g["b_in"] = dz0.sum(axis=0)
    return L, pack(g)


def adam_step(params, grad, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (Kingma and Ba, 2015, Algorithm 1: bias-corrected
    first and second moment estimates).  t is the 1-based step count.
    Returns (params, m, v) as new arrays."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v
