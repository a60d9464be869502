"""Parity of the warm-start network's CUDA kernels (called through the C ABI)
with the CPU oracle: forward pass, loss and gradients for both losses, Adam,
the minimal-residual scaling and the acceptance test; then online training
on a short time-stepping sequence, evaluated by the solver itself.

Tolerances.  Both sides use the same BF16 weights (round-to-nearest-even of
the same FP32 values).  The GPU keeps activations in FP32 with FP32
accumulation: a 128-term FP32 dot product is within ~128 u32 (u32 = 6e-8)
of its value relative to the sum of |terms|, and five layers compound that
to a few 1e-5 at most; 2e-4 relative (max norm) is used.  Weight gradients
are FP32 sums over every cell (per block of 256 cells, then over blocks);
1e-3 relative per parameter tensor in the 2-norm.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2410_04512_gb300 as sgp
import workloads
from gpu_common import GpuSystem, dev_tensor, oracle_system, rel_err, small_cube
from oracle import mpnn

pytestmark = pytest.mark.gpu

H = mpnn.H
OFF_WOUT = mpnn.N_PARAMS - 3 - 3 * H


@pytest.fixture(scope="module")
def ctx(cuda_device):
    return sgp.Context(0)


def head_params(seed, b_out=(0.3, 0.8, 0.2), w_scale=30.0):
    """Initial weights with an output head strong enough for every hidden
    layer to matter."""
    p = workloads.mpnn_init(seed)
    p[OFF_WOUT:-3] *= w_scale
    p[-3:] = b_out
    return p


class Case:
    def __init__(self, ctx, cells, seed=0):
        self.cells = cells
        self.gs = GpuSystem(ctx, cells)
        s = oracle_system(cells)
        self.s = s
        n = cells.n
        self.fac = oracle.tree_ldlt(oracle.prim_msf(n, s.ij, s.w), s.blocks, s.gamma0)
        Dinv = oracle.block_jacobi(n, s.ij, s.blocks, s.gamma0)
        self.F = cells.forces(seed)
        self.vprev = 0.5 * cells.forces(seed + 1)
        self.basis = np.stack([np.einsum("nij,nj->ni", Dinv, self.F), oracle.tree_solve(self.fac, self.F),
                               self.vprev])
        self.ptr, self.nbr = mpnn.adjacency(n, s.ij)
        self.mv = lambda x: oracle.matvec(n, s.ij, s.blocks, s.gamma0, x)
        self.F_d, self.vprev_d = dev_tensor(self.F), dev_tensor(self.vprev)


def cases():
    return [
        small_cube(1000, seed=1000),                          # 4 dense-layer passes of 256 + ragged tail
        workloads.ball(n=3000, seed=2000, gamma0=1e-3),       # 3000 = 11 x 256 + 184
        small_cube(700, seed=1002, side=14.0),                # sparse: many isolated cells
    ]


@pytest.fixture(scope="module", params=range(3))
def case(request, ctx):
    return Case(ctx, cases()[request.param])


def test_forward_matches_oracle(ctx, case):
    p = head_params(21)
    net = ctx.mpnn_create(p)
    v0 = ctx.mpnn_forward(net, case.gs.M, case.gs.Fac, case.F_d, case.vprev_d).cpu().numpy()
    want = mpnn.forward(p.astype(np.float64), case.basis, case.ptr, case.nbr)
    scale = np.abs(want).max()
    assert np.abs(v0 - want).max() <= 2e-4 * scale, rel_err(v0, want)
    if case.cells.n == 700:
        assert np.sum(np.diff(case.ptr) == 0) > 50      # the isolated-cell case is exercised


def test_forward_without_previous_velocity(ctx, case):
    p = head_params(22)
    net = ctx.mpnn_create(p)
    v0 = ctx.mpnn_forward(net, case.gs.M, case.gs.Fac, case.F_d, None).cpu().numpy()
    basis = case.basis.copy()
    basis[2] = 0.0
    want = mpnn.forward(p.astype(np.float64), basis, case.ptr, case.nbr)
    assert np.abs(v0 - want).max() <= 2e-4 * np.abs(want).max()


def _blocks(g):
    out, o = {}, 0
    for name, shp in mpnn.SHAPES:
        k = int(np.prod(shp))
        out[name] = g[o:o + k]
        o += k
    return out


@pytest.mark.parametrize("energy", [False, True])
def test_gradients_match_oracle(ctx, case, energy):
    p = head_params(23)
    net = ctx.mpnn_create(p)
    target = case.cells.forces(7) * 3.0
    ctx.mpnn_forward(net, case.gs.M, case.gs.Fac, case.F_d, case.vprev_d)
    kind = sgp.MPNN_LOSS_ENERGY if energy else sgp.MPNN_LOSS_L2
    L = ctx.mpnn_backward(net, dev_tensor(target), kind)
    _, g = net.params()
    mv = case.mv if energy else None
    p64 = p.astype(np.float64)
    # ReLU decisions within FP32 rounding of zero may go either way on the
    # GPU: any choice of those masks gives a valid gradient.  Start from the
    # oracle's own masks and flip ambiguous entries one at a time while that
    # brings the oracle closer (only needed when the plain comparison fails).
    amb = mpnn.relu_ambiguous(p64, case.basis, case.ptr, case.nbr)
    assert len(amb) <= 1e-3 * 4 * H * case.cells.n, len(amb)
    got = _blocks(g.astype(np.float64))

    def worst(flips):
        L_or, g_or = mpnn.backward(p64, case.basis, case.ptr, case.nbr, target, matvec=mv, flips=flips)
        want = _blocks(g_or)
        return max(rel_err(got[name], want[name]) for name in want), L_or

    best, L_or = worst([])
    flips = []
    for _ in range(3):
        if best <= 1e-3:
            break
        for a in amb:
            trial = [f for f in flips if f != a] if a in flips else flips + [a]
            e, _ = worst(trial)
            if e < best:
                best, flips = e, trial
    assert abs(L - L_or) <= 1e-5 * abs(L_or)
    assert best <= 1e-3, (best, len(amb), len(flips))
    # flips stay the exception: a handful of units at a kink, not a drift of
    # the FP32 forward pass (run with -s to see the counts)
    print("relu units within rounding of a kink: %d; flipped to match: %d" % (len(amb), len(flips)))
    assert len(flips) <= max(4, len(amb) // 10), (len(amb), len(flips))


def test_backward_is_bitwise_reproducible(ctx, case):
    p = head_params(24)
    net = ctx.mpnn_create(p)
    target = dev_tensor(case.cells.forces(8))
    ctx.mpnn_forward(net, case.gs.M, case.gs.Fac, case.F_d, case.vprev_d)
    ctx.mpnn_backward(net, target, sgp.MPNN_LOSS_ENERGY)
    _, g1 = net.params()
    ctx.mpnn_forward(net, case.gs.M, case.gs.Fac, case.F_d, case.vprev_d)
    ctx.mpnn_backward(net, target, sgp.MPNN_LOSS_ENERGY)
    _, g2 = net.params()
    assert np.array_equal(g1.view(np.uint32), g2.view(np.uint32))


def test_adam_step_matches_oracle(ctx, case):
    p = head_params(25)
    net = ctx.mpnn_create(p)
    target = case.cells.forces(9)
    ctx.mpnn_forward(net, case.gs.M, case.gs.Fac, case.F_d, case.vprev_d)
    ctx.mpnn_backward(net, dev_tensor(target), sgp.MPNN_LOSS_L2)
    lr = 1e-2
    ctx.mpnn_step(net, lr)
    got, _ = net.params()
    _, g_or = mpnn.backward(p.astype(np.float64), case.basis, case.ptr, case.nbr, target)
    want, _, _ = mpnn.adam_step(p.astype(np.float64), g_or, 0.0, 0.0, 1, lr)
    step = got.astype(np.float64) - p
    # every first step has length <= lr; where the gradient is well resolved
    # both sides take the same signed step
    assert np.all(np.abs(step) <= lr + 1e-6)
    big = np.abs(g_or) > 0.1 * np.sqrt(np.mean(g_or ** 2))
    assert big.sum() > 0.1 * big.size
    off = np.abs(got[big] - want[big]) > 1e-6 + 1e-4 * lr
    # a ReLU decision taken the other way near zero (see the gradient test)
    # may flip the sign of a handful of entries
    assert off.sum() <= max(2, 0.002 * big.sum()), off.sum()


def test_warm_start_rejects_a_worse_guess(ctx, case):
    # W_out = 0, b_out = (1e3, 0, 0): v0 = 1e3 D^-1 F, whose residual is far
    # above |F|, so the zero guess must be returned
    p = workloads.mpnn_init(26)
    p[OFF_WOUT:-3] = 0.0
    p[-3:] = (1e3, 0.0, 0.0)
    net = ctx.mpnn_create(p)
    v0, used = ctx.warm_start(net, case.gs.M, case.gs.Fac, case.F_d, case.vprev_d)
    r = case.F - case.mv(1e3 * case.basis[0])
    assert np.linalg.norm(r) > np.linalg.norm(case.F)
    assert not used and torch.count_nonzero(v0).item() == 0


def test_warm_start_keeps_a_better_guess(ctx, case):
    # W_out = 0, b_out = (0, 0, 1) returns v_prev exactly; with v_prev = v*/2
    # the residual is |F|/2
    res, _ = oracle.solve_system(case.s, case.F, 1e-12)
    half = 0.5 * res.x
    p = workloads.mpnn_init(27)
    p[OFF_WOUT:-3] = 0.0
    p[-3:] = (0.0, 0.0, 1.0)
    net = ctx.mpnn_create(p)
    v0, used = ctx.warm_start(net, case.gs.M, case.gs.Fac, case.F_d, dev_tensor(half))
    assert used
    assert np.array_equal(v0.cpu().numpy(), half)


def test_minimal_residual_scaling(ctx, case):
    p = head_params(28)
    net = ctx.mpnn_create(p)
    v0, used = ctx.warm_start(net, case.gs.M, case.gs.Fac, case.F_d, case.vprev_d, mr_scale=True)
    raw = mpnn.forward(p.astype(np.float64), case.basis, case.ptr, case.nbr)
    want = mpnn.mr_scale(raw, case.F, case.mv)
    assert used                       # the scaled guess never has a larger residual
    got = v0.cpu().numpy()
    assert np.abs(got - want).max() <= 2e-4 * np.abs(want).max()
    assert np.linalg.norm(case.F - case.mv(got)) <= np.linalg.norm(case.F) * (1 + 1e-9)


def test_bad_arguments_are_rejected(ctx):
    with pytest.raises(sgp.SgpError):
        ctx.mpnn_create(np.zeros(10, dtype=np.float32))
    c = small_cube(200, seed=5)
    gs = GpuSystem(ctx, c)
    net = ctx.mpnn_create(workloads.mpnn_init(1))
    F = dev_tensor(c.forces(0))
    ctx.mpnn_forward(net, gs.M, gs.Fac, F)
    with pytest.raises(sgp.SgpError):
        ctx.mpnn_backward(net, F, 7)
    with pytest.raises(sgp.SgpError):
        ctx.mpnn_step(net, 0.0)


# ---------------------------------------------------------- online training
def _sequence(ctx, n=4000, train_steps=16, test_steps=6, epochs=8, lr=2e-3):
    """Time stepping x <- x + v dt with overlap springs and fresh active
    noise; the network is trained on the solver's solutions of the first
    steps and evaluated on the rest by the iterations of PCG to 1e-8."""
    c = workloads.ball(n=n, seed=2100, gamma0=1e-3)
    pos = dev_tensor(c.pos)
    radii = dev_tensor(c.radii)
    tp, tq = (dev_tensor(t) for t in c.tables())
    net = ctx.mpnn_create(workloads.mpnn_init(5000))
    vprev = None
    G = M = T = Fh = None
    rows = []
    for step in range(1, train_steps + test_steps + 1):
        G = ctx.collision_graph(pos, radii, G)
        ij = G.edges()
        gp, gq = workloads.pair_gamma_torch(c.seed, ij, tp, tq)
        M = ctx.friction_assemble(G, pos, gp.contiguous(), gq.contiguous(), c.gamma0, sgp.PREC_F64, M)
        T = ctx.max_spanning_tree(M, T)
        Fh = ctx.tree_factor(M, T, Fh)
        F = (workloads.spring_forces_torch(pos, radii, ij) + dev_tensor(workloads.active_noise(2100, step, n)))
        F = F.contiguous()
        vstar, inf0 = ctx.pcg_solve(M, Fh, F, tol=1e-8)
        if step <= train_steps:
            for _ in range(epochs):
                ctx.mpnn_forward(net, M, Fh, F, vprev)
                ctx.mpnn_backward(net, vstar, sgp.MPNN_LOSS_ENERGY)
                ctx.mpnn_step(net, lr)
        else:
            v0 = ctx.mpnn_forward(net, M, Fh, F, vprev)
            e = v0 - vstar
            E = float(torch.sum(e * ctx.spmv(M, e.contiguous())) / torch.sum(vstar * F))
            vw, used = ctx.warm_start(net, M, Fh, F, vprev, mr_scale=True)
            _, infw = ctx.pcg_solve(M, Fh, F, vw.clone(), tol=1e-8, x0_given=True)
            rows.append((E, used, inf0.iterations, infw.iterations, infw.true_rel_residual))
        vprev = vstar
        pos = (pos + 0.01 * vstar).contiguous()
    return rows


def test_online_training_gains(ctx):
    rows = _sequence(ctx)
    E = np.array([r[0] for r in rows])
    it0 = np.array([r[2] for r in rows])
    itw = np.array([r[3] for r in rows])
    # the zero guess has energy-norm error 1 by definition; the trained
    # network starts the solve well inside it
    assert np.median(E) < 0.85, E
    assert all(r[1] for r in rows)
    # the solve from the warm start reaches the same tolerance ...
    assert max(r[4] for r in rows) <= 1.5e-8
    # ... in no more iterations than from zero on average
    assert itw.mean() <= it0.mean() + 0.5, (itw, it0)
