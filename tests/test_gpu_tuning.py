"""The autotuner and the tuning knobs: every candidate is a valid launch
shape, so the solution must not depend on the choice (beyond rounding), and
the chosen values come from the documented candidate sets."""
import numpy as np
import pytest

import oracle
import paper_2410_04512_gb300 as sgp
import workloads
from gpu_common import GpuSystem, dev_tensor, oracle_system, rel_err, small_cube

pytestmark = pytest.mark.gpu


@pytest.fixture()
def ctx(cuda_device):
    return sgp.Context(0)


def test_set_tuning_validates(ctx):
    for bad in (dict(spmv_lpr=3), dict(tail_cap=-2), dict(batch_chunk=100), dict(batch_chunk=70000),
                dict(spmv_ilp=3), dict(bin_cap=32), dict(bin_cap=-2), dict(bin_cap=9000)):
        with pytest.raises(sgp.SgpError):
            ctx.set_tuning(**bad)
    ctx.set_tuning(spmv_lpr=4, tail_cap=512, batch_chunk=1024, spmv_ilp=2, bin_cap=512)
    assert ctx.get_tuning() == {"spmv_lpr": 4, "tail_cap": 512, "batch_chunk": 1024, "spmv_ilp": 2,
                                "bin_cap": 512, "ms_per_iteration": 0.0}
    ctx.set_tuning(bin_cap=-1)
    assert ctx.get_tuning()["bin_cap"] == -1
    ctx.set_tuning()
    assert ctx.get_tuning()["bin_cap"] == 0


@pytest.mark.parametrize("cap,bins", [(0, -1), (64, -1), (256, -1), (-1, -1), (1024, -1), (1024, 0), (-1, 0),
                                      (1024, 512), (256, 2048), (0, 1024)])
@pytest.mark.parametrize("prec", [sgp.PREC_F64, sgp.PREC_MIXED])
def test_contraction_granularity_does_not_change_the_solution(ctx, cap, bins, prec):
    c = workloads.ball(n=20000, seed=2002, gamma0=1e-3)
    ctx.set_tuning(tail_cap=cap, bin_cap=bins)
    s = GpuSystem(ctx, c, precision=prec)
    F = c.forces()
    v, info = ctx.pcg_solve(s.M, s.Fac, dev_tensor(F), tol=1e-10, precision=prec)
    # the recursive residual meets tol; the true one differs from it by
    # rounding (about eps kappa(Gamma), 1e-13 here)
    assert info.status == 0 and info.true_rel_residual <= 1.05e-10
    ctx.set_tuning(tail_cap=-1)
    ref = GpuSystem(ctx, c, precision=sgp.PREC_F64)
    vr, _ = ctx.pcg_solve(ref.M, ref.Fac, dev_tensor(F), tol=1e-12)
    assert rel_err(v.cpu().numpy(), vr.cpu().numpy()) <= 1e-8


@pytest.mark.parametrize("ilp", [1, 2])
@pytest.mark.parametrize("lpr", [1, 2, 4, 8])
def test_lanes_per_row_do_not_change_the_solution(ctx, lpr, ilp):
    c = small_cube(3000, seed=1003)
    s = GpuSystem(ctx, c)
    o = oracle_system(c)
    F = c.forces()
    ctx.set_tuning(spmv_lpr=lpr, spmv_ilp=ilp)
    v, info = ctx.pcg_solve(s.M, s.Fac, dev_tensor(F), tol=1e-12)
    ref, _ = oracle.solve_system(o, F, tol=1e-13)
    assert rel_err(v.cpu().numpy(), ref.x) <= 1e-9


def test_autotune_single_system(ctx):
    c = workloads.ball(n=30000, seed=2003, gamma0=1e-3)
    s = GpuSystem(ctx, c, precision=sgp.PREC_MIXED)
    F = dev_tensor(c.forces())
    t = ctx.autotune(s.M, s.T, s.Fac, F, precision=sgp.PREC_MIXED, iterations=20)
    assert t["tail_cap"] in (0, 256, 512, 1024, 2048, 4096, -1)
    assert t["bin_cap"] in (0, -1, 512, 1024, 2048)
    assert t["spmv_lpr"] in (1, 2, 4, 8) and t["spmv_ilp"] in (1, 2)
    assert t["ms_per_iteration"] > 0
    assert ctx.get_tuning()["tail_cap"] == t["tail_cap"]
    # the factor handle was left built with the chosen tail and still solves
    v, info = ctx.pcg_solve(s.M, s.Fac, F, tol=1e-8, precision=sgp.PREC_MIXED)
    assert info.status == 0 and info.true_rel_residual <= 1e-8
    # whole-step objective (factor build + solve to the tolerance)
    t2 = ctx.autotune(s.M, s.T, s.Fac, F, precision=sgp.PREC_MIXED, iterations=0, tol=1e-8)
    assert t2["ms_per_iteration"] > t["ms_per_iteration"]
    v, info = ctx.pcg_solve(s.M, s.Fac, F, tol=1e-8, precision=sgp.PREC_MIXED)
    assert info.status == 0 and info.true_rel_residual <= 1e-8


def test_autotune_batch(ctx):
    sizes = np.array([1500, 800, 3000, 200, 2500, 1200])
    off = workloads.sphere_offsets(sizes)
    cells = [workloads.batch_instance(int(n), s) for s, n in enumerate(sizes)]
    pos = dev_tensor(np.concatenate([c.pos for c in cells]))
    radii = dev_tensor(np.concatenate([c.radii for c in cells]))
    g = ctx.collision_graph_batched(off, pos, radii)
    tab = dev_tensor(workloads.gamma_table(0.1, 10.0))
    gp, gq = workloads.pair_gamma_torch(4000, g.edges(), tab, tab)
    M = ctx.friction_assemble(g, pos, gp.contiguous(), gq.contiguous(), 1e-2, sgp.PREC_F64)
    T = ctx.max_spanning_tree(M)
    Fh = ctx.tree_factor(M, T)
    F = dev_tensor(np.random.default_rng(0).standard_normal((int(off[-1]), 3)))
    v0, _ = ctx.pcg_solve_batched(M, Fh, off, F, tol=1e-10)
    t = ctx.autotune(M, T, Fh, F, offsets=off, iterations=10)
    assert t["batch_chunk"] in (512, 1024, 2048, 4096, 8192)
    assert t["spmv_lpr"] in (1, 2, 4)
    v1, infos = ctx.pcg_solve_batched(M, Fh, off, F, tol=1e-10)
    assert all(i.status == 0 for i in infos)
    assert rel_err(v1.cpu().numpy(), v0.cpu().numpy()) <= 1e-8


@pytest.mark.parametrize("prec", [sgp.PREC_F64, sgp.PREC_MIXED])
def test_device_loop_matches_chunk_graphs(ctx, prec):
    """The iterations run as a device-side loop (conditional WHILE graph node)
    unless per-kernel timing is on, which replays plain chunk graphs and
    polls between chunks.  Same kernels in the same order: the iterates and
    the iteration counts must agree bit for bit, single and batched."""
    c = workloads.ball(n=20000, seed=2003, gamma0=1e-3)
    s = GpuSystem(ctx, c, precision=prec)
    F = dev_tensor(c.forces())
    runs = []
    for timing in (False, True, False):
        ctx.set_kernel_timing(timing)
        v, info = ctx.pcg_solve(s.M, s.Fac, F, tol=1e-9, precision=prec)
        runs.append((v.cpu().numpy(), info.iterations, info.true_rel_residual))
    ctx.set_kernel_timing(False)
    for v, it, res in runs[1:]:
        np.testing.assert_array_equal(v, runs[0][0])
        assert it == runs[0][1] and res == runs[0][2]
    assert runs[0][2] <= 1e-9


def test_device_loop_matches_chunk_graphs_batched(ctx):
    sizes = [1500, 2600, 800, 3100]
    cells = [workloads.batch_instance(n, k) for k, n in enumerate(sizes)]
    off = workloads.sphere_offsets(np.array(sizes))
    pos = dev_tensor(np.concatenate([cl.pos for cl in cells]))
    radii = dev_tensor(np.concatenate([cl.radii for cl in cells]))
    g = ctx.collision_graph_batched(off, pos, radii)
    tab = dev_tensor(workloads.gamma_table(0.1, 10.0))
    gp, gq = workloads.pair_gamma_torch(4100, g.edges(), tab, tab)
    M = ctx.friction_assemble(g, pos, gp.contiguous(), gq.contiguous(), 1e-2, sgp.PREC_MIXED)
    Fh = ctx.tree_factor(M, ctx.max_spanning_tree(M))
    F = dev_tensor(np.random.default_rng(5).standard_normal((int(off[-1]), 3)))
    runs = []
    for timing in (False, True):
        ctx.set_kernel_timing(timing)
        v, infos = ctx.pcg_solve_batched(M, Fh, off, F, tol=1e-9, precision=sgp.PREC_MIXED)
        runs.append((v.cpu().numpy(), [i.iterations for i in infos]))
    ctx.set_kernel_timing(False)
    np.testing.assert_array_equal(runs[1][0], runs[0][0])
    assert runs[1][1] == runs[0][1]
