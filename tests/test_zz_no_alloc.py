"""sgp_spmv_dot_noalloc: the product with Gamma and v^T Gamma v for callers
that cannot allocate device memory while they run (inside a stream capture,
under an application-owned memory pool, or in loops that cannot take the
synchronisation of cudaMalloc/cudaFree).

Called directly through the C ABI and checked against the regular
sgp_spmv entry point, twice in a row (the fixed scratch array is shared
between calls and keeps the previous call's contents), inside a CUDA graph
captured on the context's stream (replayed twice, device memory unchanged),
plus the size limit of that array.  This file is collected last so that a run stopping at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2410_04512_gb300 as sgp
import workloads
from gpu_common import GpuSystem, dev_tensor

pytestmark = pytest.mark.gpu

MAX_CELLS = 4096 * 256


def _noalloc(ctx, M, v, y, dot):
    lib = sgp.load_library()
    return lib.sgp_spmv_dot_noalloc(ctx.ptr, M.ptr, ctypes.c_void_p(v.data_ptr()),
                                    ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(dot.data_ptr()))


def test_noalloc_matches_spmv_twice_in_a_row(cuda_device):
    ctx = sgp.Context(0)
    for k, cells in enumerate([workloads.ball(n=20000, seed=2002, gamma0=1e-3),
                               workloads.cube(n=1000, side=8.886, seed=1000)]):
        s = GpuSystem(ctx, cells, tree=False)
        for call in range(2):
            v = dev_tensor(np.random.default_rng(10 * k + call).standard_normal((cells.n, 3)))
            y = torch.full_like(v, float("nan"))
            dot = torch.full((1,), float("nan"), dtype=torch.float64, device=v.device)
            assert _noalloc(ctx, s.M, v, y, dot) == sgp.OK
            want = ctx.spmv(s.M, v)
            torch.cuda.synchronize()
            scale = want.abs().max().item()
            assert (y - want).abs().max().item() <= 1e-13 * scale
            ref = torch.dot(v.ravel(), want.ravel()).item()
            assert abs(dot.item() - ref) <= 1e-13 * abs(ref)


def test_noalloc_inside_a_stream_capture(cuda_device):
    """The first call on a fresh context is made inside the capture: the
    scratch address was looked up when the context was created."""
    cells = workloads.ball(n=20000, seed=2005, gamma0=1e-3)
    side = torch.cuda.Stream()
    ctx0 = sgp.Context(0)
    s = GpuSystem(ctx0, cells, tree=False)
    v = dev_tensor(np.random.default_rng(3).standard_normal((cells.n, 3)))
    y = torch.zeros_like(v)
    dot = torch.zeros((1,), dtype=torch.float64, device=v.device)
    want = ctx0.spmv(s.M, v)
    ref = torch.dot(v.ravel(), want.ravel()).item()
    torch.cuda.synchronize()
    ctx = sgp.Context(0, side)
    g = torch.cuda.CUDAGraph()
    # an allocation call inside the capture would fail the capture (and the
    # call's status); the replays then must not allocate either
    with torch.cuda.stream(side):
        g.capture_begin()
        rc = _noalloc(ctx, s.M, v, y, dot)
        g.capture_end()
    assert rc == sgp.OK
    scale = want.abs().max().item()
    free = []
    for _ in range(3):
        y.fill_(float("nan"))
        dot.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert (y - want).abs().max().item() <= 1e-13 * scale
        assert abs(dot.item() - ref) <= 1e-13 * abs(ref)
    assert free[0] == free[1] == free[2]


def test_noalloc_rejects_more_cells_than_its_scratch(cuda_device):
    ctx = sgp.Context(0)
    n = MAX_CELLS + 1
    pos = np.zeros((n, 3))
    pos[:, 0] = 3.0 * np.arange(n)          # far apart: no contacts
    cells = workloads.Cells("line", pos, np.full(n, 0.5), 1, 0.1, 10.0, 1e-2)
    s = GpuSystem(ctx, cells, tree=False)
    assert s.M.m == 0
    v = torch.ones((n, 3), dtype=torch.float64, device="cuda")
    y = torch.empty_like(v)
    dot = torch.empty((1,), dtype=torch.float64, device="cuda")
    rc = _noalloc(ctx, s.M, v, y, dot)
    assert rc == sgp.ERR_INVALID_ARG
    assert b"scratch limit" in sgp.load_library().sgp_last_error(ctx.ptr)
