"""Host-side logic of bench.py's multi-GPU path (one independent replica per
rank, max-over-ranks timing), run as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = 1.5 + rank                  # rank 1 is the slow one
        m = bench.max_over_ranks(elapsed)
        out[rank] = (bench.replica_seed(rank), m, bench.replica_throughput(world, 10, m))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] != res[1][0]                      # independent replicas
    assert res[0][1] == res[1][1] == 2.5               # every rank sees the max
    assert res[0][2] == pytest.approx(2 * 10 / 2.5)    # whole-job throughput


def test_single_process_is_the_identity():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.replica_throughput(1, 4, 2.0) == 2.0
