"""The multi-process path of bench.py, on CPU with gloo and two ranks.

Ranks process independent environments (weak scaling, no collective on the
data path); the only collectives are the timing reductions, checked here:
the reported duration is the slowest rank's and the value counts every rank's
environments."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.dist


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    ms = bench.max_over_ranks(local_ms, dist)
    e2e = bench.min_over_ranks(1000.0 - rank, dist)
    value = bench.weak_scaling_value(16384, 10, ms, world)
    out[rank] = (ms, e2e, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_reduction():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, e2e, value = res[rank]
        assert ms == 150.0
        assert e2e == 999.0
        assert value == pytest.approx(world * 16384 * 10 / 0.150)


def test_single_process_reductions_are_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.min_over_ranks(2.0) == 2.0
    assert bench.weak_scaling_value(100, 2, 1000.0, 1) == 200.0
