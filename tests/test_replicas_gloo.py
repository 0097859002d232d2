"""Multi-GPU runs are independent replicas (no collective on the data path):
the only cross-rank step is the timing reduction of bench.py, which takes the
slowest rank's time and counts every rank's pairs.  Checked with two gloo
ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        own_ms = [400.0, 250.0][rank]          # rank 0 is the slowest replica
        value, ms = bench.aggregate_over_ranks(own_ms, 100, world, dist, "cpu")
        q.put((rank, value, ms))
    finally:
        dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms in out:
        assert ms == 400.0
        assert value == pytest.approx(2 * 100 / 0.4)


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.aggregate_over_ranks(500.0, 1000, 1)
    assert ms == 500.0 and value == pytest.approx(2000.0)
