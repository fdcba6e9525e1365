"""The benchmark's multi-rank path on CPU: two gloo ranks, each timing its own
replica, reduce to the slowest rank's time, and rank 0 reports the aggregate
rate of both replicas (no data-path collective: replicas are independent)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = 0.010 * (rank + 1)          # rank 1 is the slower replica
    t = bench.max_over_ranks(dist, local, "cpu")
    rate = bench.aggregate_rate(1000, 3, world, t)
    dist.barrier()
    out.put((rank, t, rate))
    dist.destroy_process_group()


def test_two_rank_replica_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate in res:
        assert t == pytest.approx(0.020)           # every rank sees the slowest time
        assert rate == pytest.approx(1000 * 3 * 2 / 0.020)


def test_single_rank_helpers():
    import bench
    assert bench.max_over_ranks(None, 0.5, "cpu") == 0.5
    assert bench.aggregate_rate(512, 3, 1, 0.5) == pytest.approx(3072.0)
