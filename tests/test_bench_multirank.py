"""The N > 1 bench path on CPU: two gloo ranks, max-over-ranks timing and the whole-job
throughput of independent replicas (weak scaling)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [2.0, 3.5][rank]
    got = bench.max_over_ranks(ms, dist, "cpu")
    v = bench.job_throughput(world, 128 ** 4, 10, got / 1e3)
    q.put((rank, got, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, v in res:
        assert got == 3.5
        assert abs(v - 2 * 128 ** 4 * 10 / 3.5e-3) < 1e-6 * v


def test_single_rank_identity():
    import bench
    assert bench.max_over_ranks(1.25, None, "cpu") == 1.25
    assert bench.job_throughput(1, 100, 4, 2.0) == 200.0
