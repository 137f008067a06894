"""Multi-process (gloo, world size 2, CPU) test of bench.py's rank aggregation: the timed
region is the maximum over ranks and the whole-job throughput sums the replicas' bytes."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value, w = bench.aggregate_over_ranks(100.0 + 50.0 * rank, 1e9 * (rank + 1), 4, dist, "cpu")
    q.put((rank, ms, value, w))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms, value, w in res:
        assert w == 2
        assert ms == 150.0                      # max over ranks
        assert value == pytest.approx(3e9 * 4 / 0.150 / 1e9)  # summed bytes / max time


def test_single_process_aggregation():
    sys.path.insert(0, ROOT)
    import bench
    ms, value, w = bench.aggregate_over_ranks(200.0, 2e9, 5)
    assert (ms, w) == (200.0, 1) and value == pytest.approx(2e9 * 5 / 0.2 / 1e9)
