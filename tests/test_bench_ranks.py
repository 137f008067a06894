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


@pytest.mark.parametrize("rank", [0, 1])
def test_reference_arm_contract(rank):
    """`--impl reference` times the CPU oracle on rank 0 only; other ranks exit 0 silently."""
    import json
    import subprocess
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--cpu-sample", "65536"], env=env, capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    if rank != 0:
        assert lines == []
        return
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GB/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["sample_rows"] == 4096
