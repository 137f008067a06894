"""Partition-range sharding without a GPU: the ranks' ranges (spike_shard_plan, host logic)
and the exchange loop over torch.distributed with gloo, world size 2, on CPU.

The GPU arithmetic of each exchange step is covered by tests/test_gpu_shard.py (ranks of one
process on one GPU, against the oracle); here the loop and the collective are exercised with
an engine that follows the same protocol (pending / export / import) and checks that every
gathered buffer holds every rank's contribution in rank order.
"""
import os
import socket
import sys

import numpy as np
import pytest

from paper_1811_03559_gb300 import shard, spike

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    spike.lib()


@pytest.mark.parametrize("n,k,p,nranks", [(100_000, 8, 8, 2), (100_000, 8, 8, 8), (1 << 20, 128, 148, 4),
                                          (1 << 20, 128, 148, 128), (50_000, 4, 7, 2), (200_000, 16, 192, 16),
                                          (10_000, 3, 1, 1)])
def test_shard_ranges_follow_the_partitions(built, n, k, p, nranks):
    info, offs, flags = spike.plan(n, k, k, p)
    rows, leaves, ll = shard.plan(n, k, k, p, nranks)
    P, r = info["P"], info["r"]
    assert leaves[0] == 0 and leaves[-1] == info["leaves"] and np.all(np.diff(leaves) > 0)
    assert rows[0] == 0 and rows[-1] == n and np.all(rows[:-1] == offs[leaves[:-1]])
    # each rank holds P / nranks whole partitions: a 2x2 pair (flags bit 1 = top half) is never split
    for g in range(1, nranks):
        assert not (flags[leaves[g] - 1] & 2)
    per = P // nranks
    expect = (1 if r > 0 else 0) + int(np.log2(per))
    assert ll == expect and ll <= info["levels"]
    # the merges above the local levels join whole ranks: the top log2(nranks) levels
    assert info["levels"] - ll == int(np.log2(nranks))


@pytest.mark.parametrize("nranks", [0, 3, 6])
def test_shard_plan_rejects_rank_counts(built, nranks):
    with pytest.raises(spike.SpikeError) as e:
        shard.plan(100_000, 8, 8, 8, nranks)
    assert e.value.code == -5


def test_shard_plan_rejects_more_ranks_than_partitions(built):
    info, _, _ = spike.plan(100_000, 8, 8, 8)
    with pytest.raises(spike.SpikeError):
        shard.plan(100_000, 8, 8, 8, 2 * info["P"])


def test_band_columns_cover_the_couplings(built):
    n, kl, ku, p = 100_000, 5, 9, 8
    rows, _, _ = shard.plan(n, kl, ku, p, 4)
    for g in range(4):
        c0, c1 = shard.band_columns(n, kl, ku, rows, g)
        assert c0 == max(0, rows[g] - 9) and c1 == min(n, rows[g + 1] + 9)


class ScriptedEngine:
    """Follows the exchange protocol: `rounds` exchanges of growing size; each export carries
    (rank, round, index) codes, each import checks the gathered buffer."""

    def __init__(self, rank, world, rounds):
        import torch
        self.torch, self.rank, self.world, self.rounds, self.done = torch, rank, world, rounds, 0
        self.seen = []

    def pending(self):
        return 0 if self.done == self.rounds else 3 + 2 * self.done

    def _code(self, rank, count):
        return self.torch.tensor([1000.0 * rank + 10.0 * self.done + i for i in range(count)], dtype=self.torch.float64)

    def export(self, count):
        return self._code(self.rank, count)

    def import_(self, recv):
        count = self.pending()
        expect = self.torch.cat([self._code(g, count) for g in range(self.world)])
        assert self.torch.equal(recv, expect), (recv, expect)
        self.seen.append(count)
        self.done += 1


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
    from paper_1811_03559_gb300 import shard as sh
    eng = ScriptedEngine(rank, world, rounds=4)
    n = sh.exchange_loop(eng, sh.TorchCollective())
    q.put((rank, n, eng.seen))
    dist.barrier()
    dist.destroy_process_group()


def test_exchange_loop_over_gloo_two_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, n, seen in res:
        assert n == 4 and seen == [3, 5, 7, 9]


def test_exchange_loop_single_rank():
    eng = ScriptedEngine(0, 1, rounds=2)
    assert shard.exchange_loop(eng, lambda send: send.clone()) == 2
