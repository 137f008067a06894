"""Host logic of the serving engine, run in its scheduler-only mode (no GPU).

In SPIKE_SERVE_DRYRUN a "factorization" holds the bytes spike_factor_bytes predicts
and a "solve" copies F to X after a configurable sleep, so admission, LRU eviction,
request merging, budget accounting and latency statistics are checked here on the
CPU; the GPU tests run the same engine on real factorizations.
"""
import math
import time

import numpy as np
import pytest

from paper_1811_03559_gb300 import serve, spike


def _band(n, k, seed=0):
    rng = np.random.default_rng(seed)
    b = rng.uniform(-1, 1, size=(n, 2 * k + 1))
    b[:, k] = 10.0
    return b


def _reserve(n, k, p, mixed=False):
    """Bytes the engine reserves to factor (n, k) from a host band, and keeps afterwards."""
    res, tr = spike.factor_bytes(n, k, k, p, 0, mixed=mixed, host_band=True, nrhs_hint=16, stage_balance=True)
    return res + tr + (1 << 20), res + (1 << 20)


def test_roundtrip_and_counters():
    with serve.Server(1 << 30, streams=2, max_batch_rhs=16, dryrun=True) as S:
        for mid in range(3):
            S.add_matrix(mid, _band(1000 + 100 * mid, 4), 4, 4)
        rng = np.random.default_rng(1)
        reqs = []
        for i in range(30):
            mid = i % 3
            F = rng.standard_normal((1 + i % 4, 1000 + 100 * mid))
            rid, X = S.submit(mid, F, trans="NT"[i % 2], mixed=bool(i % 5 == 0))
            reqs.append((rid, F, X))
        for rid, F, X in reqs:
            assert S.wait(rid) >= 0.0
            assert np.array_equal(X, F)
        st = S.stats()
        assert st["submitted"] == st["completed"] == 30 and st["failed"] == 0
        assert st["rhs"] == sum(F.shape[0] for _, F, _ in reqs)
        # each (matrix, precision) is factored once and stays resident
        keys = {(i % 3, i % 5 == 0) for i in range(30)}
        assert st["factorizations"] == len(keys) == st["resident"]
        assert st["evictions"] == 0


def test_waiting_requests_are_merged_per_key():
    """One worker busy on matrix 1; meanwhile N and T requests for matrix 0 queue up.
    The N ones are merged into one solve, the T ones into another."""
    with serve.Server(1 << 30, streams=1, max_batch_rhs=64, dryrun=True, dryrun_solve_us=200_000) as S:
        S.add_matrix(0, _band(500, 3), 3, 3)
        S.add_matrix(1, _band(500, 3), 3, 3)
        F = np.ones((1, 500))
        r_busy, _ = S.submit(1, F)
        time.sleep(0.05)  # the worker has taken it and is "solving"
        ids = [S.submit(0, F, trans=t)[0] for t in "NTNTN"]
        for r in [r_busy] + ids:
            S.wait(r)
        st = S.stats()
        assert st["batches"] == 3
        assert st["max_batch"] == 3


def test_batch_column_cap():
    with serve.Server(1 << 30, streams=1, max_batch_rhs=7, dryrun=True, dryrun_solve_us=100_000) as S:
        S.add_matrix(0, _band(400, 2), 2, 2)
        S.add_matrix(1, _band(400, 2), 2, 2)
        r_busy, _ = S.submit(1, np.ones((1, 400)))
        time.sleep(0.05)
        ids = [S.submit(0, np.ones((3, 400)))[0] for _ in range(5)]  # 15 columns
        for r in [r_busy] + ids:
            S.wait(r)
        st = S.stats()
        # 3 + 3 fit under 7 columns, a third would not: batches of 2, 2, 1
        assert st["batches"] == 1 + 3 and st["max_batch"] == 2


def test_lru_eviction_order_and_budget():
    n, k, p = 4000, 4, 8
    reserve, keep = _reserve(n, k, p)
    ws = 24 * n  # dry-run workspace + merged right-hand sides for one column
    budget = 2 * keep + (reserve - keep) + ws + keep // 2  # room for two resident, not three
    with serve.Server(budget, streams=1, max_batch_rhs=4, p=p, dryrun=True) as S:
        for mid in "ABC":
            S.add_matrix(ord(mid), _band(n, k), k, k)
        F = np.ones((1, n))

        def run(mid):
            S.wait(S.submit(ord(mid), F)[0])
            return S.stats()

        run("A"), run("B"), run("A")
        st = run("C")  # B is the least recently used: evicted
        assert (st["factorizations"], st["evictions"]) == (3, 1)
        st = run("A")  # still resident
        assert st["factorizations"] == 3
        st = run("B")  # C is now the least recently used
        assert (st["factorizations"], st["evictions"]) == (4, 2)
        assert st["peak_bytes"] <= budget
        assert st["resident"] == 2


def test_budget_holds_under_concurrency():
    n, k = 3000, 6
    reserve, keep = _reserve(n, k, 6)
    budget = 3 * reserve + 4 * 24 * 3000 * 8
    with serve.Server(budget, streams=4, max_batch_rhs=8, p=6, dryrun=True, dryrun_factor_us=2000,
                      dryrun_solve_us=500) as S:
        for mid in range(12):
            S.add_matrix(mid, _band(n, k), k, k)
        rng = np.random.default_rng(3)
        ids = []
        for i in range(300):
            mid = int(rng.zipf(1.3)) % 12
            rid, X = S.submit(mid, rng.standard_normal((int(rng.integers(1, 8)), n)))
            ids.append(rid)
        S.drain()
        st = S.stats()
        assert st["completed"] == 300 and st["failed"] == 0
        assert st["peak_bytes"] <= budget
        assert st["evictions"] > 0
        assert st["factorizations"] == st["evictions"] + st["resident"]


def test_request_larger_than_budget_fails_cleanly():
    n, k = 20_000, 16
    reserve, _ = _reserve(n, k, 10)
    with serve.Server(reserve // 2, streams=2, p=10, dryrun=True) as S:
        S.add_matrix(0, _band(n, k), k, k)
        S.add_matrix(1, _band(500, 2), 2, 2)
        rid, _ = S.submit(0, np.ones((1, n)))
        with pytest.raises(spike.SpikeError) as e:
            S.wait(rid)
        assert e.value.code == spike.SPIKE_ENOMEM
        rid2, X = S.submit(1, np.full((1, 500), 2.0))  # the server keeps serving
        S.wait(rid2)
        assert np.all(X == 2.0)
        st = S.stats()
        assert st["failed"] == 1 and st["completed"] == 1


def test_argument_errors():
    with serve.Server(1 << 28, dryrun=True) as S:
        S.add_matrix(5, _band(300, 2), 2, 2, pivot=1)
        with pytest.raises(spike.SpikeError) as e:
            S.add_matrix(5, _band(300, 2), 2, 2)
        assert e.value.code == -2
        with pytest.raises(spike.SpikeError) as e:
            S.submit(5, np.ones((1, 300)), mixed=True)  # mixed needs a non-pivoting factorization
        assert e.value.code == spike.SPIKE_ENOTSUP
        with pytest.raises(KeyError):
            S.submit(6, np.ones((1, 300)))
        with pytest.raises(spike.SpikeError):
            S.submit(5, np.ones((1, 300)), trans="X")
    with pytest.raises(spike.SpikeError):
        serve.Server(0, dryrun=True)


def test_latency_statistics_are_nearest_rank():
    with serve.Server(1 << 30, streams=3, dryrun=True, dryrun_solve_us=300) as S:
        for mid in range(4):
            S.add_matrix(mid, _band(256, 2), 2, 2)
        for i in range(101):
            S.submit(i % 4, np.ones((1, 256)))
            if i % 10 == 0:
                time.sleep(0.002)
        S.drain()
        st = S.stats()
        lat = np.sort(S.latencies())
        assert len(lat) == 101
        rank = lambda q: lat[max(1, math.ceil(q * len(lat))) - 1]
        assert st["p50_ms"] == rank(0.5) and st["p99_ms"] == rank(0.99) and st["max_ms"] == lat[-1]
        assert st["mean_ms"] == pytest.approx(lat.mean())
        assert st["solves_per_s"] == pytest.approx(101 / st["span_s"])


def test_workers_run_concurrently():
    solve_us = 150_000
    with serve.Server(1 << 30, streams=4, dryrun=True, dryrun_solve_us=solve_us) as S:
        for mid in range(4):
            S.add_matrix(mid, _band(256, 2), 2, 2)
        t0 = time.perf_counter()
        ids = [S.submit(mid, np.ones((1, 256)))[0] for mid in range(4)]
        for r in ids:
            S.wait(r)
        dt = time.perf_counter() - t0
        assert dt < 3.5 * solve_us * 1e-6  # four solves overlapped, not serialised (4x)


def test_request_latency_query_does_not_block():
    with serve.Server(1 << 30, streams=1, dryrun=True, dryrun_solve_us=150_000) as S:
        S.add_matrix(0, _band(300, 2), 2, 2)
        rid, _ = S.submit(0, np.ones((1, 300)))
        t0 = time.perf_counter()
        assert S.latency(rid) is None  # still running
        assert time.perf_counter() - t0 < 0.05
        lat = S.wait(rid)
        assert S.latency(rid) == lat
        with pytest.raises(spike.SpikeError):
            S.latency(12345)


def test_resident_fp64_requests_of_several_matrices_share_a_solve():
    """With factorizations resident, waiting FP64 requests of the same trans on different
    matrices are solved together (one spike_solve_batch); mixed-precision ones and the
    other trans are not merged with them."""
    with serve.Server(1 << 30, streams=1, max_batch_rhs=64, dryrun=True, dryrun_solve_us=150_000,
                      batch_systems=16) as S:
        for mid in range(6):
            S.add_matrix(mid, _band(400, 2), 2, 2)
        for mid in range(5):  # factor (and keep) matrices 0..4
            S.wait(S.submit(mid, np.ones((1, 400)))[0])
        base = S.stats()
        busy, _ = S.submit(5, np.ones((1, 400)))  # keeps the single worker busy
        time.sleep(0.05)
        ids = [S.submit(mid, np.full((2, 400), float(mid)))[0] for mid in range(4)]    # FP64 N on 0..3
        ids.append(S.submit(4, np.ones((1, 400)), mixed=True)[0])                     # mixed: own solve
        ids.append(S.submit(0, np.ones((1, 400)), trans="T")[0])                      # T: own solve
        for r in [busy] + ids:
            S.wait(r)
        st = S.stats()
        assert st["batches"] - base["batches"] == 1 + 1 + 1 + 1  # busy, 4-matrix N solve, mixed, T
        assert st["multi_solves"] == 1 and st["max_systems"] == 4
    with serve.Server(1 << 30, streams=1, dryrun=True, dryrun_solve_us=100_000, batch_systems=1) as S:
        for mid in range(3):
            S.add_matrix(mid, _band(300, 2), 2, 2)
            S.wait(S.submit(mid, np.ones((1, 300)))[0])
        busy, _ = S.submit(2, np.ones((1, 300)))
        time.sleep(0.05)
        ids = [S.submit(mid, np.ones((1, 300)))[0] for mid in range(2)]
        for r in [busy] + ids:
            S.wait(r)
        assert S.stats()["multi_solves"] == 0


def test_drain_releases_request_buffers_and_shapes_are_checked():
    with serve.Server(1 << 30, streams=2, dryrun=True, dryrun_solve_us=1000) as S:
        S.add_matrix(0, _band(300, 2), 2, 2)
        for _ in range(20):
            S.submit(0, np.ones((2, 300)))
        S.drain()
        assert [key for key in S._keep if not isinstance(key, tuple)] == []
        assert S.stats()["completed"] == 20
        with pytest.raises(ValueError):
            S.submit(0, np.ones((2, 299)))
        with pytest.raises(ValueError):
            S.submit(0, np.ones((2, 300)), X=np.empty((1, 300)))


@pytest.mark.parametrize("evict,refactored", [("lru", True), ("cost", False)])
def test_cost_aware_eviction_keeps_the_frequently_used(evict, refactored):
    """Room for two of three equal factorizations: A serves three requests, B one, then C
    arrives.  LRU evicts A (used least recently); the greedy-dual size-frequency policy evicts B
    (one use against three), so a later request on A needs no new factorization."""
    n, k, p = 4000, 4, 8
    reserve, keep = _reserve(n, k, p)
    budget = 2 * keep + (reserve - keep) + 24 * n + keep // 2
    with serve.Server(budget, streams=1, max_batch_rhs=4, p=p, dryrun=True, dryrun_factor_us=20_000,
                      evict=evict) as S:
        for mid in "ABC":
            S.add_matrix(ord(mid), _band(n, k), k, k)
        F = np.ones((1, n))
        for mid in "AAABC":
            S.wait(S.submit(ord(mid), F)[0])
        before = S.stats()
        assert (before["factorizations"], before["evictions"]) == (3, 1)
        S.wait(S.submit(ord("A"), F)[0])
        assert (S.stats()["factorizations"] > before["factorizations"]) == refactored
        assert S.stats()["peak_bytes"] <= budget


@pytest.mark.parametrize("evict,refactored", [("lru", True), ("cost", False)])
def test_cost_aware_eviction_prefers_large_factorizations(evict, refactored):
    """Equal uses and build times: the greedy-dual priority is use x time / bytes, so the larger
    factorization leaves first and the small, older one stays (LRU evicts the older one)."""
    k, p = 4, 8
    rs, ks_ = _reserve(4000, k, p)
    rb, kb = _reserve(8000, k, p)
    budget = ks_ + kb + 24 * 8000 + (rs - ks_) + ks_ // 2
    with serve.Server(budget, streams=1, max_batch_rhs=4, p=p, dryrun=True, dryrun_factor_us=20_000,
                      evict=evict) as S:
        S.add_matrix(1, _band(4000, k), k, k)
        S.add_matrix(2, _band(8000, k), k, k)
        S.add_matrix(3, _band(4000, k, seed=1), k, k)
        for mid, n in ((1, 4000), (2, 8000), (3, 4000)):
            S.wait(S.submit(mid, np.ones((1, n)))[0])
        before = S.stats()
        assert (before["factorizations"], before["evictions"]) == (3, 1)
        S.wait(S.submit(1, np.ones((1, 4000)))[0])
        assert (S.stats()["factorizations"] > before["factorizations"]) == refactored
        assert S.stats()["peak_bytes"] <= budget


def test_unknown_eviction_policy_is_refused():
    with pytest.raises(KeyError):
        serve.Server(1 << 28, dryrun=True, evict="random")
    cfg = serve.ServerConfig(budget_bytes=1 << 28, streams=1, max_batch_rhs=4, flags=serve.DRYRUN, evict_policy=7)
    h = serve.ctypes.c_void_p()
    assert serve._lib().spike_server_create(serve.ctypes.byref(cfg), serve.ctypes.byref(h)) == -1


@pytest.mark.parametrize("fp64_residual", [True, False])
def test_fp64_residual_mixed_handles_fit_a_smaller_budget(fp64_residual):
    """SPIKE_SERVE_FP64_RESIDUAL: a mixed-precision factorization is reserved without the digit planes
    of the tensor-core residual.  A budget between the two sizes admits it with the option and refuses
    it (SPIKE_ENOMEM) without."""
    n, k, p = 20_000, 64, 8
    kw = dict(mixed=True, host_band=True, nrhs_hint=16, stage_balance=True)
    small = sum(spike.factor_bytes(n, k, k, p, 0, fp64_residual=True, **kw))
    large = sum(spike.factor_bytes(n, k, k, p, 0, fp64_residual=False, **kw))
    budget = small + (8 << 20)
    assert budget < large
    with serve.Server(budget, streams=1, p=p, dryrun=True, fp64_residual=fp64_residual) as S:
        S.add_matrix(0, _band(n, k), k, k)
        rid, X = S.submit(0, np.ones((1, n)), mixed=True)
        if fp64_residual:
            S.wait(rid)
            st = S.stats()
            assert st["factorizations"] == 1 and st["failed"] == 0 and st["peak_bytes"] <= budget
        else:
            with pytest.raises(spike.SpikeError) as e:
                S.wait(rid)
            assert e.value.code == spike.SPIKE_ENOMEM
