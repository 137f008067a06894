"""Partition-range sharding on the GPU: the ranks of one system run in one process on one GPU
(each with its own handle, its own rows and its own band columns), exchanging through
shard.run_local (an all-gather by concatenation; every import starts after every export has
completed, so no kernel waits on another).  Checks: every rank's rows of X against the
oracle's banded GEPP (forward error <= 1e-9 on these dominant inputs) and the whole X against
the backward-error bar 1e-13 and the single-process solve of the same plan; the number of
exchanges (log2(ranks) per factorization, log2(ranks) + 1 per solve)."""
import numpy as np
import pytest

import oracle
from oracle import metrics
from paper_1811_03559_gb300 import inputs, shard, spike

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    spike.lib()


def _ranks(band, n, kl, ku, p, nranks, **kw):
    rows, leaves, ll = shard.plan(n, kl, ku, p, nranks, **kw)
    engines = []
    for g in range(nranks):
        c0, c1 = shard.band_columns(n, kl, ku, rows, g)
        cols = torch.from_numpy(np.ascontiguousarray(band[c0:c1])).cuda()
        engines.append(shard.ShardEngine(cols, c0, n, kl, ku, p, g, nranks, **kw))
        del cols  # read during the factorization only
    return engines, rows, ll


def _solve(engines, rows, F, trans):
    parts = []
    for g, e in enumerate(engines):
        part = torch.from_numpy(np.ascontiguousarray(F[:, rows[g]:rows[g + 1]])).cuda()
        e.start_solve(part, trans)
        parts.append(part)
    rounds = shard.run_local(engines)
    torch.cuda.synchronize()
    return np.concatenate([p.cpu().numpy() for p in parts], axis=1), rounds


@pytest.mark.parametrize("n,kl,ku,p,nranks,nrhs", [(40_000, 8, 8, 8, 2, 3), (60_000, 16, 12, 12, 4, 5),
                                                   (50_000, 6, 9, 7, 2, 1), (120_000, 24, 24, 32, 8, 16),
                                                   (30_000, 5, 5, 4, 4, 2), (20_000, 4, 4, 6, 1, 2)])
def test_sharded_solve_matches_oracle(n, kl, ku, p, nranks, nrhs):
    pr = inputs.make_problem(n, kl, ku, nrhs, seed=600 + n % 97, dd=1.05)
    band = pr["band"]
    engines, rows, ll = _ranks(band, n, kl, ku, p, nranks)
    rounds = shard.run_local(engines)
    assert rounds == int(np.log2(nranks))
    info = spike.plan(n, kl, ku, p)[0]
    assert all(e.info()["boosts"] == 0 for e in engines)
    single = spike.factor(torch.from_numpy(band).cuda(), kl, ku, p)
    lu = oracle.BandLU(band, kl, ku)
    for trans in ("N", "T"):
        F = inputs.band_matvec(band, kl, ku, pr["xstar"], trans)
        X, rounds = _solve(engines, rows, F, trans)
        assert rounds == (int(np.log2(nranks)) + 1 if nranks > 1 else 0)
        xo = lu.solve(F, trans)
        assert metrics.backward_error(band, kl, ku, X, F, trans) <= 1e-13, trans
        assert metrics.forward_error(X, xo) <= 1e-9, trans
        Xs = torch.from_numpy(F).cuda()
        single.solve(Xs, trans)
        assert metrics.forward_error(X, Xs.cpu().numpy()) <= 1e-12, trans
    assert info["levels"] - ll == int(np.log2(nranks))
    for e in engines:
        e.free()
    single.free()


def test_sharded_headline_like_shape():
    """n = 2^18, k = 128, p = 148 split over 4 ranks (32 partitions each, 2x2 pairs inside),
    nrhs = 8, N and T, against the oracle."""
    n, k, p, nranks, m = 1 << 18, 128, 148, 4, 8
    pr = inputs.make_problem(n, k, k, m, seed=5, dd=1.01)
    band = pr["band"]
    engines, rows, ll = _ranks(band, n, k, k, p, nranks, nrhs_hint=m, stage_balance=True)
    shard.run_local(engines)
    lu = oracle.BandLU(band, k, k)
    for trans in ("N", "T"):
        F = inputs.band_matvec(band, k, k, pr["xstar"], trans)
        X, _ = _solve(engines, rows, F, trans)
        assert metrics.backward_error(band, k, k, X, F, trans) <= 1e-13
        assert metrics.forward_error(X, lu.solve(F, trans)) <= 1e-9
    for e in engines:
        e.free()


def test_shard_protocol_errors():
    n, k, p = 20_000, 4, 8
    pr = inputs.make_problem(n, k, k, 1, seed=9, dd=1.1)
    engines, rows, _ = _ranks(pr["band"], n, k, k, p, 2)
    # a solve before the factorization's exchanges are done is refused
    with pytest.raises(spike.SpikeError) as e:
        engines[0].start_solve(torch.zeros(rows[1] - rows[0], dtype=torch.float64, device="cuda"))
    assert e.value.code == spike.SPIKE_ENOTSUP
    shard.run_local(engines)
    # the single-system solve entry point refuses a rank's handle
    X = torch.zeros(n, dtype=torch.float64, device="cuda")
    assert spike.lib().spike_solve_ex(engines[0]._h, spike._ptr(X), n, 1, b"N") == spike.SPIKE_ENOTSUP
    for eng in engines:
        eng.free()
