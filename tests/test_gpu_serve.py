"""The serving engine on the GPU: solves against the oracle, the alone-vs-in-mix
equality of a request's result, eviction and re-factorization, byte accounting."""
import numpy as np
import pytest

import oracle
from oracle import metrics
from paper_1811_03559_gb300 import inputs, serve, spike

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BERR = 1e-13
FERR_DD = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    spike.lib()


# matrices: (n, k, dd, dist, pivot)
CAT = [(3000, 4, 1.1, "uniform", 0), (20_000, 32, 1.1, "uniform", 0), (9000, 64, 1.05, "uniform", 0),
       (12_000, 8, 0.4, "normal", 1), (1000, 12, 1.1, "uniform", 0)]


def _catalogue():
    bands = []
    for i, (n, k, dd, dist, piv) in enumerate(CAT):
        seed = 100 + i
        while True:
            band, _ = inputs.make_band(n, k, k, seed=seed, dist=dist, dd=dd, keep_sign=(dist == "normal"))
            if not piv or oracle.BandLU(band, k, k).info == 0:
                break
            seed += 1
        bands.append(band)
    return bands


@pytest.fixture(scope="module")
def cat():
    return _catalogue()


def _check(band, k, F, X, trans, dd_ok):
    assert metrics.backward_error(band, k, k, X, F, trans) <= BERR
    if dd_ok:
        xo, info = oracle.gbsv(band, k, k, F, trans)
        assert info == 0
        assert metrics.forward_error(X, xo) <= FERR_DD


def test_served_solves_match_oracle(cat):
    rng = np.random.default_rng(7)
    with serve.Server(8 << 30, streams=3, max_batch_rhs=24) as S:
        for i, band in enumerate(cat):
            S.add_matrix(i, band, CAT[i][1], CAT[i][1], pivot=CAT[i][4])
        reqs = []
        for j in range(60):
            i = int(rng.integers(len(cat)))
            n, k, _, _, piv = CAT[i]
            F = rng.uniform(-1, 1, size=(int(rng.integers(1, 9)), n))
            mixed = bool(rng.integers(2)) and not piv
            trans = "T" if rng.random() < 0.3 else "N"
            rid, X = S.submit(i, F, trans=trans, mixed=mixed)
            reqs.append((rid, i, F, X, trans))
        for rid, i, F, X, trans in reqs:
            S.wait(rid)
            _check(cat[i], CAT[i][1], F, X, trans, dd_ok=not CAT[i][4])
        st = S.stats()
        assert st["completed"] == 60 and st["failed"] == 0
        assert st["batches"] <= 60


@pytest.mark.parametrize("trans,mixed,fp64_residual", [("N", False, False), ("T", False, False), ("N", True, False),
                                                       ("T", True, False), ("N", True, True), ("T", True, True)])
def test_alone_equals_in_mix(cat, trans, mixed, fp64_residual):
    """A request served alone and the same request served inside a burst (merged with other
    requests on its matrix, other matrices solving concurrently) return the same bits, with the
    mixed-precision refinement residuals on the tensor cores or (fp64_residual) on FP64 FMAs."""
    i = 1
    n, k = CAT[i][0], CAT[i][1]
    rng = np.random.default_rng(17)
    F = rng.uniform(-1, 1, size=(3, n))
    with serve.Server(8 << 30, streams=1, max_batch_rhs=64, fp64_residual=fp64_residual) as S:
        for j, band in enumerate(cat):
            S.add_matrix(j, band, CAT[j][1], CAT[j][1], pivot=CAT[j][4])
        rid, X_alone = S.submit(i, F, trans=trans, mixed=mixed)
        S.wait(rid)
        assert S.stats()["max_batch"] == 1
        # burst: a slow head-of-line request keeps the worker busy while the rest queue
        head, _ = S.submit(2, rng.uniform(-1, 1, size=(32, CAT[2][0])))
        ids = []
        for r in range(6):
            G = rng.uniform(-1, 1, size=(int(rng.integers(1, 6)), n))
            ids.append(S.submit(i, G, trans=trans, mixed=mixed)[0])
            if r == 2:
                rid_mix, X_mix = S.submit(i, F, trans=trans, mixed=mixed)
            ids.append(S.submit(0, rng.uniform(-1, 1, size=(2, CAT[0][0])))[0])
        for r in [head, rid_mix] + ids:
            S.wait(r)
        assert S.stats()["max_batch"] >= 3  # the copy of F was merged with others
    assert np.array_equal(X_alone, X_mix)


def test_eviction_refactors_identically():
    """Four equal matrices, budget for two resident factorizations plus one being factored:
    round-robin requests evict and re-factor; every result is still right, and
    re-factoring reproduces the same bits."""
    n, k = 20_000, 32
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    p = min(max(4, 2 * sms // 1), max(1, n // (16 * k)))  # the engine's rule for one stream
    res, tr = spike.factor_bytes(n, k, k, p, 0, host_band=True, nrhs_hint=16, stage_balance=True)
    reserve, keep = res + tr + (1 << 20), res + (2 << 20)
    budget = reserve + keep + (8 << 20)  # + workspace and batch buffer for 2 columns
    assert res > (8 << 20)  # so a third factorization never fits beside two
    bands = [inputs.make_band(n, k, k, seed=200 + i, dd=1.1)[0] for i in range(4)]
    rng = np.random.default_rng(3)
    Fs = [rng.uniform(-1, 1, size=(2, n)) for _ in range(4)]
    with serve.Server(budget, streams=1, max_batch_rhs=8) as S:
        for i in range(4):
            S.add_matrix(i, bands[i], k, k)
        first = {}
        for rnd in range(3):
            for i in range(4):
                rid, X = S.submit(i, Fs[i])
                S.wait(rid)
                if rnd == 0:
                    first[i] = X
                    _check(bands[i], k, Fs[i], X, "N", True)
                else:
                    assert np.array_equal(X, first[i])
        st = S.stats()
        assert st["factorizations"] == 12 and st["evictions"] == 10, st
        assert st["peak_bytes"] <= budget


def test_device_catalogue_and_device_rhs(cat):
    i = 2
    n, k = CAT[i][0], CAT[i][1]
    bd = torch.from_numpy(cat[i]).cuda()
    F = torch.from_numpy(np.random.default_rng(1).uniform(-1, 1, size=(4, n))).cuda()
    with serve.Server(4 << 30, streams=2) as S:
        S.add_matrix(9, bd, k, k)
        rid, X = S.submit(9, F, trans="T")
        S.wait(rid)
    _check(cat[i], k, F.cpu().numpy(), X.cpu().numpy(), "T", True)


@pytest.mark.parametrize("mixed", [False, True])
def test_factor_bytes_and_workspace_solve(cat, mixed):
    i = 1
    n, k = CAT[i][0], CAT[i][1]
    p = 9
    res, tr = spike.factor_bytes(n, k, k, p, 0, mixed=mixed)
    fac = spike.factor(torch.from_numpy(cat[i]).cuda(), k, k, p, 0, mixed=mixed)
    dev = fac.info()["device_bytes"]
    assert res <= dev <= res + (2 << 20)  # plus the descriptor buffer
    F = np.random.default_rng(2).uniform(-1, 1, size=(5, n))
    X1 = torch.from_numpy(F).cuda()
    fac.solve(X1, "N")
    ws = torch.empty(fac.workspace_bytes(5, "N"), dtype=torch.uint8, device="cuda")
    X2 = torch.from_numpy(F).cuda()
    fac.solve_ws(X2, ws, "N")
    torch.cuda.synchronize()
    assert torch.equal(X1, X2)
    fac.free()


def test_graph_buckets_replay_and_keep_results(cat):
    """SPIKE_SERVE_GRAPHS: FP64 solves run as power-of-two column buckets from captured graphs;
    every result equals the plain server's bit for bit (zero padding columns do not change the
    others on batch-invariant handles; replays are the direct launches)."""
    rng = np.random.default_rng(21)
    jobs = [(i, int(rng.integers(1, 12)), "NT"[int(rng.integers(0, 2))]) for i in (0, 1, 2, 4) for _ in range(6)]
    Fs = [rng.uniform(-1, 1, size=(m, CAT[i][0])) for i, m, _ in jobs]
    outs = {}
    for graphs in (False, True):
        res = []
        with serve.Server(8 << 30, streams=1, max_batch_rhs=16, graphs=graphs) as S:
            for i, band in enumerate(cat):
                if not CAT[i][4]:
                    S.add_matrix(i, band, CAT[i][1], CAT[i][1])
            for (i, m, tr), F in zip(jobs, Fs):  # one at a time: the same merges in both servers
                rid, X = S.submit(i, F, trans=tr)
                S.wait(rid)
                res.append(X.copy())
            st = S.stats()
        outs[graphs] = (res, st)
    for a, b in zip(outs[False][0], outs[True][0]):
        assert np.array_equal(a, b)
    assert outs[True][1]["graph_replays"] > 0 and outs[False][1]["graph_replays"] == 0
    for (i, m, tr), F, X in zip(jobs, Fs, outs[True][0]):
        _check(cat[i], CAT[i][1], F, X, tr, True)


def test_tuned_worker_counts(cat):
    """SPIKE_SERVE_TUNED: the first factorization of each size class runs spike_tune and later
    ones reuse its worker count; served results still match the oracle."""
    rng = np.random.default_rng(22)
    bands = {0: cat[1], 1: inputs.make_band(21_000, 32, 32, seed=77, dd=1.1)[0]}  # one size class
    with serve.Server(8 << 30, streams=2, max_batch_rhs=16, tuned=True, nrhs_hint=4) as S:
        for i, b in bands.items():
            S.add_matrix(i, torch.from_numpy(b).cuda(), 32, 32)
        reqs = []
        for i in (0, 1, 0, 1):
            F = rng.uniform(-1, 1, size=(3, bands[i].shape[0]))
            rid, X = S.submit(i, F, trans="N", mixed=bool(i))
            reqs.append((rid, i, F, X))
        for rid, i, F, X in reqs:
            S.wait(rid)
            _check(bands[i], 32, F, X, "N", True)
        assert S.stats()["tuned_classes"] == 1
