"""Mixed precision (SPIKE_FLAG_MIXED): FP32 block factorizations and sweeps, FP64 reduced system,
FP64 iterative refinement.  Every result must meet the FP64 bar: backward error <= 1e-13 and, on
dominant inputs, forward error <= 1e-9 against the oracle."""
import numpy as np
import pytest

import oracle
from oracle import metrics
from paper_1811_03559_gb300 import inputs, spike

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    spike.lib()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("p", [1, 2, 5, 9])
@pytest.mark.parametrize("trans", ["N", "T"])
def test_mixed_small(p, trans):
    n, k = 20_000, 8
    pr = inputs.make_problem(n, k, k, 3, seed=40 + p, dd=1.1, trans=trans)
    fac = spike.factor(_dev(pr["band"]), k, k, p, mixed=True)
    X = _dev(pr["F"])
    fac.solve(X, trans)
    Xh = X.cpu().numpy()
    info = fac.info()
    assert info["mixed"] == 1 and 1 <= info["refine_steps"] <= 10
    assert info["refine_berr"] <= spike.MIXED_TOL
    assert metrics.backward_error(pr["band"], k, k, Xh, pr["F"], trans) <= 1e-13
    xo, _ = oracle.gbsv(pr["band"], k, k, pr["F"], trans)
    assert metrics.forward_error(Xh, xo) <= 1e-9


@pytest.mark.parametrize("k,p,nrhs", [(32, 148, 8), (128, 148, 64)])
def test_mixed_large(k, p, nrhs):
    n = 1 << 20
    pr = inputs.make_problem(n, k, k, nrhs, seed=3, dd=1.05)
    bd = _dev(pr["band"])
    fac = spike.factor(bd, k, k, p, nrhs_hint=nrhs, mixed=True, stage_balance=True)
    for trans in ("N", "T"):
        F = inputs.band_matvec(pr["band"], k, k, pr["xstar"], trans)
        X = _dev(F)
        fac.solve(X, trans)
        be = spike.backward_error(bd, k, k, X, _dev(F), trans)
        assert be.max() <= 1e-13, be.max()
        assert fac.info()["refine_steps"] <= 6
        assert metrics.forward_error(X.cpu().numpy(), pr["xstar"]) <= 1e-9


def test_mixed_host_pointers_and_reuse():
    pr = inputs.make_problem(9000, 6, 6, 2, seed=7, dd=1.2)
    fac = spike.factor(np.ascontiguousarray(pr["band"]), 6, 6, 4, mixed=True)
    for trans in ("N", "T", "N"):
        F = inputs.band_matvec(pr["band"], 6, 6, pr["xstar"], trans)
        X = F.copy()
        fac.solve(X, trans)
        assert metrics.backward_error(pr["band"], 6, 6, X, F, trans) <= 1e-13


def test_mixed_with_pivoting_is_not_supported():
    band, _ = inputs.make_band(500, 2, 2, seed=1, dd=1.2)
    with pytest.raises(spike.SpikeError) as e:
        spike.factor(_dev(band), 2, 2, 2, pivot=1, mixed=True)
    assert e.value.code == spike.SPIKE_ENOTSUP


def test_mixed_borrowed_band_matches_copy():
    """SPIKE_FLAG_BORROW_BAND: the handle reads the caller's device band for its residuals
    instead of a copy -- same bits, 8 n (kl+ku+1) fewer resident bytes."""
    n, k, p = 50_000, 24, 12
    pr = inputs.make_problem(n, k, k, 3, seed=8, dd=1.05)
    bd = torch.from_numpy(pr["band"]).cuda()
    a = spike.factor(bd, k, k, p, mixed=True)
    lent = bd.clone()
    b = spike.factor(lent, k, k, p, mixed=True, borrow_band=True)
    del lent  # the Factorization keeps the borrowed tensor alive until free()
    assert a.info()["device_bytes"] - b.info()["device_bytes"] >= 8 * n * (2 * k + 1)
    res_a, _ = spike.factor_bytes(n, k, k, p, mixed=True)
    res_b, _ = spike.factor_bytes(n, k, k, p, mixed=True, borrow_band=True)
    assert res_a - res_b >= 8 * n * (2 * k + 1)
    for trans in ("N", "T"):
        F = inputs.band_matvec(pr["band"], k, k, pr["xstar"], trans)
        Xa, Xb = torch.from_numpy(F).cuda(), torch.from_numpy(F).cuda()
        a.solve(Xa, trans)
        b.solve(Xb, trans)
        assert torch.equal(Xa, Xb)
        assert metrics.backward_error(pr["band"], k, k, Xb.cpu().numpy(), F, trans) <= 1e-13
    assert b._borrowed is not None
    b.free()
    assert b._borrowed is None
