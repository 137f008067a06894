"""GPU parity at the full workload sizes (properties that hold at any size plus oracle checks).

Large dominant workloads: n = 2^20 with kl = ku in {32, 128, 320}, p in {64, 148, 192},
dominance 1.01 / 1.5, nrhs in {1, 64}, N and T.  Pivoting workload: n = 262,144, kl = ku in
{16, 64}, nrhs = 8, p = 148, N(0,1) entries with the diagonal at 0.3 x the row's off-diagonal
absolute sum (sign kept).  Tolerances as in test_gpu_spike: backward error <= 1e-13, and
forward error <= 1e-9 against the manufactured solution on the dominant inputs.
"""
import numpy as np
import pytest

import oracle
from oracle import condest, metrics
from paper_1811_03559_gb300 import inputs, spike

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BERR = 1e-13
FERR_DD = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    spike.lib()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(pr, k, p, nrhs, pivot=0, **kw):
    band = pr["band"]
    bd = _dev(band)
    fac = spike.factor(bd, k, k, p, pivot, nrhs_hint=nrhs, **kw)
    out = {}
    for trans in ("N", "T"):
        F = inputs.band_matvec(band, k, k, pr["xstar"], trans)
        X = _dev(F)
        fac.solve(X, trans)
        be_gpu = spike.backward_error(bd, k, k, X, _dev(F), trans)
        out[trans] = (X.cpu().numpy(), F, be_gpu)
    return fac, out


@pytest.mark.parametrize("k,p,dd,nrhs", [(320, 148, 1.5, 1), (32, 192, 1.01, 64), (128, 64, 1.5, 1),
                                         (128, 192, 1.01, 1)])
def test_large_dominant(k, p, dd, nrhs):
    n = 1 << 20
    pr = inputs.make_problem(n, k, k, nrhs, seed=1, dd=dd)
    fac, out = _run(pr, k, p, nrhs)
    info = fac.info()
    assert info["boosts"] == 0 and info["p_effective"] == p
    for trans, (X, F, be_gpu) in out.items():
        assert be_gpu.max() <= BERR, (trans, be_gpu)
        assert metrics.backward_error(pr["band"], k, k, X, F, trans) <= BERR
        assert metrics.forward_error(X, pr["xstar"]) <= FERR_DD


def test_large_against_oracle_k32():
    """n = 2^20, k = 32: element-wise against the oracle's banded GEPP."""
    n, k, p = 1 << 20, 32, 148
    pr = inputs.make_problem(n, k, k, 2, seed=3, dd=1.01)
    fac, out = _run(pr, k, p, 2)
    for trans, (X, F, _) in out.items():
        xo, info = oracle.gbsv(pr["band"], k, k, F, trans)
        assert info == 0
        assert metrics.forward_error(X, xo) <= FERR_DD


@pytest.mark.parametrize("k", [16, 64])
def test_pivoting_workload(k):
    n, p, nrhs = 262_144, 148, 8
    seed = 2
    while True:  # regenerate until the oracle finds the matrix nonsingular
        pr = inputs.make_problem(n, k, k, nrhs, seed=seed, dist="normal", dd=0.3, keep_sign=True)
        if oracle.BandLU(pr["band"], k, k).info == 0:
            break
        seed += 1
    fac, out = _run(pr, k, p, nrhs, pivot=1)
    assert fac.status == 0 and fac.info()["zero_pivot_col"] == 0
    cond = condest.cond1_estimate(pr["band"], k, k)
    for trans, (X, F, be_gpu) in out.items():
        be = metrics.backward_error(pr["band"], k, k, X, F, trans)
        assert be <= BERR, (trans, be, cond)
        xo, _ = oracle.gbsv(pr["band"], k, k, F, trans)
        bo = metrics.backward_error(pr["band"], k, k, xo, F, trans)
        # forward error is governed by the conditioning: compare with the oracle's own
        assert metrics.forward_error(X, xo) <= max(1e-9, 1e3 * cond * max(be, bo)), (trans, cond)


@pytest.mark.parametrize("k,p,mixed", [(64, 152, False), (64, 148, True), (256, 148, False), (256, 152, True)])
def test_mixed_precision_workload(k, p, mixed):
    """n = 2^20, DD 1.05, k in {64, 256}, p = SM count (152) or 148, nrhs in {1, 32, 256}, N and T,
    FP64 and mixed (FP32 blocks + FP64 refinement): backward error <= 1e-13 and forward error
    <= 1e-9 against the manufactured solution, both evaluated on the device."""
    n, dd = 1 << 20, 1.05
    band, rng = inputs.make_band(n, k, k, seed=3, dd=dd)
    bd = _dev(band)
    fac = spike.factor(bd, k, k, p, 0, nrhs_hint=32, mixed=mixed, stage_balance=True)
    assert fac.info()["boosts"] == 0
    for m in (1, 32, 256):
        xs = torch.from_numpy(rng.uniform(-1.0, 1.0, size=(m, n))).cuda()
        for trans in ("N", "T"):
            F = inputs.band_matvec_torch(bd, k, k, xs, trans)
            X = F.clone()
            fac.solve(X, trans)
            be = spike.backward_error(bd, k, k, X, F, trans)
            assert be.max() <= BERR, (m, trans, be.max())
            fe = ((X - xs).abs().amax(dim=1) / xs.abs().amax(dim=1)).max().item()
            assert fe <= FERR_DD, (m, trans, fe)
            if mixed:
                assert fac.info()["refine_steps"] <= 4
    fac.free()


def test_pivoting_wide_interfaces():
    """k = 80 with pivoting on N(0,1) entries: interface blocks whose W tip has entries above 1
    take the full 2k x 2k LU (160 x 160, factored in global memory) while the others take the
    k x k Schur complement (in shared memory), often within one merge level."""
    n, k, p, nrhs = 40_000, 80, 8, 3
    seed = 5
    while True:
        pr = inputs.make_problem(n, k, k, nrhs, seed=seed, dist="normal", dd=0.3, keep_sign=True)
        if oracle.BandLU(pr["band"], k, k).info == 0:
            break
        seed += 1
    fac, out = _run(pr, k, p, nrhs, pivot=1)
    assert fac.status == 0
    for trans, (X, F, be_gpu) in out.items():
        be = metrics.backward_error(pr["band"], k, k, X, F, trans)
        assert be <= BERR, (trans, be)
