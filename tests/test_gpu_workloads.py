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


def test_headline_shape_against_oracle():
    """The benchmarked shape: n = 2^20, k = 128, nrhs = 64, p = 148 with the benchmark's
    stage-balanced sizing, N and T, element-wise against the oracle's banded GEPP (one
    factorization reused for both, Sec. 4), plus the GPU backward error."""
    n, k, p, m = 1 << 20, 128, 148, 64
    pr = inputs.make_problem(n, k, k, m, seed=1, dd=1.01)
    bd = _dev(pr["band"])
    fac = spike.factor(bd, k, k, p, nrhs_hint=m, stage_balance=True)
    assert fac.info()["boosts"] == 0 and fac.info()["leaves"] == 148
    lu = oracle.BandLU(pr["band"], k, k)
    assert lu.info == 0
    xs = _dev(pr["xstar"])
    for trans in ("N", "T"):
        Fd = inputs.band_matvec_torch(bd, k, k, xs, trans)
        X = Fd.clone()
        fac.solve(X, trans)
        be_gpu = spike.backward_error(bd, k, k, X, Fd, trans)
        assert be_gpu.max() <= BERR, (trans, be_gpu.max())
        xo = lu.solve(Fd.cpu().numpy(), trans)
        fe = metrics.forward_error(X.cpu().numpy(), xo)
        assert fe <= FERR_DD, (trans, fe)
    fac.free()


CONFIG1 = [(k, p, dd) for k in (32, 128, 320) for p in (64, 148, 192) for dd in (1.01, 1.5)]


@pytest.mark.parametrize("k,p,dd", CONFIG1)
def test_large_dominant_grid(k, p, dd):
    """Every point of the large dominant workload: n = 2^20, k in {32, 128, 320}, p in
    {64, 148, 192}, DD in {1.01, 1.5}; one factorization per point, solved with nrhs = 1 and
    64, N and T.  Inputs are drawn on the device (the same recipe as make_band, torch's
    generator); checks: GPU backward error <= 1e-13 and forward error <= 1e-9 against the
    manufactured solution."""
    n = 1 << 20
    bd = inputs.make_band_torch(n, k, k, seed=11 + k + p, dd=dd, device="cuda")
    fac = spike.factor(bd, k, k, p, nrhs_hint=64)
    info = fac.info()
    assert info["boosts"] == 0 and info["p_effective"] == p
    g = torch.Generator(device="cuda")
    g.manual_seed(k * 1000 + p)
    for m in (1, 64):
        xs = torch.rand((m, n), generator=g, dtype=torch.float64, device="cuda") * 2.0 - 1.0
        for trans in ("N", "T"):
            F = inputs.band_matvec_torch(bd, k, k, xs, trans)
            X = F.clone()
            fac.solve(X, trans)
            be = spike.backward_error(bd, k, k, X, F, trans)
            assert be.max() <= BERR, (m, trans, be.max())
            fe = ((X - xs).abs().amax(dim=1) / xs.abs().amax(dim=1)).max().item()
            assert fe <= FERR_DD, (m, trans, fe)
    fac.free()
    del bd
    torch.cuda.empty_cache()


def transpose_band(band, kl, ku):
    """Band of A^T: A(i, j) = band[j, ku + i - j] goes to A^T(j, i) = bt[i, kl + j - i]."""
    n = band.shape[0]
    bt = np.zeros((n, kl + ku + 1))
    for d in range(kl + ku + 1):
        off = d - ku  # band[j, d] = A(j + off, j) -> bt[j + off, kl - off]
        j0, j1 = max(0, -off), min(n, n - off)
        bt[j0 + off:j1 + off, kl - off] = band[j0:j1, d]
    return bt


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
    # Forward error bound.  A backward error eta = ||r|| / (||op(A)|| ||x||) means x solves
    # (op(A) + dA) x = f with ||dA|| = eta ||op(A)|| (dA = r x^T-shaped, infinity norms), so
    # ||x - x_true|| / ||x_true|| <= kappa eta / (1 - kappa eta) with kappa the infinity-norm
    # condition number of op(A): kappa_inf(A) = kappa_1(A^T) for N, kappa_1(A) for T.  Between the
    # GPU result and the oracle's (backward errors be, bo) the triangle inequality gives
    # ~kappa (be + bo).  kappa comes from Hager's estimator, a lower bound that is rarely off by
    # more than a factor 3; the bound below allows 10, and a factor 2 for the first-order terms.
    conds = {"N": condest.cond1_estimate(transpose_band(pr["band"], k, k), k, k),
             "T": condest.cond1_estimate(pr["band"], k, k)}
    for trans, (X, F, be_gpu) in out.items():
        be = metrics.backward_error(pr["band"], k, k, X, F, trans)
        assert be <= BERR, (trans, be, conds[trans])
        xo, _ = oracle.gbsv(pr["band"], k, k, F, trans)
        bo = metrics.backward_error(pr["band"], k, k, xo, F, trans)
        fe = metrics.forward_error(X, xo)
        bound = 20.0 * conds[trans] * (be + bo)
        assert fe <= max(1e-9, bound), (trans, fe, bound, conds[trans], be, bo)


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
