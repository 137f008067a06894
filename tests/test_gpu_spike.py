"""GPU parity tests: libspike.so (through its C ABI) against the CPU oracle.

Tolerances: every FP64
result must have backward error ||op(A)x - f|| / (||op(A)|| ||x||) <= 1e-13,
and on diagonally dominant inputs a relative forward error <= 1e-9 against the
oracle.  SPIKE and banded GEPP agree only up to rounding (different operation
order), so nothing here is compared bit for bit.
"""
import numpy as np
import pytest

import oracle
from oracle import metrics
from paper_1811_03559_gb300 import inputs, spike

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BERR = 1e-13
FERR_DD = 1e-9


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_solve(band, kl, ku, F, p, trans="N", pivot=0, **kw):
    fac = spike.factor(_dev(band), kl, ku, p, pivot, **kw)
    X = _dev(F)
    fac.solve(X, trans)
    torch.cuda.synchronize()
    return X.cpu().numpy(), fac


def check(band, kl, ku, F, X, trans, dd=True, xref=None):
    be = metrics.backward_error(band, kl, ku, X, F, trans)
    assert be <= BERR, be
    if xref is None:
        xref, info = oracle.gbsv(band, kl, ku, F, trans)
        assert info == 0
    if dd:
        fe = metrics.forward_error(X, xref)
        assert fe <= FERR_DD, fe
    return be


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    spike.lib()


# --------------------------------------------------------------- small workload (n=1e4, k=8, p=4)
def test_small_workload_p4():
    p = inputs.make_problem(10_000, 8, 8, 1, seed=0, dd=1.1)
    X, fac = gpu_solve(p["band"], 8, 8, p["F"], 4)
    check(p["band"], 8, 8, p["F"], X, "N")
    assert metrics.forward_error(X, p["xstar"]) <= FERR_DD
    inf = fac.info()
    assert inf["P"] == 4 and inf["leaves"] == 4 and inf["boosts"] == 0


@pytest.mark.parametrize("p", list(range(1, 10)))
@pytest.mark.parametrize("trans", ["N", "T"])
def test_p_invariance(p, trans):
    n, k = 4000, 8
    pr = inputs.make_problem(n, k, k, 3, seed=10 + p, dd=1.1, trans=trans)
    X, fac = gpu_solve(pr["band"], k, k, pr["F"], p, trans)
    check(pr["band"], k, k, pr["F"], X, trans)


@pytest.mark.parametrize("kl,ku,p", [(3, 7, 5), (7, 3, 6), (0, 4, 3), (5, 0, 4), (1, 1, 7)])
@pytest.mark.parametrize("trans", ["N", "T"])
def test_unequal_bandwidths(kl, ku, p, trans):
    pr = inputs.make_problem(3001, kl, ku, 2, seed=kl * 10 + ku, dd=1.2, trans=trans)
    band = pr["band"].copy()
    band[:, ku] += 1.0  # rows with no off-diagonal entries (kl or ku = 0) would otherwise get a zero diagonal
    F = inputs.band_matvec(band, kl, ku, pr["xstar"], trans)
    X, _ = gpu_solve(band, kl, ku, F, p, trans)
    check(band, kl, ku, F, X, trans)


@pytest.mark.parametrize("nrhs", [1, 2, 7, 33, 130])
@pytest.mark.parametrize("trans", ["N", "T"])
def test_many_rhs(nrhs, trans):
    pr = inputs.make_problem(5003, 16, 16, nrhs, seed=nrhs, dd=1.05, trans=trans)
    X, _ = gpu_solve(pr["band"], 16, 16, pr["F"], 6, trans)
    check(pr["band"], 16, 16, pr["F"], X, trans)


@pytest.mark.parametrize("p", [64, 148, 192])
@pytest.mark.parametrize("trans", ["N", "T"])
@pytest.mark.parametrize("stage_balance", [False, True])
def test_large_p(p, trans, stage_balance):
    n, k = 200_000, 16
    pr = inputs.make_problem(n, k, k, 2, seed=p, dd=1.01, trans=trans)
    X, fac = gpu_solve(pr["band"], k, k, pr["F"], p, trans, nrhs_hint=2, stage_balance=stage_balance)
    check(pr["band"], k, k, pr["F"], X, trans)
    assert fac.info()["p_effective"] == p


@pytest.mark.parametrize("k", [32, 64, 128])
def test_wide_band(k):
    n = 60_000
    pr = inputs.make_problem(n, k, k, 4, seed=k, dd=1.5)
    for trans in ("N", "T"):
        F = inputs.band_matvec(pr["band"], k, k, pr["xstar"], trans)
        X, _ = gpu_solve(pr["band"], k, k, F, 9, trans)
        check(pr["band"], k, k, F, X, trans)


def test_p1_is_banded_lu():
    """One block: SPIKE(p=1) is a single non-pivoting banded LU (Sec. 2.3)."""
    pr = inputs.make_problem(3000, 5, 5, 2, seed=4, dd=1.3)
    X, fac = gpu_solve(pr["band"], 5, 5, pr["F"], 1)
    xlu, info = oracle.nopiv_solve(pr["band"], 5, 5, pr["F"], "N", "LU")
    assert info == 0 and fac.info()["leaves"] == 1
    assert metrics.forward_error(X, xlu) <= 1e-13


def test_host_pointers_match_device():
    pr = inputs.make_problem(7000, 6, 6, 3, seed=8, dd=1.1)
    Xd, _ = gpu_solve(pr["band"], 6, 6, pr["F"], 5)
    fac = spike.factor(np.ascontiguousarray(pr["band"]), 6, 6, 5)
    Xh = np.ascontiguousarray(pr["F"]).copy()
    fac.solve(Xh, "N")
    np.testing.assert_array_equal(Xh, Xd)


@pytest.mark.parametrize("mixed", [False, True])
def test_pinned_host_band_matches_device(mixed):
    """A pinned host band (read in place by the setup kernels for FP64 handles, copied straight
    into the FP64 band of mixed ones), a pageable one (staged) and a device one give the same
    bits, for host and device right-hand sides, N and T."""
    n, kl, ku, p, m = 30_011, 9, 5, 12, 4
    pr = inputs.make_problem(n, kl, ku, m, seed=31, dd=1.05)
    band = np.ascontiguousarray(pr["band"])
    pinned = torch.from_numpy(band).pin_memory()
    assert pinned.is_pinned()
    facs = [spike.factor(b, kl, ku, p, mixed=mixed) for b in (_dev(band), pinned.numpy(), band.copy())]
    for trans in ("N", "T"):
        F = inputs.band_matvec(band, kl, ku, pr["xstar"], trans)
        outs = []
        for i, fac in enumerate(facs):
            X = _dev(F)
            fac.solve(X, trans)
            outs.append(X.cpu().numpy())
            Fh = torch.from_numpy(F.copy()).pin_memory() if i == 1 else None
            Xh = Fh.numpy() if Fh is not None else F.copy()
            fac.solve(Xh, trans)
            outs.append(Xh.copy())
        for o in outs[1:]:
            np.testing.assert_array_equal(o, outs[0])
        check(band, kl, ku, F, outs[0], trans)
    for fac in facs:
        fac.free()


def test_refactor_and_reuse_for_both_transposes():
    pr = inputs.make_problem(9000, 10, 10, 2, seed=21, dd=1.1)
    fac = spike.factor(_dev(pr["band"]), 10, 10, 7)
    for trans in ("N", "T", "N"):
        F = inputs.band_matvec(pr["band"], 10, 10, pr["xstar"], trans)
        X = _dev(F)
        fac.solve(X, trans)
        torch.cuda.synchronize()
        check(pr["band"], 10, 10, F, X.cpu().numpy(), trans)


def test_gpu_backward_error_kernel_matches_oracle():
    pr = inputs.make_problem(20_000, 12, 9, 3, seed=2, dd=1.1)
    X, _ = gpu_solve(pr["band"], 12, 9, pr["F"], 5)
    X[1, 100] += 1e-9  # make the residual visible
    for trans in ("N", "T"):
        F = pr["F"] if trans == "N" else inputs.band_matvec(pr["band"], 12, 9, X, "T")
        if trans == "T":
            F[:, 50] += 1e-9  # a residual well above rounding in every column
        be_gpu = spike.backward_error(_dev(pr["band"]), 12, 9, _dev(X), _dev(F), trans)
        for c in range(3):
            be_cpu = metrics.backward_error(pr["band"], 12, 9, X[c:c + 1], F[c:c + 1], trans)
            # two evaluations of the same residual in different summation orders differ by at
            # most ~(kl+ku+1) u ||A|| ||x||, i.e. (kl+ku+1) u in backward-error units
            assert abs(be_gpu[c] - be_cpu) <= 4 * (12 + 9 + 1) * np.finfo(float).eps, (trans, c)
            if trans == "T" or c == 1:
                assert be_cpu > 1e-12  # the planted residual is visible


@pytest.mark.parametrize("n,kl,ku,m", [(1000, 12, 9, 8), (20_011, 5, 17, 40), (50, 3, 2, 16),
                                        (5000, 320, 320, 33), (3000, 0, 7, 9), (4099, 128, 128, 64)])
def test_gpu_backward_error_many_columns(n, kl, ku, m):
    """The tiled residual (8 or more right-hand sides) against the oracle's, column by column:
    ragged row tiles, n below one tile, a band too wide for 32-column chunks, kl = 0."""
    band, rng = inputs.make_band(n, kl, ku, seed=4, dd=1.2)
    X = rng.uniform(-1.0, 1.0, size=(m, n))
    F = rng.uniform(-1.0, 1.0, size=(m, n))
    for trans in ("N", "T"):
        be_gpu = spike.backward_error(_dev(band), kl, ku, _dev(X), _dev(F), trans)
        for c in range(m):
            be_cpu = metrics.backward_error(band, kl, ku, X[c:c + 1], F[c:c + 1], trans)
            assert be_gpu[c] == pytest.approx(be_cpu, rel=1e-12), (trans, c)


# ------------------------------------------------------------------ spike tips vs definition
def _sub_band(band, kl, ku, s, e):
    """Band of the diagonal block A[s:e, s:e]."""
    nl = e - s
    sub = np.zeros((nl, kl + ku + 1))
    for d in range(kl + ku + 1):
        off = d - ku  # row = col + off
        for c in range(nl):
            r = c + off
            if 0 <= r < nl:
                sub[c, d] = band[s + c, d]
    return sub


def _block(band, kl, ku, rows, cols):
    n = band.shape[0]
    out = np.zeros((len(rows), len(cols)))
    for a, i in enumerate(rows):
        for b, j in enumerate(cols):
            if 0 <= j < n and -ku <= i - j <= kl:
                out[a, b] = band[j, ku + i - j]
    return out


def _groups_per_level(offs, flags):
    """Leaf ranges of the groups that own spikes at each merge level (Sec. 2.2 / 3.1)."""
    nb = len(offs) - 1
    levels = []
    groups = [(i, i + 1) for i in range(nb)]
    has_pairs = any(f & 2 for f in flags)
    if has_pairs:
        levels.append(groups)
        merged, i = [], 0
        while i < nb:
            if flags[i] & 2:
                merged.append((i, i + 2))
                i += 2
            else:
                merged.append((i, i + 1))
                i += 1
        groups = merged
    while len(groups) > 1:
        levels.append(groups)
        groups = [(groups[j][0], groups[j + 1][1]) for j in range(0, len(groups), 2)]
    return levels


@pytest.mark.parametrize("p,k", [(6, 4), (5, 3), (8, 2), (14, 3)])
def test_spike_tips_equal_block_solves(p, k):
    """V^[l], W^[l] tips equal the tips of A_G^{-1} B_G and A_G^{-1} C_G for every group G (Eq. spikes,
    applied to the merged blocks of Sec. 2.2)."""
    n = 1200
    band, _ = inputs.make_band(n, k, k, seed=p, dd=1.2)
    fac = spike.factor(_dev(band), k, k, p)
    info = fac.info()
    _, offs, flags = spike.plan(n, k, k, p)
    levels = _groups_per_level(offs, flags)
    assert len(levels) == info["levels"]
    nb = info["leaves"]
    for lv, groups in enumerate(levels):
        tips = fac.tips(lv)
        for (g0, g1) in groups:
            s, e = offs[g0], offs[g1]
            sub = _sub_band(band, k, k, s, e)
            lu = oracle.BandLU(sub, k, k)
            V = W = None
            if g1 < nb:
                B = _block(band, k, k, range(s, e), range(e, e + k))
                V = lu.solve(B.T.copy(), "N").T  # (e-s) x k
            if g0 > 0:
                C = _block(band, k, k, range(s, e), range(s - k, s))
                W = lu.solve(C.T.copy(), "N").T
            for i in range(g0, g1):
                rs, re_ = offs[i] - s, offs[i + 1] - s
                if V is not None:
                    if i > 0:
                        np.testing.assert_allclose(tips[i, 0], V[rs:rs + k], atol=1e-12)
                    np.testing.assert_allclose(tips[i, 1], V[re_ - k:re_], atol=1e-12)
                if W is not None:
                    np.testing.assert_allclose(tips[i, 2], W[rs:rs + k], atol=1e-12)
                    if i < nb - 1:
                        np.testing.assert_allclose(tips[i, 3], W[re_ - k:re_], atol=1e-12)


# ------------------------------------------------------------------------- pivoting
@pytest.mark.parametrize("p,k", [(1, 4), (2, 8), (5, 16), (8, 16)])
@pytest.mark.parametrize("trans", ["N", "T"])
def test_pivoting_nondominant(p, k, trans):
    n = 6000
    pr = inputs.make_problem(n, k, k, 3, seed=100 + p, dist="normal", dd=0.3, keep_sign=True, trans=trans)
    X, fac = gpu_solve(pr["band"], k, k, pr["F"], p, trans, pivot=1)
    be = metrics.backward_error(pr["band"], k, k, X, pr["F"], trans)
    assert be <= BERR, be


def test_pivoting_matches_gepp_when_p1():
    """One pivoted block is exactly banded GEPP: same pivots, same result up to summation order."""
    pr = inputs.make_problem(2000, 6, 6, 2, seed=5, dist="normal", dd=0.2, keep_sign=True)
    X, _ = gpu_solve(pr["band"], 6, 6, pr["F"], 1, pivot=1)
    xo, _ = oracle.gbsv(pr["band"], 6, 6, pr["F"])
    from oracle import condest
    cond = condest.cond1_estimate(pr["band"], 6, 6)
    assert metrics.forward_error(X, xo) <= 1e-14 * cond


@pytest.mark.parametrize("k,n", [(40, 3000), (128, 3000), (300, 2400)])
def test_pivoting_one_block_matches_gepp(k, n):
    """One pivoted block at bandwidths that run the look-ahead block GEPP with one trailing chunk
    (k = 40), with several (k = 128), and the single-buffer block GEPP (k = 300): the pivots are
    those of the oracle's banded GEPP, so the results agree to rounding times the condition."""
    pr = inputs.make_problem(n, k, k, 2, seed=7, dist="normal", dd=0.3, keep_sign=True)
    assert oracle.BandLU(pr["band"], k, k).info == 0
    from oracle import condest
    cond = condest.cond1_estimate(pr["band"], k, k)
    for trans in ("N", "T"):
        F = pr["F"]
        X, _ = gpu_solve(pr["band"], k, k, F, 1, trans, pivot=1)
        xo, _ = oracle.gbsv(pr["band"], k, k, F, trans)
        be = metrics.backward_error(pr["band"], k, k, X, F, trans)
        bo = metrics.backward_error(pr["band"], k, k, xo, F, trans)
        assert be <= BERR
        # two solutions with backward errors be, bo differ by about cond * (be + bo) (the bound of
        # test_pivoting_workload, with the same allowance for the estimator and first-order terms)
        assert metrics.forward_error(X, xo) <= max(1e-12, 20.0 * cond * (be + bo)), (trans, cond, be, bo)


@pytest.mark.parametrize("k,p,n", [(128, 3, 6000), (300, 2, 4000)])
@pytest.mark.parametrize("trans", ["N", "T"])
def test_pivoting_wide_bands(k, p, n, trans):
    pr = inputs.make_problem(n, k, k, 3, seed=11 + p, dist="normal", dd=0.3, keep_sign=True, trans=trans)
    X, fac = gpu_solve(pr["band"], k, k, pr["F"], p, trans, pivot=1)
    assert metrics.backward_error(pr["band"], k, k, X, pr["F"], trans) <= BERR


@pytest.mark.parametrize("kl,ku,p", [(3, 9, 1), (3, 9, 4), (9, 2, 1), (9, 2, 5)])
@pytest.mark.parametrize("trans", ["N", "T"])
def test_pivoting_unequal_bandwidths(kl, ku, p, trans):
    """kl != ku with pivoting: the blocks are padded to k = max(kl, ku) (Sec. 2.1) and the GEPP's
    candidates beyond kl are zero; against the oracle's banded GEPP (kl, ku as given)."""
    n = 3000
    pr = inputs.make_problem(n, kl, ku, 2, seed=40 + kl + p, dist="normal", dd=0.5, keep_sign=True, trans=trans)
    assert oracle.BandLU(pr["band"], kl, ku).info == 0
    X, _ = gpu_solve(pr["band"], kl, ku, pr["F"], p, trans, pivot=1)
    xo, _ = oracle.gbsv(pr["band"], kl, ku, pr["F"], trans)
    be = metrics.backward_error(pr["band"], kl, ku, X, pr["F"], trans)
    bo = metrics.backward_error(pr["band"], kl, ku, xo, pr["F"], trans)
    assert be <= BERR
    from oracle import condest
    cond = condest.cond1_estimate(pr["band"], kl, ku)
    assert metrics.forward_error(X, xo) <= max(1e-12, 20.0 * cond * (be + bo)), (cond, be, bo)


def test_pivot_zero_column_reports_singular():
    n, k = 400, 3
    band, _ = inputs.make_band(n, k, k, seed=1, dist="normal", dd=0.5, keep_sign=True)
    j = 150
    for d in range(2 * k + 1):  # zero column j of A
        band[j, d] = 0.0
    fac = spike.Factorization(_dev(band), k, k, 1, pivot=1)
    assert fac.status == j + 1 and fac.info()["zero_pivot_col"] == j + 1
    with pytest.raises(spike.SpikeError) as e:
        fac.solve(_dev(np.ones((1, n))))
    assert e.value.code == j + 1


# ----------------------------------------------------------- full-size property checks
@pytest.mark.parametrize("p", [148])
def test_full_size_k128(p):
    """n = 2^20, k = 128 (the benchmark's factor+solve shape): backward error on the GPU and on the
    host from the original band; forward error against the manufactured solution."""
    n, k = 1 << 20, 128
    pr = inputs.make_problem(n, k, k, 1, seed=1, dd=1.01)
    bd = _dev(pr["band"])
    fac = spike.factor(bd, k, k, p, nrhs_hint=1)
    for trans in ("N", "T"):
        F = pr["F"] if trans == "N" else inputs.band_matvec(pr["band"], k, k, pr["xstar"], "T")
        X = _dev(F)
        fac.solve(X, trans)
        be_gpu = spike.backward_error(bd, k, k, X, _dev(F), trans)
        assert be_gpu.max() <= BERR
        Xh = X.cpu().numpy()
        rows = np.random.default_rng(0).choice(n, 2000, replace=False)
        assert metrics.forward_error(Xh, pr["xstar"]) <= FERR_DD
        be = metrics.backward_error(pr["band"], k, k, Xh, F, trans)
        assert be <= BERR
        assert np.all(np.isfinite(Xh[:, rows]))


def test_gpu_measure_K_and_tune():
    """The machine constant K (Sec. 3.3) measured on one block, and the timed search: the best
    configuration is the minimum of the returned table and the table is complete."""
    n, k = 200_000, 32
    pr = inputs.make_problem(n, k, k, 1, seed=9, dd=1.1)
    bd = _dev(pr["band"])
    K = spike.measure_K(bd, k, k)
    assert 0.2 < K < 20.0
    res, table = spike.tune(bd, k, k, 8, [16, 64], r13_candidates=[1.5, 3.0], nsolves=1)
    assert res["tried"] == table.size == 8 and np.all(table > 0)
    assert res["best_ms"] == pytest.approx(table.min())
    assert res["best_p"] in (16, 64) and res["K_measured"] > 0
    i, c = np.unravel_index(np.argmin(table), table.shape)
    assert res["best_p"] == [16, 64][i] and res["best_mode"] == min(c, 2)
