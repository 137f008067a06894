"""Pins for the CPU oracle (runs without a GPU).

Each check ties the oracle to something other than itself: exact rational
arithmetic, LAPACK's own banded factorization (pivot sequence), an independent
dense elimination, closed-form solutions, the transpose identity, the factors
multiplied back into A, and the identities between GEPP, non-pivoting LU and UL
that the SPIKE partitions rely on (Sec. 2.3, Sec. 5.2).
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.linalg.lapack as lapack

import oracle
from oracle import condest, exact, metrics
from paper_1811_03559_gb300 import inputs

EPS = np.finfo(np.float64).eps


def int_band(n, kl, ku, rng, dominant=False):
    band = rng.integers(-5, 6, size=(n, kl + ku + 1)).astype(np.float64)
    inputs._mask_outside(band, kl, ku)
    if dominant:
        band[:, ku] = inputs.row_offdiag_abs_sum(band, kl, ku) + rng.integers(1, 4, size=n)
    return band


def transpose_band(band, kl, ku):
    """Band of A^T (lower/upper bandwidths swapped)."""
    n = band.shape[0]
    bt = np.zeros((n, kl + ku + 1))
    for j in range(n):
        for i in range(max(0, j - ku), min(n, j + kl + 1)):
            # A(i,j) -> A^T(j,i): stored in column i of the transposed band at row ku' + j - i, ku' = kl
            bt[i, kl + j - i] = band[j, ku + i - j]
    return bt


# ----------------------------------------------------------------- exact pins

@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("trans", ["N", "T"])
def test_exact_rational_tiny(seed, trans):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 17))
    kl, ku = int(rng.integers(0, 4)), int(rng.integers(0, 4))
    band = int_band(n, kl, ku, rng)
    A = oracle.band_to_dense(band, kl, ku)
    if abs(np.linalg.det(A)) < 0.5:
        band = int_band(n, kl, ku, rng, dominant=True)
        A = oracle.band_to_dense(band, kl, ku)
    f = rng.integers(-9, 10, size=n)
    xe = exact.solve_exact(A.astype(int).tolist(), f.tolist(), trans)
    assert xe is not None
    xe = np.array([float(v) for v in xe])
    x, info = oracle.gbsv(band, kl, ku, f.astype(np.float64), trans)
    assert info == 0
    cond = np.linalg.cond(A, np.inf)
    err = np.abs(x - xe).max() / max(np.abs(xe).max(), 1e-300)
    assert err <= 8 * n * EPS * cond + 1e-300


@pytest.mark.parametrize("kind", ["LU", "UL"])
@pytest.mark.parametrize("seed", range(6))
def test_exact_rational_nopiv(kind, seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(2, 17))
    kl, ku = int(rng.integers(1, 4)), int(rng.integers(1, 4))
    band = int_band(n, kl, ku, rng, dominant=True)
    A = oracle.band_to_dense(band, kl, ku)
    f = rng.integers(-9, 10, size=n)
    for trans in ("N", "T"):
        xe = np.array([float(v) for v in exact.solve_exact(A.astype(int).tolist(), f.tolist(), trans)])
        x, info = oracle.nopiv_solve(band, kl, ku, f.astype(np.float64), trans, kind)
        assert info == 0
        cond = np.linalg.cond(A, np.inf)
        assert np.abs(x - xe).max() / np.abs(xe).max() <= 8 * n * EPS * cond


# ------------------------------------------------------------- LAPACK pins

@pytest.mark.parametrize("seed", range(8))
def test_pivots_match_lapack_dgbtrf(seed):
    """Pivot order is exactly LAPACK's (first index of the largest |entry| in the band)."""
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(5, 200))
    kl, ku = int(rng.integers(1, 7)), int(rng.integers(1, 7))
    band, _ = inputs.make_band(n, kl, ku, seed=seed, dist="normal", dd=0.3, keep_sign=True)
    lu = oracle.BandLU(band, kl, ku)
    # LAPACK dgbtrf wants the band with kl extra rows on top, ldab = 2kl+ku+1, rows = diagonals
    ab = np.zeros((2 * kl + ku + 1, n))
    for d in range(kl + ku + 1):
        ab[kl + d, :] = band[:, d]
    lab, ipiv, info = lapack.dgbtrf(ab, kl, ku)
    assert info == lu.info == 0
    np.testing.assert_array_equal(ipiv, lu.ipiv)  # both 0-based
    # factors agree to rounding (LAPACK scales by a reciprocal, the oracle divides)
    np.testing.assert_allclose(lab.T, lu.fac, rtol=1e-12, atol=1e-12 * np.abs(lu.fac).max())


@pytest.mark.parametrize("trans", ["N", "T"])
def test_solution_matches_scipy_banded(trans):
    rng = np.random.default_rng(7)
    n, kl, ku = 300, 5, 3
    band, _ = inputs.make_band(n, kl, ku, seed=7, dist="normal", dd=0.5, keep_sign=True)
    F = rng.standard_normal((3, n))
    x, info = oracle.gbsv(band, kl, ku, F, trans)
    assert info == 0
    A = oracle.band_to_dense(band, kl, ku)
    if trans == "N":
        ab = np.zeros((kl + ku + 1, n))
        for d in range(kl + ku + 1):
            ab[d, :] = band[:, d]
        xs = scipy.linalg.solve_banded((kl, ku), ab, F.T).T
    else:
        xs = np.linalg.solve(A.T, F.T).T
    cond = np.linalg.cond(A, np.inf)
    assert np.abs(x - xs).max() / np.abs(xs).max() <= 50 * n * EPS * cond


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("trans", ["N", "T"])
def test_band_equals_dense_bitwise(seed, trans):
    """The banded GEPP does the same operations as dense GEPP (same pivots): identical N solves."""
    rng = np.random.default_rng(400 + seed)
    n = int(rng.integers(3, 60))
    kl, ku = int(rng.integers(1, 5)), int(rng.integers(1, 5))
    band, _ = inputs.make_band(n, kl, ku, seed=seed, dist="normal", dd=0.2, keep_sign=True)
    A = oracle.band_to_dense(band, kl, ku)
    F = rng.standard_normal((2, n))
    xb, ib = oracle.gbsv(band, kl, ku, F, trans)
    xd, idn = oracle.dense_solve(A, F, trans)
    assert ib == idn == 0
    if trans == "N":
        np.testing.assert_array_equal(xb, xd)
    else:
        # dense GEPP stores L with later row swaps applied, so the L^T dot products run in a
        # permuted order: same terms, different summation order
        assert np.abs(xb - xd).max() / np.abs(xd).max() <= 16 * n * EPS * np.linalg.cond(A, np.inf)


# ------------------------------------------------------------ closed forms

@pytest.mark.parametrize("n", [1, 2, 7, 100, 1001])
def test_tridiagonal_closed_form(n):
    """T = tridiag(-1, 2, -1), F = 1  =>  x_i = i (n+1-i) / 2 (1-based i)."""
    band = np.zeros((n, 3))
    band[:, 0] = -1.0
    band[:, 1] = 2.0
    band[:, 2] = -1.0
    inputs._mask_outside(band, 1, 1)
    i = np.arange(1, n + 1, dtype=np.float64)
    xe = i * (n + 1 - i) / 2.0
    for trans in ("N", "T"):
        x, info = oracle.gbsv(band, 1, 1, np.ones(n), trans)
        assert info == 0
        cond = (n + 1) ** 2  # kappa_inf(T) = O(n^2)
        assert np.abs(x - xe).max() / xe.max() <= 4 * EPS * cond
        x2, _ = oracle.nopiv_solve(band, 1, 1, np.ones(n), trans, "LU")
        x3, _ = oracle.nopiv_solve(band, 1, 1, np.ones(n), trans, "UL")
        assert np.abs(x2 - xe).max() / xe.max() <= 4 * EPS * cond
        assert np.abs(x3 - xe).max() / xe.max() <= 4 * EPS * cond


@pytest.mark.parametrize("s,sigma,jmode", [(2, 0.5, 1), (3, 1.0, 3), (4, 2.0, 7)])
def test_toeplitz_power_eigenvector(s, sigma, jmode):
    """(T + sigma I)^s has bandwidth s; x_i = sin(j pi i/(n+1)) is an eigenvector with
    eigenvalue (sigma + 2 - 2 cos(j pi/(n+1)))^s."""
    n = 240
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1) + sigma * np.eye(n)
    M = np.linalg.matrix_power(T, s)  # integer-valued when sigma is a half-integer multiple
    band = np.zeros((n, 2 * s + 1))
    for j in range(n):
        for i in range(max(0, j - s), min(n, j + s + 1)):
            band[j, s + i - j] = M[i, j]
    i = np.arange(1, n + 1)
    x = np.sin(jmode * np.pi * i / (n + 1))
    lam = (sigma + 2 - 2 * np.cos(jmode * np.pi / (n + 1))) ** s
    F = lam * x
    cond = ((sigma + 4) / sigma) ** s
    for trans in ("N", "T"):
        xo, info = oracle.gbsv(band, s, s, F, trans)
        assert info == 0
        assert np.abs(xo - x).max() <= 20 * n * EPS * cond


# ------------------------------------------------------- manufactured / identities

@pytest.mark.parametrize("dd", [1.01, 1.5])
@pytest.mark.parametrize("k", [2, 8])
def test_manufactured_solution(dd, k):
    p = inputs.make_problem(3000, k, k, 2, seed=11, dd=dd)
    for trans in ("N", "T"):
        F = inputs.band_matvec(p["band"], k, k, p["xstar"], trans)
        x, info = oracle.gbsv(p["band"], k, k, F, trans)
        assert info == 0
        assert metrics.forward_error(x, p["xstar"]) < 1e-12
        assert metrics.backward_error(p["band"], k, k, x, F, trans) < 1e-15


def test_transpose_identity():
    rng = np.random.default_rng(5)
    n, kl, ku = 157, 4, 2
    band, _ = inputs.make_band(n, kl, ku, seed=5, dist="normal", dd=0.4, keep_sign=True)
    F = rng.standard_normal((2, n))
    xt, _ = oracle.gbsv(band, kl, ku, F, "T")
    xn, _ = oracle.gbsv(transpose_band(band, kl, ku), ku, kl, F, "N")
    A = oracle.band_to_dense(band, kl, ku)
    assert np.abs(xt - xn).max() / np.abs(xn).max() <= 100 * n * EPS * np.linalg.cond(A, np.inf)


def test_gepp_on_column_dominant_is_plain_lu():
    """Column diagonal dominance => GEPP never swaps, so it equals the non-pivoting LU bit for bit.
    This is the reference for SPIKE(p=1), which is a single non-pivoting banded LU."""
    n, kl, ku = 400, 6, 6
    band, _ = inputs.make_band(n, kl, ku, seed=9, dd=1.1)
    bt = transpose_band(band, kl, ku)  # row dominance of A == column dominance of A^T
    lu = oracle.BandLU(bt, kl, ku)
    assert np.all(lu.ipiv == np.arange(n))
    fac, info = oracle.nopiv_factor(bt, kl, ku, "LU")
    assert info == 0
    np.testing.assert_array_equal(lu.fac[:, kl:], fac)
    assert np.all(lu.fac[:, :kl] == 0.0)


def test_ul_is_reversed_lu():
    """UL of A equals LU of Q A Q read backwards (Sec. 5.2, Eq. Qmat), bit for bit."""
    n, k = 300, 5
    band, _ = inputs.make_band(n, k, k, seed=13, dd=1.2)
    ul, info = oracle.nopiv_factor(band, k, k, "UL")
    assert info == 0
    # band of QAQ: (QAQ)(i,j) = A(n-1-i, n-1-j); with kl = ku the diagonal index flips
    qb = np.zeros_like(band)
    for j in range(n):
        for d in range(2 * k + 1):
            qb[j, d] = band[n - 1 - j, 2 * k - d]
    lu, info2 = oracle.nopiv_factor(qb, k, k, "LU")
    assert info2 == 0
    back = np.zeros_like(lu)
    for j in range(n):
        for d in range(2 * k + 1):
            back[j, d] = lu[n - 1 - j, 2 * k - d]
    np.testing.assert_array_equal(ul, back)


# ------------------------------------------------------------- factor checks

@pytest.mark.parametrize("seed", range(6))
def test_gepp_factors_rebuild_the_matrix(seed):
    """Multiplying the stored GEPP factors back together gives A: undo the elimination steps
    from the last to the first (apply L_j, then the row swap j <-> ipiv[j]) starting from U,
    and compare with the band's dense copy (Wilkinson's bound for GEPP: |A - P L U| is at
    most a small multiple of n * eps * |L| |U|)."""
    rng = np.random.default_rng(600 + seed)
    n = int(rng.integers(20, 160))
    kl, ku = int(rng.integers(1, 6)), int(rng.integers(1, 6))
    band, _ = inputs.make_band(n, kl, ku, seed=seed, dist="normal", dd=0.3, keep_sign=True)
    A = oracle.band_to_dense(band, kl, ku)
    lu = oracle.BandLU(band, kl, ku)
    assert lu.info == 0
    kv = kl + ku  # row of the diagonal in the factor storage: fac[j, kv + i - j] holds entry (i, j)
    U = np.zeros((n, n))
    L = np.eye(n)
    for j in range(n):
        for i in range(max(0, j - kv), j + 1):
            U[i, j] = lu.fac[j, kv + i - j]
        for i in range(j + 1, min(n, j + kl + 1)):
            L[i, j] = lu.fac[j, kv + i - j]
    M = U.copy()
    for j in range(n - 1, -1, -1):
        M[j + 1:, :] += np.outer(L[j + 1:, j], M[j, :])
        p = lu.ipiv[j]
        assert j <= p <= min(n - 1, j + kl)  # a pivot comes from inside the band
        M[[j, p], :] = M[[p, j], :]
    assert np.all(np.abs(np.tril(L, -1)) <= 1.0)  # partial pivoting bounds the multipliers
    bound = 4 * n * EPS * (np.abs(L) @ np.abs(U)).max()
    assert np.abs(M - A).max() <= bound
    # U fills to bandwidth kl + ku and no further
    assert np.all(np.triu(U, kv + 1) == 0.0)


@pytest.mark.parametrize("kind", ["LU", "UL"])
@pytest.mark.parametrize("k", [(1, 1), (3, 2), (2, 5)])
def test_nopiv_factors_rebuild_the_matrix(kind, k):
    """A = L U (unit L) and A = U L (unit U) from the in-place non-pivoting band factors of
    Sec. 2.3: the factors keep the band, L below and U above the diagonal."""
    kl, ku = k
    n = 90
    band, _ = inputs.make_band(n, kl, ku, seed=31 + kl + 7 * ku, dd=1.2)
    A = oracle.band_to_dense(band, kl, ku)
    fac, info = oracle.nopiv_factor(band, kl, ku, kind)
    assert info == 0
    F = oracle.band_to_dense(fac, kl, ku)
    lower, upper = np.tril(F, -1), np.triu(F, 1)
    diag = np.diag(np.diag(F))
    if kind == "LU":
        L, U = np.eye(n) + lower, diag + upper
        R = L @ U
    else:
        U, L = np.eye(n) + upper, diag + lower
        R = U @ L
    bound = 4 * n * EPS * (np.abs(L) @ np.abs(U) if kind == "LU" else np.abs(U) @ np.abs(L)).max()
    assert np.abs(R - A).max() <= bound
    if kind == "UL":
        # the UL factorization eliminates from the bottom: its last diagonal entry is A(n-1, n-1)
        assert F[n - 1, n - 1] == A[n - 1, n - 1]
    else:
        assert F[0, 0] == A[0, 0]


def test_singular_reports_info():
    n, k = 20, 2
    band = np.zeros((n, 2 * k + 1))
    band[:, k] = 1.0
    band[7, k] = 0.0  # column 7 entirely zero -> GEPP info = 8
    x, info = oracle.gbsv(band, k, k, np.ones(n))
    assert info == 8


def test_generator_matvec_matches_oracle_gbmv():
    p = inputs.make_problem(5000, 7, 3, 3, seed=3, dd=1.05)
    for trans in ("N", "T"):
        y1 = inputs.band_matvec(p["band"], 7, 3, p["xstar"], trans)
        y2 = oracle.gbmv(p["band"], 7, 3, p["xstar"], trans)
        np.testing.assert_allclose(y1, y2, rtol=0, atol=1e-13 * np.abs(y2).max())


def test_generator_dominance_and_determinism():
    b1, _ = inputs.make_band(1000, 8, 8, seed=0, dd=1.1)
    b2, _ = inputs.make_band(1000, 8, 8, seed=0, dd=1.1)
    np.testing.assert_array_equal(b1, b2)
    s = inputs.row_offdiag_abs_sum(b1, 8, 8)
    np.testing.assert_allclose(b1[:, 8], 1.1 * s)
    assert np.all(b1[:, 8] > s)


# ------------------------------------------------------------- condition estimate

@pytest.mark.parametrize("seed", range(4))
def test_condest_bounds(seed):
    n, k = 120, 3
    band, _ = inputs.make_band(n, k, k, seed=seed, dist="normal", dd=0.3, keep_sign=True)
    A = oracle.band_to_dense(band, k, k)
    true = np.linalg.cond(A, 1)
    est = condest.cond1_estimate(band, k, k)
    assert est <= true * (1 + 1e-10)
    assert est >= true / 10


def test_metrics_detect_planted_error():
    p = inputs.make_problem(2000, 4, 4, 1, seed=21, dd=1.1)
    x, _ = oracle.gbsv(p["band"], 4, 4, p["F"])
    assert metrics.backward_error(p["band"], 4, 4, x, p["F"]) < 1e-15
    x2 = x.copy()
    x2[0, 1000] += 1e-8
    assert metrics.backward_error(p["band"], 4, 4, x2, p["F"]) > 1e-10
    assert metrics.forward_error(x2, p["xstar"]) > 1e-9


# ------------------------------------------------------------------ metric pins
# The acceptance bars (backward error <= 1e-13, forward error <= 1e-9) are read through
# oracle.metrics, so its norms are pinned to their definitions (Sec. 3.4 "relative
# residual"; infinity norms, per column, max over columns): the band norms against
# numpy's matrix norms of a dense copy built here, the error formulas against a 3 x 3
# example worked by hand.  A swapped row/column sum, or a normalisation by the largest
# entry of the whole X instead of each column's, fails these.

def dense_from_band(band, kl, ku):
    """Dense A from the LAPACK band layout, built independently of the oracle's helper."""
    n = band.shape[0]
    A = np.zeros((n, n))
    for d in range(kl + ku + 1):
        off = d - ku  # A(j + off, j) = band[j, d]
        for j in range(n):
            i = j + off
            if 0 <= i < n:
                A[i, j] = band[j, d]
    return A


@pytest.mark.parametrize("kl,ku", [(0, 0), (0, 3), (3, 0), (1, 4), (5, 2), (7, 7)])
@pytest.mark.parametrize("ints", [True, False])
def test_band_norms_equal_dense_norms(kl, ku, ints):
    rng = np.random.default_rng(1000 + 31 * kl + ku)
    n = 37
    band = rng.integers(-9, 10, size=(n, kl + ku + 1)).astype(np.float64) if ints else rng.normal(size=(n, kl + ku + 1))
    # entries outside the matrix (band corners) must be ignored: fill them with large values
    for j in range(n):
        for d in range(kl + ku + 1):
            if not 0 <= j + d - ku < n:
                band[j, d] = 1e6
    A = dense_from_band(band, kl, ku)
    rt = 0.0 if ints else 1e-15  # integer sums are exact in any order
    assert metrics.band_norm_inf(band, kl, ku, "N") == pytest.approx(np.linalg.norm(A, np.inf), rel=rt, abs=0)
    assert metrics.band_norm_inf(band, kl, ku, "T") == pytest.approx(np.linalg.norm(A.T, np.inf), rel=rt, abs=0)
    assert condest.band_norm_1(band, kl, ku) == pytest.approx(np.linalg.norm(A, 1), rel=rt, abs=0)
    if kl + ku > 0:
        # row and column sums differ on these matrices, so a swap would be seen
        assert np.linalg.norm(A, np.inf) != np.linalg.norm(A, 1)


def hand_band():
    """A = [[4, 1, 0], [2, 5, 3], [0, 1, 6]] (kl = ku = 1): row sums 5, 10, 7; column sums 6, 7, 9."""
    A = np.array([[4.0, 1.0, 0.0], [2.0, 5.0, 3.0], [0.0, 1.0, 6.0]])
    band = np.zeros((3, 3))
    for j in range(3):
        for i in range(max(0, j - 1), min(3, j + 2)):
            band[j, 1 + i - j] = A[i, j]
    return band


def test_backward_error_hand_example_N():
    band = hand_band()
    # column 0: x = (1, 2, -1), A x = (6, 9, -4), f = (6, 9, -3.5): ||r|| = 0.5, ||x|| = 2 -> 0.5 / (10 * 2) = 0.025
    # column 1: x = (0.5, 0, 0), A x = (2, 1, 0), f = (2, 1.25, 0): ||r|| = 0.25, ||x|| = 0.5 -> 0.25 / (10 * 0.5) = 0.05
    X = np.array([[1.0, 2.0, -1.0], [0.5, 0.0, 0.0]])
    F = np.array([[6.0, 9.0, -3.5], [2.0, 1.25, 0.0]])
    assert metrics.band_norm_inf(band, 1, 1, "N") == 10.0
    assert metrics.backward_error(band, 1, 1, X[:1], F[:1], "N") == pytest.approx(0.025, rel=1e-15)
    assert metrics.backward_error(band, 1, 1, X[1:], F[1:], "N") == pytest.approx(0.05, rel=1e-15)
    # max over columns, each column normalised by its own ||x||
    assert metrics.backward_error(band, 1, 1, X, F, "N") == pytest.approx(0.05, rel=1e-15)


def test_backward_error_hand_example_T():
    band = hand_band()
    # A^T = [[4, 2, 0], [1, 5, 1], [0, 3, 6]], ||A^T||_inf = 9 (column sums of A)
    # column 0: A^T x = (8, 10, 0), f = (8, 10, 0.9): 0.9 / (9 * 2) = 0.05
    # column 1: A^T x = (2, 0.5, 0), f = (2, 0.5, 0.3): 0.3 / (9 * 0.5) = 1/15
    X = np.array([[1.0, 2.0, -1.0], [0.5, 0.0, 0.0]])
    F = np.array([[8.0, 10.0, 0.9], [2.0, 0.5, 0.3]])
    assert metrics.band_norm_inf(band, 1, 1, "T") == 9.0
    assert metrics.backward_error(band, 1, 1, X[:1], F[:1], "T") == pytest.approx(0.05, rel=1e-15)
    assert metrics.backward_error(band, 1, 1, X, F, "T") == pytest.approx(1.0 / 15.0, rel=1e-15)


def test_forward_error_hand_example():
    # per column ||x - x_ref||_inf / ||x_ref||_inf, max over columns:
    # column 0: |(1, 2.5, -1) - (1, 2, -1)| = 0.5, ||x_ref|| = 2 -> 0.25
    # column 1: |(0.5, 0.1, 0) - (0.5, 0, 0)| = 0.1, ||x_ref|| = 0.5 -> 0.2
    X = np.array([[1.0, 2.5, -1.0], [0.5, 0.1, 0.0]])
    Xref = np.array([[1.0, 2.0, -1.0], [0.5, 0.0, 0.0]])
    assert metrics.forward_error(X[1:], Xref[1:]) == pytest.approx(0.2, rel=1e-15)
    assert metrics.forward_error(X, Xref) == pytest.approx(0.25, rel=1e-15)


@pytest.mark.parametrize("seed", range(3))
def test_inverse_norm_estimate_is_a_lower_bound(seed):
    # Hager's estimate maximises ||A^{-1} x||_1 over unit vectors, so it never exceeds
    # ||A^{-1}||_1; on small diagonally dominant matrices it reaches it.
    n, kl, ku = 40, 2, 3
    band, _ = inputs.make_band(n, kl, ku, seed=50 + seed, dd=1.3)
    A = dense_from_band(band, kl, ku)
    true = np.linalg.norm(np.linalg.inv(A), 1)
    est = condest.inv_norm_1_estimate(oracle.BandLU(band, kl, ku))
    assert est <= true * (1 + 1e-12)
    assert est >= true * 0.5


# ------------------------------------------------------------ exact residual pins

def test_residual_exact_integer_inputs_match_plain_residual():
    # integer entries: every product and sum is exact in FP64, so both must agree bit for bit
    rng = np.random.default_rng(71)
    n, kl, ku = 60, 3, 5
    band = rng.integers(-50, 51, size=(n, kl + ku + 1)).astype(np.float64)
    X = rng.integers(-1000, 1001, size=(3, n)).astype(np.float64)
    F = rng.integers(-10 ** 6, 10 ** 6, size=(3, n)).astype(np.float64)
    for trans in ("N", "T"):
        plain = F - oracle.gbmv(band, kl, ku, X, trans)
        assert np.array_equal(metrics.residual_exact(band, kl, ku, X, F, trans), plain)


def test_residual_exact_recovers_cancelled_bits():
    # a x = (1 + 2^-30)(1 - 2^-30) = 1 - 2^-60: FP64 rounds the product to 1 and loses r
    band = np.array([[1.0 + 2.0 ** -30]])
    X = np.array([[1.0 - 2.0 ** -30]])
    F = np.array([[1.0]])
    assert (F - band[0, 0] * X)[0, 0] == 0.0
    assert metrics.residual_exact(band, 0, 0, X, F)[0, 0] == 2.0 ** -60


@pytest.mark.parametrize("trans", ["N", "T"])
def test_residual_exact_against_rationals(trans):
    from fractions import Fraction
    rng = np.random.default_rng(72)
    n, kl, ku = 14, 2, 3
    band = rng.normal(size=(n, kl + ku + 1))
    X = rng.normal(size=(2, n))
    F = rng.normal(size=(2, n))
    A = dense_from_band(band, kl, ku)
    Aop = A if trans == "N" else A.T
    R = metrics.residual_exact(band, kl, ku, X, F, trans)
    for c in range(2):
        for i in range(n):
            exact = Fraction(F[c, i]) - sum(Fraction(Aop[i, j]) * Fraction(X[c, j]) for j in range(n))
            assert R[c, i] == float(exact)  # correctly rounded
