"""Degenerate sizes and cases of the solver on the GPU: one row, a band as wide as the
matrix, no right-hand sides, and an exact zero pivot without pivoting (boosting, Sec. 2.3)."""
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


def test_single_row():
    band = np.array([[4.0]])
    fac = spike.factor(_dev(band), 0, 0, 3)
    assert fac.info()["p_effective"] == 1
    for trans in ("N", "T"):
        X = _dev(np.array([[2.0], [-6.0]]))
        fac.solve(X, trans)
        assert np.array_equal(X.cpu().numpy(), np.array([[0.5], [-1.5]]))


@pytest.mark.parametrize("n,kl,ku", [(5, 4, 4), (6, 5, 2), (2, 1, 1)])
def test_band_as_wide_as_the_matrix(n, kl, ku):
    band, rng = inputs.make_band(n, kl, ku, seed=3, dd=1.3)
    F = rng.uniform(-1, 1, size=(3, n))
    fac = spike.factor(_dev(band), kl, ku, 8)
    assert fac.info()["p_effective"] == 1  # no block of 2k rows fits: one block
    for trans in ("N", "T"):
        X = _dev(F)
        fac.solve(X, trans)
        xo, info = oracle.gbsv(band, kl, ku, F, trans)
        assert info == 0
        assert metrics.forward_error(X.cpu().numpy(), xo) <= 1e-12


def test_zero_right_hand_sides_is_a_no_op():
    band, _ = inputs.make_band(2000, 3, 3, seed=1)
    fac = spike.factor(_dev(band), 3, 3, 4)
    # no columns: nothing is read or written, so any non-null pointer is accepted
    assert spike.lib().spike_solve_ex(fac._h, spike.ctypes.c_void_p(8), 2000, 0, b"N") == 0
    assert spike.lib().spike_solve_ex(fac._h, spike.ctypes.c_void_p(8), 2000, 0, b"T") == 0


def test_zero_pivot_without_pivoting_is_boosted():
    """A(0,0) = 0 with a non-pivoting factorization: the pivot is replaced by +tau
    (tau = 2^-26 max|a_ij|), counted in info.boosts, and the solve stays finite; the
    factorization is approximate (Sec. 2.3), the pivoting one is exact."""
    n, k = 3000, 2
    band, rng = inputs.make_band(n, k, k, seed=4, dd=1.5)
    band[0, k] = 0.0  # A(0,0)
    F = rng.uniform(-1, 1, size=(2, n))
    fac = spike.factor(_dev(band), k, k, 4)
    assert fac.info()["boosts"] >= 1
    X = _dev(F)
    fac.solve(X, "N")
    assert torch.isfinite(X).all()
    piv = spike.factor(_dev(band), k, k, 4, pivot=1)
    assert piv.info()["boosts"] == 0
    Xp = _dev(F)
    piv.solve(Xp, "N")
    assert metrics.backward_error(band, k, k, Xp.cpu().numpy(), F, "N") <= 1e-13


def test_library_pool_keeps_and_releases_memory():
    """Freed factorizations stay in the library's pool (reused by the next one) until
    spike_release_cached hands them back to the driver."""
    band, _ = inputs.make_band(200_000, 16, 16, seed=2)
    fac = spike.factor(_dev(band), 16, 16, 32)
    fac.free()
    before, after = spike.release_cached()
    assert before >= 8 * 200_000 * 33  # at least the freed factor storage was still held
    assert after < before


def test_nan_in_the_matrix_is_reported_not_an_error():
    """A NaN on the diagonal of one block: the factorization and the solve succeed (LAPACK
    semantics), the result carries NaN, and spike_info.numerics flags the NaN pivot; a clean
    matrix reports no flag."""
    n, k = 3000, 2
    band, rng = inputs.make_band(n, k, k, seed=6, dd=1.5)
    clean = spike.factor(_dev(band), k, k, 4)
    assert clean.info()["numerics"] == 0
    band[1500, k] = np.nan  # A(1500, 1500)
    fac = spike.factor(_dev(band), k, k, 4)
    assert fac.info()["numerics"] & spike.NUMERICS_NAN_PIVOT
    X = _dev(rng.uniform(-1, 1, size=(1, n)))
    fac.solve(X, "N")
    assert torch.isnan(X).any()


def test_singular_interface_block_is_reported():
    """Two diagonal blocks of 2s coupled through the 2 x 2 block [[2, 2], [2, 2]] at their
    boundary (rows 19 and 20): the tips are V_b = W_t = 2 / 2 = 1 exactly, so the interface
    block S = I - W V of the reduced system (Sec. 2.2) is exactly 0 and A is singular (the
    oracle's GEPP agrees).  The factorization succeeds and flags it in spike_info.numerics."""
    n, k = 40, 1
    _, offs, _ = spike.plan(n, k, k, 2)
    assert list(offs) == [0, 20, 40]
    band = np.zeros((n, 3))
    band[:, 1] = 2.0    # diagonal
    band[20, 0] = 2.0   # A(19, 20)
    band[19, 2] = 2.0   # A(20, 19)
    assert oracle.gbsv(band, k, k, np.ones(n))[1] > 0
    fac = spike.factor(_dev(band), k, k, 2)
    info = fac.info()
    assert info["numerics"] & spike.NUMERICS_SINGULAR_INTERFACE and info["boosts"] == 0
    X = _dev(np.ones((1, n)))
    fac.solve(X, "N")
    assert not torch.isfinite(X).all()
