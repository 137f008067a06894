"""The backward-error entry point that allocates nothing, checked against the allocating one.

Callers that cannot allocate during a call (device memory held entirely by their own
pool, or loops that cannot absorb cudaFree's device-wide synchronisation) use
spike_backward_error_noalloc, whose reduction scratch is a fixed device array.  This
file is collected last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_1811_03559_gb300 import inputs, spike

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    spike.lib()


def _call_noalloc(band, kl, ku, X, F, trans):
    L = spike.lib()
    n, ldab = band.shape
    nrhs = X.shape[0]
    out = np.full(nrhs, -1.0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.spike_backward_error_noalloc(ctypes.c_void_p(band.data_ptr()), ldab, n, kl, ku,
                                        ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(F.data_ptr()), nrhs,
                                        trans.encode(), stream, out.ctypes.data_as(ctypes.c_void_p))
    assert rc == 0, rc
    return out


def test_noalloc_matches_allocating_entry_point_twice():
    n, kl, ku = 30_000, 9, 6
    pr = inputs.make_problem(n, kl, ku, 5, seed=31, dd=1.1)
    band = torch.from_numpy(pr["band"]).cuda()
    for call, (trans, nrhs) in enumerate([("N", 5), ("T", 3)]):  # two calls in a row, different sizes
        X = torch.from_numpy(pr["xstar"][:nrhs].copy()).cuda()
        X[:, 17 + call] += 1e-7 * (call + 1)  # a residual well above rounding
        F = torch.from_numpy(inputs.band_matvec(pr["band"], kl, ku, pr["xstar"][:nrhs], trans)).cuda()
        ref = spike.backward_error(band, kl, ku, X, F, trans)
        got = _call_noalloc(band, kl, ku, X, F, trans)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
        assert np.all(got > 1e-12)


@pytest.mark.parametrize("n,kl,ku,nrhs,trans", [(20_000, 7, 4, 8, "N"), (20_000, 7, 4, 40, "T"),
                                                (300, 2, 3, spike.NOALLOC_MAX_NRHS, "N")])
def test_noalloc_tiled_path_and_limit(n, kl, ku, nrhs, trans):
    """Eight or more right-hand sides take the tiled residual kernel; nrhs at exactly the limit
    fills the whole fixed array (its last words hold the finished per-column errors)."""
    pr = inputs.make_problem(n, kl, ku, nrhs, seed=33 + nrhs, dd=1.1)
    band = torch.from_numpy(pr["band"]).cuda()
    X = torch.from_numpy(pr["xstar"].copy()).cuda()
    X[:, n // 3] += 1e-6  # a residual well above rounding in every column
    F = torch.from_numpy(inputs.band_matvec(pr["band"], kl, ku, pr["xstar"], trans)).cuda()
    for _ in range(2):  # the second call must not see the first one's maxima
        ref = spike.backward_error(band, kl, ku, X, F, trans)
        got = _call_noalloc(band, kl, ku, X, F, trans)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
        assert np.all(got > 1e-12)
    # a smaller residual afterwards: the words reused from the larger call are cleared
    X2 = torch.from_numpy(pr["xstar"].copy()).cuda()
    got2 = _call_noalloc(band, kl, ku, X2, F, trans)
    ref2 = spike.backward_error(band, kl, ku, X2, F, trans)
    np.testing.assert_allclose(got2, ref2, rtol=1e-12, atol=1e-300)
    assert np.all(got2 < 1e-13)


def test_noalloc_rejects_nrhs_above_limit():
    L = spike.lib()
    band = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    X = torch.zeros((spike.NOALLOC_MAX_NRHS + 1, 10), dtype=torch.float64, device="cuda")
    out = np.zeros(spike.NOALLOC_MAX_NRHS + 1)
    rc = L.spike_backward_error_noalloc(ctypes.c_void_p(band.data_ptr()), 3, 10, 1, 1, ctypes.c_void_p(X.data_ptr()),
                                        ctypes.c_void_p(X.data_ptr()), spike.NOALLOC_MAX_NRHS + 1, b"N", None,
                                        out.ctypes.data_as(ctypes.c_void_p))
    assert rc == spike.SPIKE_ELIMIT
    assert "limit" in L.spike_strerror(rc).decode()
