"""The tensor-core residual of mixed-precision handles (spike_residual, the kernel the FP64
iterative refinement uses) against the exact residual (oracle.metrics.residual_exact:
error-free products, exactly rounded sums).

Bars: with small integer inputs every fixed-point digit is exact, so the result must equal
the exact residual bit for bit; with random FP64 inputs each element must lie within the
worst-case error bound of the method, (W + 4) 2^-53 ||op(A)||_inf ||x_c||_inf, W = kl + ku + 1
(two fixed-point roundings of 2^-54 of the row / column scale per term, then the final
roundings), which is also the bound of a plain FP64 dot product of length W.
"""
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


def _gpu_residual(fac, X, F, trans):
    Xd, Fd = _dev(X), _dev(F)
    R = torch.empty_like(Fd)
    berr = fac.residual(Xd, Fd, R, trans)
    torch.cuda.synchronize()
    return R.cpu().numpy(), berr


@pytest.mark.parametrize("n,kl,ku,nrhs", [(5003, 3, 7, 1), (4001, 16, 16, 33), (3001, 0, 5, 8), (2000, 6, 0, 40)])
@pytest.mark.parametrize("trans", ["N", "T"])
def test_integer_inputs_are_exact(n, kl, ku, nrhs, trans):
    rng = np.random.default_rng(n + kl + 7 * ku)
    band = rng.integers(-20, 21, size=(n, kl + ku + 1)).astype(np.float64)
    inputs._mask_outside(band, kl, ku)
    band[:, ku] = inputs.row_offdiag_abs_sum(band, kl, ku) + 5.0  # dominant: the factorization exists
    X = rng.integers(-1000, 1001, size=(nrhs, n)).astype(np.float64)
    F = rng.integers(-10 ** 6, 10 ** 6, size=(nrhs, n)).astype(np.float64)
    fac = spike.factor(_dev(band), kl, ku, 4, 0, mixed=True)
    R, _ = _gpu_residual(fac, X, F, trans)
    ref = metrics.residual_exact(band, kl, ku, X, F, trans)
    assert np.array_equal(R, ref), np.abs(R - ref).max()
    fac.free()


@pytest.mark.parametrize("n,kl,ku,nrhs", [(5003, 3, 7, 1), (4001, 16, 16, 33), (3001, 0, 5, 8), (2000, 128, 128, 40),
                                          (1500, 40, 0, 64)])
@pytest.mark.parametrize("trans", ["N", "T"])
def test_random_inputs_within_bound(n, kl, ku, nrhs, trans):
    band, rng = inputs.make_band(n, kl, ku, seed=n + kl, dd=1.1)
    X = rng.uniform(-1.0, 1.0, size=(nrhs, n)) * np.exp(rng.uniform(-3, 3, size=(nrhs, 1)))
    F = inputs.band_matvec(band, kl, ku, X, trans) + rng.uniform(-1e-6, 1e-6, size=(nrhs, n))
    fac = spike.factor(_dev(band), kl, ku, 4, 0, mixed=True)
    R, berr = _gpu_residual(fac, X, F, trans)
    ref = metrics.residual_exact(band, kl, ku, X, F, trans)
    anorm = metrics.band_norm_inf(band, kl, ku, trans)
    xn = np.abs(X).max(axis=1)
    W = kl + ku + 1
    err = np.abs(R - ref).max(axis=1) / (anorm * xn)
    assert np.all(err <= (W + 4) * 2.0 ** -53), err.max()
    # the per-column backward errors it returns are those of the exact residual, to the same bound
    be_ref = np.abs(ref).max(axis=1) / (anorm * xn)
    np.testing.assert_allclose(berr, be_ref, rtol=1e-12, atol=(W + 4) * 2.0 ** -53)
    fac.free()


@pytest.mark.parametrize("nrhs", [3, 16])
@pytest.mark.parametrize("trans", ["N", "T"])
def test_mixed_refinement_with_either_residual(nrhs, trans):
    """The refinement reaches the same accuracy with the tensor-core residual (8 or more
    columns) as with FP64 FMAs, in the same number of steps, and matches the oracle."""
    n, k, p = 60_000, 24, 12
    pr = inputs.make_problem(n, k, k, nrhs, seed=77, dd=1.02, trans=trans)
    xo, info = oracle.gbsv(pr["band"], k, k, pr["F"], trans)
    assert info == 0
    steps = {}
    for fp64 in (False, True):
        fac = spike.factor(_dev(pr["band"]), k, k, p, 0, mixed=True, fp64_residual=fp64, nrhs_hint=nrhs)
        X = _dev(pr["F"])
        fac.solve(X, trans)
        Xh = X.cpu().numpy()
        steps[fp64] = fac.info()["refine_steps"]
        assert metrics.backward_error(pr["band"], k, k, Xh, pr["F"], trans) <= 1e-13
        assert metrics.forward_error(Xh, xo) <= 1e-9
        fac.free()
    assert steps[False] == steps[True], steps


def test_residual_needs_a_split_handle():
    band, _ = inputs.make_band(1000, 4, 4, seed=5, dd=1.1)
    X = _dev(np.ones((2, 1000)))
    for kw in ({}, {"mixed": True, "fp64_residual": True}):
        fac = spike.factor(_dev(band), 4, 4, 2, 0, **kw)
        with pytest.raises(spike.SpikeError) as e:
            fac.residual(X, X, torch.empty_like(X))
        assert e.value.code == spike.SPIKE_ENOTSUP
        fac.free()
