"""spike_factor_batch: several systems of uneven n, k and p factored together (all their blocks in
one launch from a work queue, their reduced systems level by level in shared launches) must give
the handles a separate spike_factor_ex gives, bit for bit, and solves that match the oracle."""
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


# (n, kl, ku, p): p = 1 (no reduced system), pairs (p = 5, 7, 12, 40), unequal bandwidths, and
# systems with 0 to 6 merge levels, so the levels line up only partly
SYSTEMS = [(3000, 4, 4, 1), (20_000, 32, 32, 10), (9000, 64, 40, 5), (50_000, 16, 16, 40), (12_000, 8, 12, 7),
           (100_000, 128, 128, 12), (2500, 3, 3, 2)]


@pytest.mark.parametrize("trans", ["N", "T"])
def test_batch_factor_equals_separate(trans):
    bands, probs = [], []
    for i, (n, kl, ku, p) in enumerate(SYSTEMS):
        pr = inputs.make_problem(n, kl, ku, 3, seed=700 + i, dd=1.05, trans=trans)
        probs.append(pr)
        bands.append(torch.from_numpy(pr["band"]).cuda())
    facs = spike.factor_batch(bands, [s[1] for s in SYSTEMS], [s[2] for s in SYSTEMS], [s[3] for s in SYSTEMS])
    for i, ((n, kl, ku, p), pr, fb) in enumerate(zip(SYSTEMS, probs, facs)):
        solo = spike.factor(bands[i], kl, ku, p)
        assert fb.info()["leaves"] == solo.info()["leaves"] and fb.info()["boosts"] == 0
        Xb, Xs = torch.from_numpy(pr["F"]).cuda(), torch.from_numpy(pr["F"]).cuda()
        fb.solve(Xb, trans)
        solo.solve(Xs, trans)
        torch.cuda.synchronize()
        assert torch.equal(Xb, Xs), (i, (Xb - Xs).abs().max().item())
        X = Xb.cpu().numpy()
        assert metrics.backward_error(pr["band"], kl, ku, X, pr["F"], trans) <= 1e-13, i
        xo, info = oracle.gbsv(pr["band"], kl, ku, pr["F"], trans)
        assert info == 0 and metrics.forward_error(X, xo) <= 1e-9, i
        if i > 0:  # the reduced system's spike tips are those of the separate factorization
            assert np.array_equal(fb.tips(0), solo.tips(0))
        solo.free()
        fb.free()


def test_batch_factor_many_small_systems():
    """64 systems of 5,000-40,000 rows, k 4-32: more blocks than SMs in the shared launch."""
    rng = np.random.default_rng(3)
    sys_, bands, probs = [], [], []
    for i in range(64):
        n, k = int(rng.integers(5000, 40_000)), int(rng.choice([4, 8, 16, 32]))
        p = int(rng.integers(1, 9))
        pr = inputs.make_problem(n, k, k, 1, seed=900 + i, dd=1.1)
        sys_.append((n, k, p))
        probs.append(pr)
        bands.append(torch.from_numpy(pr["band"]).cuda())
    facs = spike.factor_batch(bands, [s[1] for s in sys_], [s[1] for s in sys_], [s[2] for s in sys_])
    for (n, k, p), pr, f in zip(sys_, probs, facs):
        X = torch.from_numpy(pr["F"]).cuda()
        f.solve(X, "N")
        assert metrics.forward_error(X.cpu().numpy(), pr["xstar"]) <= 1e-9
        f.free()


def test_batch_factor_rejects_unsupported():
    band = torch.from_numpy(inputs.make_band(2000, 4, 4, seed=1, dd=1.1)[0]).cuda()
    import ctypes
    opt = spike.SpikeOptions(flags=spike.FLAG_MIXED)
    ptrs = (ctypes.c_void_p * 1)(band.data_ptr())
    out = (ctypes.c_void_p * 1)()
    rc = spike.lib().spike_factor_batch(ptrs, (ctypes.c_int64 * 1)(9), (ctypes.c_int64 * 1)(2000),
                                        (ctypes.c_int * 1)(4), (ctypes.c_int * 1)(4), (ctypes.c_int * 1)(4), 1,
                                        ctypes.byref(opt), out)
    assert rc == spike.SPIKE_ENOTSUP and not out[0]
