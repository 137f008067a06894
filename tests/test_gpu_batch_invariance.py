"""Batch invariance: a right-hand side gets the same bits whether it is solved alone or
together with other right-hand sides, at any position in the batch.

This is what lets a server merge the solves of independent requests on one matrix
(same trans, same precision) into one multi-column solve without changing any
request's answer.  Covered: FP64 without and with pivoting, mixed precision (per-column
refinement stop), N and T, one and several staged window chunks (k = 160 with pivoting
gives a 320-row U window).
"""
import numpy as np
import pytest

import oracle
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


CASES = [
    # n, k, p, pivot, mixed, dist, dd
    (20_000, 16, 10, 0, False, "uniform", 1.1),
    (20_000, 16, 10, 1, False, "normal", 0.5),
    (20_000, 16, 10, 0, True, "uniform", 1.1),
    (24_000, 128, 6, 0, False, "uniform", 1.01),
    (24_000, 160, 5, 1, False, "uniform", 1.5),
    (24_000, 64, 7, 0, True, "uniform", 1.05),
]


@pytest.mark.parametrize("n,k,p,pivot,mixed,dist,dd", CASES)
def test_alone_equals_batched(n, k, p, pivot, mixed, dist, dd):
    seed = 11
    while True:
        band, _ = inputs.make_band(n, k, k, seed=seed, dist=dist, dd=dd, keep_sign=(dist == "normal"))
        if not pivot:
            break
        if oracle.BandLU(band, k, k).info == 0:
            break
        seed += 1
    rng = np.random.default_rng(5)
    F = rng.uniform(-1.0, 1.0, size=(40, n))
    fac = spike.factor(_dev(band), k, k, p, pivot, mixed=mixed, batch_invariant=True)
    for trans in ("N", "T"):
        Xb = _dev(F[:13])
        fac.solve(Xb, trans)
        Xb = Xb.cpu().numpy()
        Xw = _dev(F[::-1].copy())  # 40 columns, reversed order: column j sits at 39 - j
        fac.solve(Xw, trans)
        Xw = Xw.cpu().numpy()[::-1]
        for j in (0, 5, 12):
            Xa = _dev(F[j:j + 1])
            fac.solve(Xa, trans)
            Xa = Xa.cpu().numpy()[0]
            assert np.array_equal(Xa, Xb[j]), (trans, j, np.abs(Xa - Xb[j]).max())
            assert np.array_equal(Xa, Xw[j]), (trans, j, np.abs(Xa - Xw[j]).max())
    fac.free()
