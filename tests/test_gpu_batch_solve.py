"""spike_solve_batch: several systems of uneven n, k, p and nrhs solved together, stage by
stage in shared launches, must return bitwise what each system's own solve returns."""
import ctypes

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


# (n, k, p, nrhs, batch_invariant): p = 1 has no reduced system; the others have 1 to 6
# merge levels, so the levels of different systems line up only partly
SYSTEMS = [(3000, 4, 3, 1, False), (20_000, 32, 10, 7, True), (9000, 64, 6, 16, False),
           (50_000, 16, 40, 3, False), (1000, 12, 1, 5, True), (20_000, 32, 10, 2, False)]


@pytest.fixture(scope="module")
def systems():
    out = []
    for i, (n, k, p, m, inv) in enumerate(SYSTEMS):
        band, _ = inputs.make_band(n, k, k, seed=300 + i, dd=1.1)
        fac = spike.factor(torch.from_numpy(band).cuda(), k, k, p, 0, batch_invariant=inv)
        F = np.random.default_rng(i).uniform(-1, 1, size=(m, n))
        out.append((band, k, fac, F))
    return out


@pytest.mark.parametrize("trans", ["N", "T"])
def test_batch_equals_separate_solves(systems, trans):
    facs, Fs, alone = [], [], []
    for band, k, fac, F in systems:
        X = torch.from_numpy(F).cuda()
        fac.solve(X, trans)
        alone.append(X)
        facs.append(fac)
        Fs.append(torch.from_numpy(F).cuda())
    # the same handle twice, with other right-hand sides
    extra = np.random.default_rng(99).uniform(-1, 1, size=(4, systems[1][3].shape[1]))
    facs.append(systems[1][2])
    Fs.append(torch.from_numpy(extra).cuda())
    Xe = torch.from_numpy(extra).cuda()
    systems[1][2].solve(Xe, trans)
    alone.append(Xe)
    spike.solve_batch(facs, Fs, trans)
    torch.cuda.synchronize()
    for i, (a, b) in enumerate(zip(alone, Fs)):
        assert torch.equal(a, b), (i, (a - b).abs().max().item())
    # every system against the oracle: backward error <= 1e-13 and forward error <= 1e-9
    # against banded GEPP (the bands are diagonally dominant), the reused handle included
    rhs = [F for _, _, _, F in systems] + [extra]
    owners = list(range(len(systems))) + [1]
    for i, (own, F) in enumerate(zip(owners, rhs)):
        band, k, _, _ = systems[own]
        X = Fs[i].cpu().numpy()
        assert metrics.backward_error(band, k, k, X, F, trans) <= 1e-13, i
        xo, info = oracle.gbsv(band, k, k, F, trans)
        assert info == 0
        assert metrics.forward_error(X, xo) <= 1e-9, i


def test_batch_argument_checks(systems):
    band, k, fac, F = systems[0]
    mixed = spike.factor(torch.from_numpy(band).cuda(), k, k, 3, 0, mixed=True)
    with pytest.raises(spike.SpikeError) as e:
        spike.solve_batch([fac, mixed], [torch.from_numpy(F).cuda(), torch.from_numpy(F).cuda()])
    assert e.value.code == spike.SPIKE_ENOTSUP
    hs = (ctypes.c_void_p * 1)(fac._h.value)
    X = torch.from_numpy(F).cuda()
    ptrs = (ctypes.c_void_p * 1)(X.data_ptr())
    nr = (ctypes.c_int * 1)(F.shape[0])
    need = ctypes.c_int64(0)
    assert spike.lib().spike_solve_batch_workspace(hs, nr, 1, b"N", ctypes.byref(need)) == 0 and need.value > 0
    ws = torch.empty(need.value - 1, dtype=torch.uint8, device="cuda")
    rc = spike.lib().spike_solve_batch(hs, ptrs, nr, 1, b"N", None, ctypes.c_void_p(ws.data_ptr()), ws.numel())
    assert rc == -8
    assert spike.lib().spike_solve_batch(hs, ptrs, nr, 1, b"X", None, ctypes.c_void_p(ws.data_ptr()), ws.numel()) == -5


@pytest.mark.parametrize("trans", ["N", "T"])
def test_batch_with_more_blocks_than_sms(trans):
    """14 systems x 16 blocks: the merged sweep stages have more blocks than SMs and run from
    the work queue (persistent CTAs, largest blocks first); results stay bitwise per system."""
    facs, Fs, alone = [], [], []
    for i in range(14):
        n, k, p = 12_000 + 1500 * i, 4 + 2 * (i % 5), 16
        band, _ = inputs.make_band(n, k, k, seed=500 + i, dd=1.1)
        fac = spike.factor(torch.from_numpy(band).cuda(), k, k, p, 0)
        F = np.random.default_rng(50 + i).uniform(-1, 1, size=(1 + i % 3, n))
        X = torch.from_numpy(F).cuda()
        fac.solve(X, trans)
        facs.append(fac)
        alone.append(X)
        Fs.append(torch.from_numpy(F).cuda())
    spike.solve_batch(facs, Fs, trans)
    torch.cuda.synchronize()
    for i, (a, b) in enumerate(zip(alone, Fs)):
        assert torch.equal(a, b), i
