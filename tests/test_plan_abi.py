"""Host-side tests: the partition planner (Sec. 3.1, 3.3) and the C ABI surface (no GPU needed)."""
import json
import os
import re

import numpy as np
import pytest

from paper_1811_03559_gb300 import spike

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    if not os.path.exists(spike.LIB_PATH):
        from paper_1811_03559_gb300 import build
        build.build()
    return spike.lib()


def test_abi_exports_every_declared_symbol(built):
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            hdr = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"\b(spike_[a-z0-9_]+)\s*\(", hdr))
    assert {"spike_factor", "spike_solve", "spike_free", "spike_plan", "spike_server_create",
            "spike_server_submit", "spike_solve_ws", "spike_factor_bytes"} <= names
    for nm in names:
        assert hasattr(built, nm), nm


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLD, "thread_distribution.json")))["cases"])
def test_thread_distribution(built, case):
    info, offs, flags = spike.plan(1 << 20, 4, 4, case["t"])
    assert (info["P"], info["r"], info["p_effective"]) == (case["P"], case["r"], case["t_eff"])
    assert info["leaves"] == case["P"] + case["r"]
    # 2x2 pairs are partitions 2..r+1: leaves 1..2r alternate top (LU) / bottom (UL)
    for j in range(case["r"]):
        assert flags[1 + 2 * j] == 2 and flags[2 + 2 * j] == 5
    assert flags[0] == 0
    if info["leaves"] > 1:
        assert flags[-1] == 1  # last block: UL
    assert offs[0] == 0 and offs[-1] == 1 << 20 and np.all(np.diff(offs) > 0)


def test_ratios_match_paper_table(built):
    g = json.load(open(os.path.join(GOLD, "partition_ratios.json")))
    for row in g["rows"]:
        info, _, _ = spike.plan(10**6, g["k"], g["k"], 12, K=g["K"], nrhs_hint=row["nrhs"])
        assert abs(info["R13"] - row["R13"]) <= 0.1 + 1e-12
        assert abs(info["R12"] - row["R12"]) <= 0.05 + 1e-12
        assert info["R12"] == pytest.approx(info["R13"] / 2)
    lim, _, _ = spike.plan(10**6, g["k"], g["k"], 12, K=g["K"], nrhs_hint=0)
    assert lim["R13"] == pytest.approx(g["factor_limit"]["R13"])
    assert lim["R12"] == pytest.approx(g["factor_limit"]["R12"])
    big, _, _ = spike.plan(10**6, 1, 1, 12, K=g["K"], nrhs_hint=10**7)
    assert big["R13"] == pytest.approx(g["solve_limit"]["R13"], abs=1e-5)


@pytest.mark.parametrize("t", [4, 5, 6, 9, 14, 64, 148, 192])
@pytest.mark.parametrize("K,rho", [(2.0, 0), (4 / 3, 0.5), (2.0, 1.0)])
def test_partition_sizes_follow_ratios(built, t, K, rho):
    n, k = 1_048_576, 128
    info, offs, flags = spike.plan(n, k, k, t, K=K, nrhs_hint=int(rho * k))
    sizes = np.diff(offs)
    assert sizes.sum() == n
    P, r = info["P"], info["r"]
    n1, n2, n3 = info["n1"], info["n2"], info["n3"]
    # constraint n = 2 n1 + r n2 + (P-2-r) n3 (before the remainder rows)
    assert 0 <= n - (2 * n1 + r * n2 + (P - 2 - r) * n3) <= P
    assert n1 / n3 == pytest.approx(info["R13"], rel=1e-3)
    assert abs(n2 - 2 * n3) <= 1
    # leaves: ends are n1, pairs split n2 floor/ceil, singles n3 (+ at most one remainder row)
    assert sizes[0] == n1 and sizes[-1] == n1
    for j in range(r):
        assert sizes[1 + 2 * j] + sizes[2 + 2 * j] in (n2, n2 + 1)
    for s in sizes[1 + 2 * r:-1]:
        assert s in (n3, n3 + 1)


def test_small_matrix_lowers_worker_count(built):
    # every block needs >= 2k rows; with n = 10 k only a few blocks fit
    info, offs, _ = spike.plan(1000, 50, 50, 64)
    assert np.all(np.diff(offs) >= 100)
    assert info["p_effective"] < 64


def test_bad_arguments(built):
    with pytest.raises(spike.SpikeError) as e:
        spike.plan(0, 2, 2, 4)
    assert e.value.code == -1
    with pytest.raises(spike.SpikeError) as e:
        spike.plan(100, 2, 2, 0)
    assert e.value.code == -4
    with pytest.raises(spike.SpikeError) as e:
        spike.plan(100, -1, 2, 2)
    assert e.value.code == -2
    import ctypes
    h = ctypes.c_void_p()
    assert built.spike_factor(None, 100, 2, 2, 4, 0, ctypes.byref(h)) == -1
    x = np.zeros((100, 5))
    assert built.spike_factor_ex(x.ctypes.data_as(ctypes.c_void_p), 5, 0, 2, 2, 4, 0, None, ctypes.byref(h)) == -3
    assert built.spike_factor_ex(x.ctypes.data_as(ctypes.c_void_p), 4, 100, 2, 2, 4, 0, None, ctypes.byref(h)) == -2
    assert built.spike_factor_ex(x.ctypes.data_as(ctypes.c_void_p), 5, 100, 2, 2, 4, 3, None, ctypes.byref(h)) == -7
    assert built.spike_solve(None, None, 1, b"N") == spike.SPIKE_EHANDLE
    assert built.spike_strerror(-1002).decode().startswith("CUDA")


def test_stage_balance_uses_paper_limits(built):
    """SPIKE_FLAG_STAGE_BALANCE: R13 = 2 (Eq. ratios) when a solve is expected, else 1 + 1.5 K (Eq. ratiof)."""
    info, offs, _ = spike.plan(1_048_576, 128, 128, 148, K=2.0, nrhs_hint=64, stage_balance=True)
    assert info["R13"] == 2.0 and info["R12"] == 1.0
    sizes = np.diff(offs)
    assert abs(sizes[0] - 2 * info["n3"]) <= 1 and abs(sizes[1] + sizes[2] - 2 * info["n3"]) <= 2
    f, _, _ = spike.plan(1_048_576, 128, 128, 148, K=4 / 3, nrhs_hint=0, stage_balance=True)
    assert f["R13"] == pytest.approx(3.0)


@pytest.mark.parametrize("r13", [1.0, 1.7, 3.0])
def test_explicit_ratio_override(built, r13):
    """options.R13 > 0 replaces both the formula and the stage-balance choice (Sec. 3.3 sizing
    with a given ratio): n1 / n3 = R13 and n2 = 2 n3 up to the integer rounding."""
    for sb in (False, True):
        info, offs, flags = spike.plan(1 << 20, 16, 16, 148, nrhs_hint=64, stage_balance=sb, R13=r13)
        assert info["R13"] == r13 and info["R12"] == pytest.approx(r13 / 2)
        assert abs(info["n1"] / info["n3"] - r13) < 1e-3
        assert abs(info["n2"] - 2 * info["n3"]) <= 1
        assert offs[-1] == 1 << 20


@pytest.mark.parametrize("n,k,p", [(200_000, 16, 32), (1 << 20, 128, 148), (50_001, 7, 9)])
def test_factor_bytes_accounting(built, n, k, p):
    """spike_factor_bytes (computed without a GPU, used by the serving engine's budget) against the
    storage the header documents: the FP64 band copy of mixed handles (8 n (kl+ku+1) bytes, none when
    the band is borrowed), the staged copy of a host band in the transient figure, FP32 block factors
    and reciprocals in mixed handles (ldf = 2k+2 values per row), and the pivoting layout (U fill to
    2k above the diagonal: ldf = 3k+1 rounded up to even, plus one int pivot per row)."""
    ldab = 2 * k + 1
    band_bytes = 8 * n * ldab
    slack = 256 * 16  # each carved buffer is rounded up to 256 bytes

    def fb(**kw):
        return spike.factor_bytes(n, k, k, p, **kw)

    r64, t64 = fb()
    r64h, t64h = fb(host_band=True)
    assert r64h == r64 and r64 == fb(borrow_band=True)[0]  # FP64 handles keep no band
    assert abs((t64h - t64) - band_bytes) <= slack           # staged host band
    rmix, tmix = fb(mixed=True, fp64_residual=True)
    rbor, _ = fb(mixed=True, borrow_band=True, fp64_residual=True)
    assert abs((rmix - rbor) - band_bytes) <= slack           # the FP64 band copy, unless borrowed
    assert fb(mixed=True, borrow_band=True, host_band=True, fp64_residual=True)[0] == rmix  # needs a device band
    # the tensor-core residual's digit planes of A and A^T: per 16-row block, 8 planes x
    # ceil((16 + kl + ku + 3) / 32) chunks x 512 bytes, plus one int32 row exponent per row
    nch = (16 + 2 * k + 3 + 31) // 32
    split = 2 * (((n + 15) // 16) * 8 * nch * 512 + 4 * n)
    assert abs((fb(mixed=True)[0] - rmix) - split) <= slack
    ldf = 2 * k + 2
    assert abs((r64 - rbor) - 4 * n * (ldf + 1)) <= slack     # factors and 1/u_jj: 8 -> 4 bytes
    assert abs((t64 - tmix) - 4 * n * 2 * k) <= slack         # the spike right-hand sides Z in FP32
    rpiv, _ = fb(pivot=1)
    ldf_piv = (3 * k + 1 + 1) // 2 * 2
    assert abs((rpiv - r64) - (8 * n * (ldf_piv - ldf) + 4 * n)) <= slack
    assert r64 >= 8 * n * (ldf + 1)
    with pytest.raises(spike.SpikeError) as e:
        fb(pivot=1, mixed=True)
    assert e.value.code == spike.SPIKE_ENOTSUP


def test_bandwidth_limit(built):
    """max(kl, ku) up to SPIKE_MAX_K = 512 is planned (blocks of >= 2k rows); one more is refused
    with SPIKE_ENOTSUP, by the planner, the factorization and the serving engine alike."""
    import ctypes
    info, offs, _ = spike.plan(1 << 20, 512, 200, 64)
    assert info["k"] == 512 and np.all(np.diff(offs) >= 1024)
    for kl, ku in ((513, 0), (0, 513)):
        with pytest.raises(spike.SpikeError) as e:
            spike.plan(1 << 20, kl, ku, 64)
        assert e.value.code == spike.SPIKE_ENOTSUP
        res, tr = ctypes.c_int64(0), ctypes.c_int64(0)
        rc = built.spike_factor_bytes(1 << 20, kl, ku, 64, 0, None, 0, ctypes.byref(res), ctypes.byref(tr))
        assert rc == spike.SPIKE_ENOTSUP
    from paper_1811_03559_gb300 import serve
    with serve.Server(1 << 30, dryrun=True) as S:
        with pytest.raises(spike.SpikeError) as e:
            S.add_matrix(0, np.zeros((5000, 1027)), 513, 513)
        assert e.value.code == spike.SPIKE_ENOTSUP


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without libspike.so every entry point of the binding raises."""
    monkeypatch.setattr(spike, "_lib", None)
    monkeypatch.setattr(spike, "LIB_PATH", str(tmp_path / "libspike.so"))
    with pytest.raises(RuntimeError, match="libspike.so not found"):
        spike.plan(1000, 2, 2, 4)
    with pytest.raises(RuntimeError, match="libspike.so not found"):
        spike.factor(np.zeros((1000, 5)), 2, 2, 4)
    with pytest.raises(RuntimeError, match="libspike.so not found"):
        spike.factor_bytes(1000, 2, 2, 4)


def test_plan_structure_on_random_sizes(built):
    """Structure of 400 random plans (Sec. 3.1): the blocks tile [0, n) with at least 2k rows each
    (one block may be shorter: then it is the only one); P = 2^m partitions of which partitions
    2..r+1 (1-based) are SPIKE 2x2 pairs (top half flag 2, bottom half flag 4|1: a UL block) and the
    last block is UL; t_eff = P + r <= t blocks in all; one merge level for the pairs plus m; and the
    plan is a fixed point (planning again with t_eff gives the same blocks)."""
    rng = np.random.default_rng(12)
    for _ in range(400):
        n = int(np.exp(rng.uniform(0, np.log(2e6))))
        k = int(rng.integers(0, 65))
        k = min(k, max(n - 1, 0))
        t = int(rng.integers(1, 400))
        info, offs, flags = spike.plan(n, k, k, t)
        kk = max(1, k)
        sizes = np.diff(offs)
        nb = len(sizes)
        assert offs[0] == 0 and offs[-1] == n and np.all(sizes >= 1)
        assert nb == 1 or np.all(sizes >= 2 * kk), (n, k, t)
        P, r, m = info["P"], info["r"], info["m"]
        assert P == 1 << m and nb == P + r == info["p_effective"] == info["leaves"] <= t
        assert r <= max(P - 2, 0)
        expect = [0] * nb
        for j in range(r):
            expect[1 + 2 * j], expect[2 + 2 * j] = 2, 5
        if nb > 1:
            expect[-1] = 1
        assert list(flags) == expect, (n, k, t)
        assert info["levels"] == m + (1 if r > 0 else 0)
        again, offs2, _ = spike.plan(n, k, k, info["p_effective"])
        assert again["p_effective"] == info["p_effective"] and np.array_equal(offs2, offs)


@pytest.mark.parametrize("m", [2, 3, 5, 7])
def test_one_below_a_power_of_two_idles_a_worker(built, m):
    """t = 2^(m+1) - 1 would need r = 2^m - 1 pairs, but only the P - 2 inner partitions can be
    split (the first and last use LU / UL alone); the paper runs it as 2^(m+1) - 2 workers with
    one idle (Sec. 3.1)."""
    t = (2 << m) - 1
    info, _, _ = spike.plan(1 << 22, 4, 4, t)
    assert info["p_effective"] == t - 1 and info["P"] == 1 << m and info["r"] == (1 << m) - 2
