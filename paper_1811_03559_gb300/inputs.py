"""Seeded synthetic inputs for banded solves.

This module only builds inputs: a band matrix A, a known solution X* and the
right-hand side F = op(A) X*.  It holds none of the solver's arithmetic and is
shared by the GPU path's tests/benchmark and by the CPU oracle's tests.

Recipe (the paper's own test matrices, Sec. 5.3: random band entries with the
diagonal set from a degree of diagonal dominance DD):
  * NumPy PCG64 stream ``default_rng(seed)``; all draws in float64.
  * The full band array (n columns x (kl+ku+1) rows, column-major band order)
    is drawn first; entries that fall outside the matrix are then zeroed.
  * Each diagonal entry is overwritten with DD x (sum of |off-diagonal entries
    in its row)  -- DD > 1 gives a strictly row diagonally dominant matrix.
    With ``keep_sign`` the drawn entry's sign is kept (used for the
    non-dominant N(0,1) systems).
  * X* (nrhs x n, column-major) is drawn next from the same stream.
  * F = op(A) X* is formed in FP64.

Array conventions: band has shape (n, kl+ku+1) with band[j, ku+i-j] = A(i, j)
(LAPACK band layout); X* and F have shape (nrhs, n) with F[c, i] = F(i, c).
"""
import numpy as np


def _mask_outside(band, kl, ku):
    n = band.shape[0]
    for d in range(kl + ku + 1):
        off = d - ku  # row i = j + off
        if off < 0:
            band[: min(n, -off), d] = 0.0
        elif off > 0:
            band[max(0, n - off):, d] = 0.0


def row_offdiag_abs_sum(band, kl, ku):
    n = band.shape[0]
    tot = np.zeros(n)
    for d in range(kl + ku + 1):
        if d == ku:
            continue
        off = d - ku  # A(j+off, j) = band[j, d]
        if off >= 0:
            tot[off:] += np.abs(band[: n - off, d])
        else:
            tot[: n + off] += np.abs(band[-off:, d])
    return tot


def make_band(n, kl, ku, seed, dist="uniform", dd=1.1, keep_sign=False, rng=None):
    """Return (band, rng).  dist: 'uniform' (U[-1,1]) or 'normal' (N(0,1))."""
    if rng is None:
        rng = np.random.default_rng(seed)
    ldab = kl + ku + 1
    if dist == "uniform":
        band = rng.uniform(-1.0, 1.0, size=(n, ldab))
    elif dist == "normal":
        band = rng.standard_normal(size=(n, ldab))
    else:
        raise ValueError(dist)
    _mask_outside(band, kl, ku)
    s = row_offdiag_abs_sum(band, kl, ku)
    if keep_sign:
        sign = np.where(band[:, ku] < 0, -1.0, 1.0)
        band[:, ku] = sign * dd * s
    else:
        band[:, ku] = dd * s
    return band, rng


def band_matvec(band, kl, ku, X, trans="N"):
    """op(A) X in FP64 (input construction only)."""
    n = band.shape[0]
    X = np.atleast_2d(X)
    Y = np.zeros_like(X, dtype=np.float64)
    for d in range(kl + ku + 1):
        off = d - ku  # A(j+off, j) = band[j, d]
        j0, j1 = max(0, -off), min(n, n - off)
        if j1 <= j0:
            continue
        cols = slice(j0, j1)
        rows = slice(j0 + off, j1 + off)
        if trans == "N":
            Y[:, rows] += band[cols, d] * X[:, cols]
        else:
            Y[:, cols] += band[cols, d] * X[:, rows]
    return Y


def make_problem(n, kl, ku, nrhs, seed, dist="uniform", dd=1.1, keep_sign=False, trans="N"):
    """Return dict(band, xstar, F) for the recipe in the module docstring."""
    band, rng = make_band(n, kl, ku, seed, dist=dist, dd=dd, keep_sign=keep_sign)
    xstar = rng.uniform(-1.0, 1.0, size=(nrhs, n))
    F = band_matvec(band, kl, ku, xstar, trans)
    return {"band": band, "xstar": xstar, "F": F, "n": n, "kl": kl, "ku": ku}


# The workloads (synthetic stand-ins for the paper's n = 10^6, b = 321 runs of Sec. 3.4 and the
# pivoting runs of Sec. 5.3).  Seeds: workload index c uses seed c.
SMALL_P4 = dict(n=10_000, kl=8, ku=8, nrhs=1, p=4, dist="uniform", dd=1.1, seed=0)
LARGE = dict(n=1_048_576, kls=(32, 128, 320), nrhs=(1, 64), ps=(64, 148, 192), dds=(1.01, 1.5), seed=1)
PIVOT = dict(n=262_144, kls=(16, 64), nrhs=8, p=148, dist="normal", dd=0.3, keep_sign=True, seed=2)
# Many-matrix serving workload: 10,000 requests arriving as a Poisson process at
# 2000/s over a catalogue of 500 matrices (n log-uniform in [1e3, 2e5], k uniform in
# {4, 8, ..., 128}, DD 1.1), matrix chosen by Zipf(1.1) rank, nrhs uniform in [1, 32],
# 30 % transpose solves, 50 % mixed precision, 40 GB device budget.
SERVING = dict(requests=10_000, rate=2000.0, matrices=500, n_lo=1_000, n_hi=200_000, k_choices=tuple(range(4, 129, 4)),
               dd=1.1, zipf=1.1, nrhs_max=32, trans_t=0.3, mixed=0.5, budget_gb=40, seed=4)


def serving_catalogue(cfg=SERVING, rng=None):
    """(n, k) of every catalogue matrix, from the workload seed."""
    rng = np.random.default_rng(cfg["seed"]) if rng is None else rng
    m = cfg["matrices"]
    ns = np.exp(rng.uniform(np.log(cfg["n_lo"]), np.log(cfg["n_hi"]), m)).astype(np.int64)
    ks = rng.choice(np.asarray(cfg["k_choices"]), m)
    return ns, ks, rng


def serving_trace(cfg=SERVING, rng=None):
    """Request stream: arrival times (s), matrix ids, nrhs, trans ('N'/'T'), mixed flags."""
    rng = np.random.default_rng(cfg["seed"] + 1000) if rng is None else rng
    r = cfg["requests"]
    ranks = np.arange(1, cfg["matrices"] + 1, dtype=np.float64)
    pz = ranks ** (-cfg["zipf"])
    pz /= pz.sum()
    arrivals = np.cumsum(rng.exponential(1.0 / cfg["rate"], r))
    mids = rng.choice(cfg["matrices"], size=r, p=pz)  # matrix id = popularity rank - 1
    nrhs = rng.integers(1, cfg["nrhs_max"] + 1, r)
    trans = np.where(rng.random(r) < cfg["trans_t"], "T", "N")
    mixed = rng.random(r) < cfg["mixed"]
    return arrivals, mids, nrhs, trans, mixed


def make_band_torch(n, kl, ku, seed, dd=1.1, device="cuda"):
    """A band drawn on `device` with torch's generator (U[-1, 1], zero outside the matrix,
    diagonal = dd x row off-diagonal |.| sum, as make_band).  Used where a catalogue of
    hundreds of matrices is generated in device memory; its stream differs from make_band's."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    ldab = kl + ku + 1
    band = torch.rand((n, ldab), generator=g, dtype=torch.float64, device=device) * 2.0 - 1.0
    tot = torch.zeros(n, dtype=torch.float64, device=device)
    for d in range(ldab):
        off = d - ku  # A(j+off, j) = band[j, d]
        if off < 0:
            band[: min(n, -off), d] = 0.0
        elif off > 0:
            band[max(0, n - off):, d] = 0.0
        if d == ku:
            continue
        if off >= 0:
            tot[off:] += band[: n - off, d].abs()
        else:
            tot[: n + off] += band[-off:, d].abs()
    band[:, ku] = dd * tot
    return band


def band_matvec_torch(band, kl, ku, X, trans="N"):
    """band_matvec on torch tensors (any device): op(A) X in FP64, input construction only."""
    import torch
    n = band.shape[0]
    Y = torch.zeros_like(X, dtype=torch.float64)
    for d in range(kl + ku + 1):
        off = d - ku  # A(j+off, j) = band[j, d]
        j0, j1 = max(0, -off), min(n, n - off)
        if j1 <= j0:
            continue
        if trans == "N":
            Y[:, j0 + off:j1 + off] += band[j0:j1, d] * X[:, j0:j1]
        else:
            Y[:, j0:j1] += band[j0:j1, d] * X[:, j0 + off:j1 + off]
    return Y
