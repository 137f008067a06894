"""Error metrics for banded solves -- TEST INFRASTRUCTURE ONLY.

Norms are infinity norms taken per right-hand-side column, and the reported
value is the maximum over columns:
  backward error  ||op(A) x - f|| / (||op(A)|| * ||x||)   (residual in FP64 from the original band)
  forward error   ||x - x_ref|| / ||x_ref||
The paper reports "relative residuals" without naming a norm (Sec. 3.4); the
infinity norm is the reading used here.
"""
import math

import numpy as np

from . import gbmv


def band_norm_inf(band, kl, ku, trans="N"):
    """||op(A)||_inf: max row sum of |A| ('N') or max column sum ('T')."""
    n = band.shape[0]
    if trans in ("T", "t"):
        # column j of A lives in band[j, :]; mask entries outside the matrix
        tot = np.zeros(n)
        for d in range(kl + ku + 1):
            i = np.arange(n) + d - ku
            ok = (i >= 0) & (i < n)
            tot += np.where(ok, np.abs(band[:, d]), 0.0)
        return float(tot.max())
    tot = np.zeros(n)
    for d in range(kl + ku + 1):
        j = np.arange(n)
        i = j + d - ku
        ok = (i >= 0) & (i < n)
        np.add.at(tot, i[ok], np.abs(band[j[ok], d]))
    return float(tot.max())


def backward_error(band, kl, ku, X, F, trans="N"):
    X = np.atleast_2d(X)
    F = np.atleast_2d(F)
    R = gbmv(band, kl, ku, X, trans) - F
    an = band_norm_inf(band, kl, ku, trans)
    num = np.abs(R).max(axis=1)
    den = an * np.abs(X).max(axis=1)
    return float((num / den).max())


def forward_error(X, Xref):
    X = np.atleast_2d(X)
    Xref = np.atleast_2d(Xref)
    return float((np.abs(X - Xref).max(axis=1) / np.abs(Xref).max(axis=1)).max())


def _split(a):
    """Veltkamp split of float64 values: a = hi + lo with hi, lo of at most 26 significant bits."""
    c = 134217729.0 * a  # 2^27 + 1
    hi = c - (c - a)
    return hi, a - hi


def _two_product(a, b):
    """Dekker's error-free product: p + e == a * b exactly (no overflow or underflow)."""
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def residual_exact(band, kl, ku, X, F, trans="N"):
    """R = F - op(A) X rounded once to FP64 from its exact value: every product a_ij x_jc is
    split exactly into two doubles (Dekker) and each row's terms are summed exactly by
    math.fsum (Shewchuk's algorithm, correctly rounded).  Reference for residual kernels;
    moderate sizes only (one fsum per row and column)."""
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    F = np.atleast_2d(np.asarray(F, dtype=np.float64))
    n = band.shape[0]
    lo, hi = (kl, ku) if trans in ("N", "n") else (ku, kl)
    W = lo + hi + 1
    # A_op[i, d] = op(A)(i, i - lo + d), zero outside the matrix
    Aop = np.zeros((n, W))
    for d in range(W):
        j = np.arange(n) - lo + d
        ok = (j >= 0) & (j < n)
        i = np.arange(n)[ok]
        jj = j[ok]
        Aop[ok, d] = band[jj, ku + i - jj] if trans in ("N", "n") else band[i, ku + jj - i]
    R = np.empty_like(F)
    idx = np.clip(np.arange(n)[:, None] - lo + np.arange(W)[None, :], 0, n - 1)
    valid = (np.arange(n)[:, None] - lo + np.arange(W)[None, :] >= 0) & \
            (np.arange(n)[:, None] - lo + np.arange(W)[None, :] < n)
    for c in range(X.shape[0]):
        xw = np.where(valid, X[c][idx], 0.0)
        p, e = _two_product(Aop, xw)
        for i in range(n):
            R[c, i] = math.fsum([F[c, i]] + list(-p[i]) + list(-e[i]))
    return R
