"""Error metrics for banded solves -- TEST INFRASTRUCTURE ONLY.

Norms are infinity norms taken per right-hand-side column, and the reported
value is the maximum over columns:
  backward error  ||op(A) x - f|| / (||op(A)|| * ||x||)   (residual in FP64 from the original band)
  forward error   ||x - x_ref|| / ||x_ref||
The paper reports "relative residuals" without naming a norm (Sec. 3.4); the
infinity norm is the reading used here.
"""
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
