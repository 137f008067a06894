"""1-norm condition estimate of a band matrix -- TEST INFRASTRUCTURE ONLY.

Stands in for LAPACK DGBCON, which the paper uses to report the condition of
its pivoting test matrices (Sec. 5.3).  Method: Hager's (1984) estimate of
||A^{-1}||_1 by maximising ||A^{-1} x||_1 over the unit 1-norm ball with a
gradient step (one solve with A and one with A^T per step), plus Higham's
(1988) alternating-sign test vector as a safeguard.  The solves are the
oracle's banded GEPP solves.
"""
import numpy as np

from . import BandLU


def band_norm_1(band, kl, ku):
    n = band.shape[0]
    tot = np.zeros(n)
    for d in range(kl + ku + 1):
        i = np.arange(n) + d - ku
        ok = (i >= 0) & (i < n)
        tot += np.where(ok, np.abs(band[:, d]), 0.0)
    return float(tot.max())


def inv_norm_1_estimate(lu, max_iter=5):
    n = lu.n
    x = np.full(n, 1.0 / n)
    est = 0.0
    jlast = -1
    for _ in range(max_iter):
        y = lu.solve(x, "N")
        est_new = float(np.abs(y).sum())
        if est_new <= est and jlast >= 0:
            break
        est = est_new
        xi = np.where(y >= 0, 1.0, -1.0)
        z = lu.solve(xi, "T")
        j = int(np.argmax(np.abs(z)))
        if np.abs(z).max() <= float(z @ x):
            break
        x = np.zeros(n)
        x[j] = 1.0
        jlast = j
    # Higham's safeguard vector b_i = (-1)^i (1 + i/(n-1))
    i = np.arange(n)
    b = (-1.0) ** i * (1.0 + i / max(n - 1, 1))
    alt = 2.0 * float(np.abs(lu.solve(b, "N")).sum()) / (3.0 * n)
    return max(est, alt)


def cond1_estimate(band, kl, ku):
    """Estimated kappa_1(A) = ||A||_1 * est(||A^{-1}||_1); inf if A is singular."""
    lu = BandLU(band, kl, ku)
    if lu.info != 0:
        return float("inf")
    return band_norm_1(band, kl, ku) * inv_norm_1_estimate(lu)
