"""Exact rational Gaussian elimination for tiny integer systems -- TEST INFRASTRUCTURE ONLY.

Pins the banded oracle to arithmetic with no rounding at all: an n <= 16 system
with integer entries is solved in fractions.Fraction, so the FP64 oracle's
error can be measured against the true solution op(A)^{-1} F.
"""
from fractions import Fraction


def solve_exact(A, F, trans="N"):
    """A: list-of-lists / array of ints (n x n); F: list of n ints (one RHS).
    Returns the exact solution as a list of Fractions, or None if A is singular."""
    n = len(A)
    M = [[Fraction(int(A[i][j]) if trans == "N" else int(A[j][i])) for j in range(n)] + [Fraction(int(F[i]))]
         for i in range(n)]
    for c in range(n):
        p = next((r for r in range(c, n) if M[r][c] != 0), None)
        if p is None:
            return None
        M[c], M[p] = M[p], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    return [M[i][n] / M[i][i] for i in range(n)]
