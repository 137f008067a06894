"""The benchmark's flop accounting (the numerator of its roofline figures) against the paper's
per-partition operation counts (no GPU needed).

Table tab:sweeps and Table Computation_Cost_Table (Sec. 2.3, 3.3): every partition is factored
once; the first and last partitions need no full sweep in the factorization stage and two per
solve; inner partitions, single blocks or SPIKE 2x2 pairs alike, need three full sweeps over the
k spike columns in the factorization and four per solve.  A full sweep of a triangular factor
with k off-diagonals over c vectors on n_i rows is 2 n_i k c flops, and a band LU with
kl = ku = k is n_i (2k^2 + k).  The accounting may add only the truncated tip sweeps and the
reduced system on top of these leading terms.
"""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1811_03559_gb300 import spike  # noqa: E402


def table_counts(offs, flags, k, m):
    """Leading flop terms from the paper's tables, one entry per partition (a 2x2 pair is one)."""
    sizes = np.diff(offs).astype(np.float64)
    parts, i = [], 0
    while i < len(sizes):
        if flags[i] & 2:  # top half of a SPIKE 2x2 pair: the partition spans both leaves
            parts.append(sizes[i] + sizes[i + 1])
            i += 2
        else:
            parts.append(sizes[i])
            i += 1
    lu = sum(ni * (2 * k * k + k) for ni in parts)
    fsweeps = sum(3 * 2 * ni * k * k for ni in parts[1:-1])
    ssweeps = sum((2 if j in (0, len(parts) - 1) else 4) * 2 * ni * k * m for j, ni in enumerate(parts))
    return lu, fsweeps, ssweeps


@pytest.mark.parametrize("n,k,p,m", [(1 << 20, 128, 148, 64), (1 << 20, 128, 64, 1), (1 << 20, 32, 192, 64),
                                     (200_000, 16, 9, 8)])
def test_method_flops_follow_the_sweep_tables(n, k, p, m):
    _, offs, flags = spike.plan(n, k, k, p, nrhs_hint=m, stage_balance=True)
    f = bench.method_flops(offs, flags, k, m)
    lu, fsweeps, ssweeps = table_counts(offs, flags, k, m)
    nb = len(offs) - 1
    # block LU + the factorization's spike sweeps: the tables' terms plus, per block, the diagonal
    # scaling of the spike columns (2k per row) and truncated tip sweeps (a few k^3)
    extra = f["block_lu"] - (lu + fsweeps)
    assert 0 <= extra <= 2 * k * n + 4 * nb * k ** 3
    # each solve: the tables' sweeps plus the tip products and the reduced system, a few per cent
    for key in ("solve_n", "solve_t"):
        assert ssweeps <= f[key] <= 1.05 * ssweeps + 8 * nb * k * k * m * np.log2(max(nb, 2)), key
    assert f["step"] == pytest.approx(f["factor"] + f["solve_n"] + f["solve_t"])


def test_two_partitions_do_the_work_of_one_lu():
    """With only a first and a last partition, SPIKE performs as many full sweeps as a banded LU
    factorization and solve (the remark after Table tab:sweeps): no sweeps in the factorization,
    two per solve, over all n rows."""
    n, k, m = 100_000, 8, 4
    _, offs, flags = spike.plan(n, k, k, 2, nrhs_hint=m)
    assert len(offs) == 3
    lu, fsweeps, ssweeps = table_counts(offs, flags, k, m)
    assert fsweeps == 0 and ssweeps == 2 * 2 * n * k * m
    f = bench.method_flops(offs, flags, k, m)
    assert f["block_lu"] - lu <= 4 * 2 * k ** 3


def _gepp_flops_brute(nl, k):
    """Flops of an unblocked banded GEPP on nl rows whose U fills to 2k superdiagonals: per column,
    one multiply per multiplier (the rows below within k) and one FMA (2 flops) per update of (row
    below, column to the right within 2k) -- counted by walking the columns."""
    f = 0
    for j in range(nl):
        below = min(k, nl - 1 - j)
        right = min(2 * k, nl - 1 - j)
        f += below + 2 * below * right
    return f


def test_pivot_block_flops_leading_terms():
    """bench.pivot_block_flops: the GEPP term is 4k^2 + k flop per row (the brute-force count
    above, up to the end rows where fewer rows remain below and to the right), middle blocks add
    2k^2 (L sweep of the top spike, k columns) + 8k^2 (U sweep of both spikes, 2k columns and 2k
    superdiagonals) per row, and each end block adds 8k^3 for its truncated sweeps."""
    k = 8
    offs = np.array([0, 300, 700, 1100, 1400])
    got = bench.pivot_block_flops(offs, k)
    sizes = np.diff(offs)
    want = sum(s * (4 * k * k + k) for s in sizes) + sum(s * 10 * k * k for s in sizes[1:-1]) + 2 * 8 * k ** 3
    assert got == pytest.approx(want, rel=1e-12)
    # the GEPP term agrees with the brute-force count to within the end effects (< 2k rows' worth)
    for s in sizes:
        brute = _gepp_flops_brute(int(s), k)
        assert s * (4 * k * k + k) - brute <= 2 * k * (4 * k * k + k)
        assert brute <= s * (4 * k * k + k)
