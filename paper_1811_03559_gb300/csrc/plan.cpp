// Partition planner: worker count -> partitions, 2x2 pairs and block sizes.
//
// Sec. 3.1 (thread distribution): with t workers, P = 2^m partitions where
// 2^m <= t; r = t - 2^m inner partitions receive two workers and run as a
// SPIKE 2x2 pair (LU on the top half, UL on the bottom half, Sec. 2.3/3.2),
// allocated in order from the second partition.  The first and last
// partitions always keep one worker, so r <= P - 2 and t = 2^(m+1) - 1 runs
// as 2^(m+1) - 2 (the paper's "seven threads are distributed as six").
//
// Sec. 3.3 (load balancing): first/last partitions have size n1, 2x2
// partitions n2 = 2 n3, single inner partitions n3, with
//   R13 = n1/n3 = (1 + 1.5 K + 2 K rho) / (1 + K rho),  rho = n_rhs / k,
//   R12 = n1/n2 = R13 / 2
// (Eq. R13_calculation, restated over a common denominator; the limits are
// Eq. ratiof R12 = 1/2 + 3K/4 as rho -> 0 and Eq. ratios R12 = 1, R13 = 2 as
// rho -> infinity), and n = 2 n1 + x n2 + y n3 with x = r pairs and y = P-2-r
// single inner partitions, solved for n1, n2, n3.
//
// With SPIKE_FLAG_STAGE_BALANCE the ratio is instead the paper's solve-stage limit
// R13 = 2 (or its factorization limit when no solve is expected), which balances
// each stage separately (see spike.h); an explicit R13 (options.R13 > 0) overrides both.
//
// Readings where the paper is silent: sizes are floored, the remainder rows go
// one at a time to the inner partitions starting at the second one; a 2x2
// partition is split floor/ceil; every factored block must have at least 2k
// rows (so its top and bottom k-row tips do not overlap), otherwise t is
// lowered until they do.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace spk {

static void build_levels(Plan &pl, const std::vector<int> &part_first_leaf) {
  pl.levels.clear();
  const int P = pl.P;
  // groups as leaf ranges
  std::vector<std::pair<int, int>> groups;
  if (pl.r > 0) {
    std::vector<Merge> lv0;
    for (int i = 0; i < P; ++i) {
      int a = part_first_leaf[i];
      int c = part_first_leaf[i + 1];
      if (c - a == 2) lv0.push_back(Merge{a, a + 1, c, 0, 0});
    }
    pl.levels.push_back(lv0);
  }
  for (int i = 0; i < P; ++i) groups.push_back({part_first_leaf[i], part_first_leaf[i + 1]});
  while (groups.size() > 1) {
    std::vector<Merge> lv;
    std::vector<std::pair<int, int>> next;
    for (size_t g = 0; g + 1 < groups.size(); g += 2) {
      lv.push_back(Merge{groups[g].first, groups[g].second, groups[g + 1].second, 0, 0});
      next.push_back({groups[g].first, groups[g + 1].second});
    }
    pl.levels.push_back(lv);
    groups = next;
  }
  for (auto &lv : pl.levels)
    for (auto &mg : lv) {
      mg.hasV = (mg.c != pl.nleaves) ? 1 : 0;
      mg.hasW = (mg.a != 0) ? 1 : 0;
    }
}

int make_plan(int64_t n, int kl, int ku, int t, double K, int nrhs_hint, int flags, double r13, Plan &pl) {
  if (n < 1) return -1;
  if (kl < 0) return -2;
  if (ku < 0) return -3;
  if (t < 1) return -4;
  if (n > 1 && (int64_t)kl >= n) return -2;
  if (n > 1 && (int64_t)ku >= n) return -3;
  pl = Plan();
  pl.n = n;
  pl.kl = kl;
  pl.ku = ku;
  pl.k = std::max(1, std::max(kl, ku));
  if (pl.k > SPIKE_MAX_K) return SPIKE_ENOTSUP;
  pl.t_req = t;
  pl.K = (K > 0) ? K : 2.0;
  const double rho = (nrhs_hint > 0) ? (double)nrhs_hint / pl.k : 0.0;
  pl.R13 = (1.0 + 1.5 * pl.K + 2.0 * pl.K * rho) / (1.0 + pl.K * rho);
  if (flags & SPIKE_FLAG_STAGE_BALANCE) pl.R13 = (rho > 0.0) ? 2.0 : 1.0 + 1.5 * pl.K;
  if (r13 > 0.0) pl.R13 = r13;
  pl.R12 = pl.R13 / 2.0;
  const int64_t k = pl.k;

  for (int tt = t; tt >= 1; --tt) {
    int m = 0;
    while ((2LL << m) <= tt) ++m;
    const int P = 1 << m;
    int r = tt - P;
    if (r > P - 2) r = std::max(P - 2, 0);
    std::vector<int64_t> sizes(P, 0);
    int64_t n1 = n, n2 = 0, n3 = 0;
    if (P >= 2) {
      const int x = r, y = P - 2 - r;
      const double D = 2.0 * pl.R12 * pl.R13 + x * pl.R13 + y * pl.R12;
      n1 = (int64_t)std::floor((double)n * pl.R12 * pl.R13 / D);
      n2 = (int64_t)std::floor((double)n * pl.R13 / D);
      n3 = (int64_t)std::floor((double)n * pl.R12 / D);
      for (int i = 0; i < P; ++i) sizes[i] = (i == 0 || i == P - 1) ? n1 : (i <= r ? n2 : n3);
      int64_t rem = n;
      for (int i = 0; i < P; ++i) rem -= sizes[i];
      int i = (P > 2) ? 1 : 0;
      while (rem > 0) {
        sizes[i] += 1;
        --rem;
        if (P > 2) i = (i + 1 <= P - 2) ? i + 1 : 1;
        else i = (i + 1) % P;
      }
    } else {
      sizes[0] = n;
    }
    // leaves
    std::vector<Leaf> leaves;
    std::vector<int> first_leaf(P + 1, 0);
    int64_t pos = 0;
    bool ok = true;
    for (int i = 0; i < P; ++i) {
      first_leaf[i] = (int)leaves.size();
      const bool split = (P >= 2) && (i >= 1) && (i <= r);
      if (split) {
        int64_t top = sizes[i] / 2, bot = sizes[i] - top;
        leaves.push_back(Leaf{pos, top, 0, 0, 0, i, 1});
        leaves.push_back(Leaf{pos + top, bot, 1, 0, 0, i, 2});
      } else {
        leaves.push_back(Leaf{pos, sizes[i], (P >= 2 && i == P - 1) ? 1 : 0, 0, 0, i, 0});
      }
      pos += sizes[i];
    }
    first_leaf[P] = (int)leaves.size();
    const int nl = (int)leaves.size();
    for (int b = 0; b < nl; ++b) {
      leaves[b].has_prev = b > 0;
      leaves[b].has_next = b + 1 < nl;
      if (nl > 1 && leaves[b].len < 2 * k) ok = false;
      if (leaves[b].len < 1) ok = false;
    }
    if (!ok && tt > 1) continue;
    if (!ok) return -1;  // unreachable: tt == 1 gives a single block of n >= 1 rows
    pl.t_eff = P + r;
    pl.m = m;
    pl.P = P;
    pl.r = r;
    pl.nleaves = nl;
    pl.n1 = n1;
    pl.n2 = n2;
    pl.n3 = n3;
    pl.leaves = leaves;
    build_levels(pl, first_leaf);
    return 0;
  }
  return -4;
}

// Partition-range sharding (the SPIKE-MPI direction of Sec. 3 with the recursion of Sec. 2.2):
// rank g of nranks owns partitions [g P / nranks, (g + 1) P / nranks) of the plan, i.e. a
// contiguous power-of-two range of the 2^m partitions with the 2x2 pairs inside them.  The
// pair level and the first log2(P / nranks) power-of-two levels merge groups inside one rank;
// the remaining log2(nranks) levels merge groups of several ranks.  Returns 0, or -1 when
// nranks is not a power of two between 1 and P.
int shard_ranges(const Plan &pl, int nranks, std::vector<int> &leaf_first, int &local_levels) {
  if (nranks < 1 || (nranks & (nranks - 1)) != 0 || nranks > pl.P) return -1;
  const int per = pl.P / nranks;
  leaf_first.assign(nranks + 1, pl.nleaves);
  for (int g = 0; g < nranks; ++g) {
    for (int i = 0; i < pl.nleaves; ++i)
      if (pl.leaves[i].part >= g * per) {
        leaf_first[g] = i;
        break;
      }
  }
  leaf_first[nranks] = pl.nleaves;
  int lg = 0;
  while ((1 << lg) < per) ++lg;
  local_levels = (pl.r > 0 ? 1 : 0) + lg;
  return 0;
}

}  // namespace spk
