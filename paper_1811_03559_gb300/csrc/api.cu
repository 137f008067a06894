// C ABI of libspike.so: handle lifecycle, workspace and the launch pipelines of
// the factorization (Sec. 2.1-2.3, 3, 5) and of the N / T solves (Sec. 2.1, 2.2, 4).
//
// Frames: every vector (F, X, the scratch H and the reduced right-hand sides Y)
// is stored in the GLOBAL row order; each leaf kernel reads its block through a
// view whose row stride is -1 for the reversed (UL) blocks.  Spike tips and the
// reduced unknowns are always in global orientation.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

using namespace spk;

namespace spk {
static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[16] = {};

static cudaMemPool_t lib_pool(int dev) {
  std::lock_guard<std::mutex> g(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = pool;
  }
  return g_pools[dev];
}

cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t s) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) {
    cudaGetLastError();
    return cudaMallocAsync(p, bytes, s);
  }
  cudaMemPool_t pool = lib_pool(dev);
  if (!pool) return cudaMallocAsync(p, bytes, s);
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}
}  // namespace spk

extern "C" int spike_release_cached(int64_t *reserved_before, int64_t *reserved_after) {
  if (reserved_before) *reserved_before = 0;
  if (reserved_after) *reserved_after = 0;
  std::lock_guard<std::mutex> g(spk::g_pool_mu);
  uint64_t before = 0, after = 0;
  for (int dev = 0; dev < 16; ++dev) {
    cudaMemPool_t pool = spk::g_pools[dev];
    if (!pool) continue;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(dev);
    if (cudaDeviceSynchronize() != cudaSuccess) {
      cudaSetDevice(cur);
      return SPIKE_ECUDA;
    }
    uint64_t v = 0;
    cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &v);
    before += v;
    cudaMemPoolTrimTo(pool, 0);
    cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &v);
    after += v;
    cudaSetDevice(cur);
  }
  if (reserved_before) *reserved_before = (int64_t)before;
  if (reserved_after) *reserved_after = (int64_t)after;
  return 0;
}

namespace {

thread_local std::string g_cuda_err;

#define SP_CUDA(x)                                                       \
  do {                                                                   \
    cudaError_t e_ = (cudaError_t)(x);                                   \
    if (e_ != cudaSuccess) {                                             \
      g_cuda_err = std::string(#x) + ": " + cudaGetErrorString(e_);      \
      return SPIKE_ECUDA;                                                \
    }                                                                    \
  } while (0)

#define SP_TRY(x)                      \
  do {                                 \
    int r_ = (x);                      \
    if (r_ != 0) return r_;            \
  } while (0)

constexpr uint32_t kMagic = 0x5350494bu;  // "SPIK"
constexpr double kBoostEps = 1.4901161193847656e-08;  // 2^-26: boost threshold relative to max|a_ij|

// Host-side arena of descriptors: everything a pipeline launches is laid out
// here, uploaded once, and referenced by offset.
struct Arena {
  std::vector<char> h;
  template <typename T>
  size_t put(const std::vector<T> &v) {
    size_t off = (h.size() + 255) & ~size_t(255);
    h.resize(off + v.size() * sizeof(T));
    if (!v.empty()) memcpy(h.data() + off, v.data(), v.size() * sizeof(T));
    return off;
  }
};

// A batch of GEMM descriptors with tile bookkeeping.  The tile size is chosen when the
// batch is launched: 64 x 64 when that gives at least one tile per SM, else 32 x 32 or
// 16 x 16 (an SM retires ~2 FP64 FMAs per clock, so a few large tiles leave the GPU idle).
struct GemmBatch {
  std::vector<GemmDesc> d;
  int tiles = 0, tsz = 64;
  void add(GemmDesc g) {
    if (g.M <= 0 || g.N <= 0) return;
    d.push_back(g);
  }
  // Batches whose products all have N <= 8 columns (few right-hand sides) use 256-row
  // tiles of 1, 4 or 8 columns instead (tsz = -columns).
  void finalize(int sms) {
    auto count = [&](int t) {
      long long c = 0;
      for (auto &g : d) c += (long long)((g.M + t - 1) / t) * ((g.N + t - 1) / t);
      return c;
    };
    int maxn = 0;
    for (auto &g : d) maxn = std::max(maxn, g.N);
    int tm, tn;
    if (maxn <= 8) {
      tn = maxn <= 1 ? 1 : (maxn <= 4 ? 4 : 8);
      tm = 256;
      tsz = -tn;
    } else {
      tsz = count(64) >= sms ? 64 : (count(32) >= sms ? 32 : 16);
      tm = tn = tsz;
    }
    tiles = 0;
    for (auto &g : d) {
      g.tiles_n = (g.N + tn - 1) / tn;
      g.tile0 = tiles;
      tiles += ((g.M + tm - 1) / tm) * g.tiles_n;
    }
  }
};

GemmDesc gd(const double *A, int64_t a_rs, int64_t a_cs, const double *B, int64_t b_rs, int64_t b_cs,
            const double *C0, int64_t c0_rs, int64_t c0_cs, double *C, int64_t c_rs, int64_t c_cs, int M, int N,
            int K, double alpha, double beta) {
  GemmDesc g;
  memset(&g, 0, sizeof(g));
  g.A = A;
  g.a_rs = a_rs;
  g.a_cs = a_cs;
  g.B = B;
  g.b_rs = b_rs;
  g.b_cs = b_cs;
  g.C0 = C0;
  g.c0_rs = c0_rs;
  g.c0_cs = c0_cs;
  g.C = C;
  g.c_rs = c_rs;
  g.c_cs = c_cs;
  g.M = M;
  g.N = N;
  g.K = K;
  g.alpha = alpha;
  g.beta = beta;
  return g;
}

struct TrsBatch {
  std::vector<TrsDesc> d;
  int tiles = 0, maxn = 0;
  void add(const double *lu, const int *ipiv, int n, int lda, double *b, int64_t ldb, int ncols, int trans,
           double alpha) {
    if (ncols <= 0) return;
    TrsDesc t;
    memset(&t, 0, sizeof(t));
    t.lu = lu;
    t.ipiv = ipiv;
    t.n = n;
    t.lda = lda;
    t.b = b;
    t.ldb = ldb;
    t.ncols = ncols;
    t.trans = trans;
    t.alpha = alpha;
    maxn = std::max(maxn, n);
    d.push_back(t);
  }
  // right-hand-side columns per CTA: 16, or 4 when 16-column tiles would not fill the GPU
  int cols = 16;
  void finalize(int sms) {
    long long c16 = 0;
    for (auto &t : d) c16 += (t.ncols + 15) / 16;
    cols = c16 >= sms ? 16 : 4;
    tiles = 0;
    for (auto &t : d) {
      t.tile0 = tiles;
      tiles += (t.ncols + cols - 1) / cols;
    }
  }
};

}  // namespace

// A solve captured as a CUDA graph (SPIKE_FLAG_GRAPHS): replayed when the same call
// (columns, trans, right-hand-side buffer, scratch) comes again.
struct GraphEntry {
  int m = 0, tr = 0;
  const double *F = nullptr;
  int64_t ld = 0;
  const char *scratch = nullptr;
  cudaGraphExec_t exec = nullptr;
  char *args = nullptr;  // the graph's own copy of the descriptor arena
  uint64_t last = 0;
};

struct spike_ctx {
  uint32_t magic = kMagic;
  Plan pl;
  int k = 0, ldf = 0, dofs = 0, pivot = 0, NL = 0, nleaves = 0;
  cudaStream_t stream = nullptr;
  // persistent device memory (one allocation, carved)
  char *mem = nullptr;
  size_t mem_bytes = 0;
  char *fbc = nullptr, *dinvc = nullptr;  // leaf factors / reciprocals, element size es
  double *couple = nullptr, *spk = nullptr, *mlu = nullptr, *ident = nullptr;
  int f32 = 0;                             // SPIKE_FLAG_MIXED: FP32 leaf factors and sweeps
  int invariant = 0;                       // SPIKE_FLAG_BATCH_INVARIANT
  int graphs = 0;                          // SPIKE_FLAG_GRAPHS
  std::vector<GraphEntry> gcache;          // captured solves (at most kGraphCache)
  std::vector<GraphEntry> gseen;           // calls seen once (captured on their second use)
  uint64_t gtick = 0;
  int64_t graph_captures = 0, graph_replays = 0;
  int in_solve = 0;                        // descriptors being built belong to a solve
  size_t es = sizeof(double);
  double *band64 = nullptr;                // mixed: FP64 copy of the band for the refinement residuals
  int64_t ldab64 = 0;
  // mixed: op(A) split into int8 digit fragments for the tensor-core residual (resid_split.cu),
  // [0] = N (rows of A), [1] = T (rows of A^T); null when the FP64 residual is used
  void *sfrag[2] = {nullptr, nullptr};
  int *srexp[2] = {nullptr, nullptr};
  unsigned long long *snorm = nullptr;     // ||A||_inf, ||A^T||_inf (bit patterns)
  double refine_tol = SPIKE_MIXED_TOL;     // mixed: per-column stopping backward error
  int last_iters = 0;                      // mixed: refinement steps of the last solve
  double last_berr = 0.0;                  //        and its final backward error
  int *ipiv = nullptr, *mpiv = nullptr;
  unsigned long long *status = nullptr;
  std::vector<LeafDev> hl;
  std::vector<int64_t> merge_off;         // first merge index of each level
  std::vector<std::vector<int>> schur;    // per level, per merge: 1 = Schur-complement path
  int total_merges = 0;
  int64_t boosts = 0, zero_col = 0;
  int nan_flag = 0;                        // SPIKE_NUMERICS_* bits of the factorization
  // solve scratch (grown on demand)
  char *scr = nullptr;
  size_t scr_bytes = 0;
  char *dargs = nullptr;
  size_t dargs_bytes = 0;
  // partition-range sharding (spike_shard_factor): this rank owns leaves [l0, l1), rows
  // [row0, row0 + nrow); its factors, work arrays and right-hand sides hold only those rows
  // (their base pointers are offset by -row0 so that kernels index them by global row).
  // Spike tips and reduced unknowns keep the global leaf numbering.  The first `lvl` merge
  // levels lie inside the rank; the others are run one per exchange (sh_op, sh_level).
  int shard = 0, rank = 0, nranks = 1, l0 = 0, l1 = 0, lvl = 0;
  int64_t row0 = 0, nrow = 0;
  std::vector<int> leaf_first;             // nranks + 1 leaf boundaries
  int sh_op = 0;                           // pending exchange: SH_* below
  int sh_level = 0;
  char *sh_fscr = nullptr;                 // factor scratch kept until the coarse levels are done
  size_t sh_tmp_off = 0, sh_tmp_bytes = 0;
  double *sh_F = nullptr;                  // the solve's own rows of F
  int64_t sh_ld = 0;
  int sh_m = 0;
  // stage timing (SPIKE_FLAG_TIMING): boundary events of the last factor / N solve / T solve
  bool timing = false;
  cudaEvent_t fev[5] = {}, nev[4] = {}, tev[4] = {};
  bool fdone = false, ndone = false, tdone = false;
};

static bool valid(spike_handle h) { return h && h->magic == kMagic; }

static int ensure(char **p, size_t *cap, size_t need, cudaStream_t s) {
  if (need <= *cap) return 0;
  if (*p) SP_CUDA(cudaFreeAsync(*p, s));
  *p = nullptr;
  *cap = 0;
  size_t want = need + need / 4 + 4096;
  cudaError_t e = dev_alloc((void **)p, want, s);
  if (e != cudaSuccess) {
    g_cuda_err = std::string("cudaMallocAsync: ") + cudaGetErrorString(e);
    *p = nullptr;
    return SPIKE_ENOMEM;
  }
  *cap = want;
  return 0;
}

static bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The device address of page-locked host memory mapped into the device's address space
// (cudaHostAlloc / cudaMallocHost, or cudaHostRegister with the mapped flag), else null:
// kernels may read such a buffer in place over the host link.  Pageable memory gives null.
static const void *mapped_host_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// pointer into the spike-tip store: level lv, spike s (0 V, 1 W), leaf i, tip t (0 top, 1 bottom)
static inline double *TIP(spike_ctx *c, int lv, int s, int i, int t) {
  return c->spk + tip_index(lv, s, i, t, c->nleaves, c->k);
}

static void fill_info(const Plan &pl, spike_info *o) {
  memset(o, 0, sizeof(*o));
  o->n = pl.n;
  o->kl = pl.kl;
  o->ku = pl.ku;
  o->k = pl.k;
  o->p_requested = pl.t_req;
  o->p_effective = pl.t_eff;
  o->m = pl.m;
  o->P = pl.P;
  o->r = pl.r;
  o->leaves = pl.nleaves;
  o->levels = (int)pl.levels.size();
  o->pivot = pl.pivot;
  o->n1 = pl.n1;
  o->n2 = pl.n2;
  o->n3 = pl.n3;
  o->R12 = pl.R12;
  o->R13 = pl.R13;
  o->K = pl.K;
}

static int map_plan_rc(int rc) {
  // make_plan: -1 n, -2 kl, -3 ku, -4 t  ->  ABI argument positions of spike_factor_ex
  switch (rc) {
    case -1: return -3;
    case -2: return -4;
    case -3: return -5;
    case -4: return -6;
    default: return rc;
  }
}

extern "C" int spike_plan(int64_t n, int kl, int ku, int p, const spike_options *opt, spike_info *out,
                          int64_t *leaf_offsets, int32_t *leaf_flags) {
  if (!out) return -6;
  Plan pl;
  const int rc = make_plan(n, kl, ku, p, opt ? opt->K : 0.0, opt ? opt->nrhs_hint : 0, opt ? opt->flags : 0,
                     opt ? opt->R13 : 0.0, pl);
  if (rc != 0) return rc;  // -1 n, -2 kl, -3 ku, -4 p, or SPIKE_ENOTSUP
  fill_info(pl, out);
  for (int i = 0; i < pl.nleaves; ++i) {
    if (leaf_offsets) leaf_offsets[i] = pl.leaves[i].start;
    if (leaf_flags)
      leaf_flags[i] = (pl.leaves[i].rev ? 1 : 0) | (pl.leaves[i].half == 1 ? 2 : 0) | (pl.leaves[i].half == 2 ? 4 : 0);
  }
  if (leaf_offsets) leaf_offsets[pl.nleaves] = n;
  return 0;
}

extern "C" int spike_shard_plan(int64_t n, int kl, int ku, int p, int nranks, const spike_options *opt,
                                int64_t *row_first, int32_t *leaf_first, int32_t *local_levels) {
  if (!row_first) return -7;
  if (!leaf_first) return -8;
  if (!local_levels) return -9;
  Plan pl;
  const int rc = make_plan(n, kl, ku, p, opt ? opt->K : 0.0, opt ? opt->nrhs_hint : 0, opt ? opt->flags : 0,
                           opt ? opt->R13 : 0.0, pl);
  if (rc != 0) return rc;
  std::vector<int> lf;
  int ll = 0;
  if (shard_ranges(pl, nranks, lf, ll) != 0) return -5;
  for (int g = 0; g <= nranks; ++g) {
    leaf_first[g] = lf[g];
    row_first[g] = (lf[g] < pl.nleaves) ? pl.leaves[lf[g]].start : n;
  }
  *local_levels = ll;
  return 0;
}

// a strided view: element (local row r, column c) at p[r*rs + c*cs]
struct View {
  double *p;
  int64_t rs, cs;
};

static SweepDesc sdesc(spike_ctx *c, int i, int kind, int r0, int r1, int ncols, View g, const double *gb,
                       View gbv, double gbs, View x) {
  const LeafDev &L = c->hl[i];
  SweepDesc d;
  memset(&d, 0, sizeof(d));
  d.fb = (const double *)(c->fbc + L.start * (int64_t)c->ldf * c->es);
  d.dinv = (const double *)(c->dinvc + L.start * (int64_t)c->es);
  d.ipiv = c->ipiv ? c->ipiv + L.start : nullptr;
  d.nl = L.len;
  d.r0 = r0;
  d.r1 = r1;
  d.ncols = ncols;
  d.kind = kind;
  d.kw = (kind == UN || kind == UT) ? c->dofs : c->k;  // U has 2k superdiagonals when pivoting
  d.fixed_split = (c->invariant && c->in_solve) ? 1 : 0;
  d.ldf = c->ldf;
  d.dofs = c->dofs;
  d.ga = g.p;
  d.ga_rs = g.rs;
  d.ga_cs = g.cs;
  d.gb = gb;
  d.gb_rs = gbv.rs;
  d.gb_cs = gbv.cs;
  d.gb_scale = gbs;
  d.x = x.p;
  d.x_rs = x.rs;
  d.x_cs = x.cs;
  return d;
}

static SweepDesc empty_sweep() {
  SweepDesc d;
  memset(&d, 0, sizeof(d));
  return d;
}

static std::vector<SweepDesc> e0_dummy(int n) { return std::vector<SweepDesc>(n, empty_sweep()); }

// A step of a solve, recorded instead of launched when several systems are solved
// together (spike_solve_batch): steps with the same key from different systems are
// merged into one launch.  Keys are (section, level, step), increasing in each system's
// own order, so merging in key order keeps every system's order.
struct PhaseKey {
  int a, b, c;
  bool operator<(const PhaseKey &o) const {
    if (a != o.a) return a < o.a;
    if (b != o.b) return b < o.b;
    return c < o.c;
  }
};
struct Phase {
  int kind = 0;  // 0 plain ops (no descriptors), 1 sweep stage, 2 GEMM, 3 LU solve, 4 block sums
  std::vector<std::function<int(char *)>> ops;
  std::vector<SweepDesc> a, b;
  int a_piv = -1, b_piv = -1, k = 0;
  GemmBatch g;
  TrsBatch t;
  std::vector<SumDesc> sums;
  int64_t maxe = 0;
};

// Upload an arena and run the recorded launches.  With rec != nullptr every call is
// instead appended to *rec as a Phase under the current key (empty ones too, so that
// systems of the same kind record the same key sequence).
struct Pipeline {
  cudaStream_t st = nullptr;
  int f32 = 0;  // sweep storage precision
  Arena ar;
  std::vector<std::function<int(char *)>> ops;
  std::map<PhaseKey, Phase> *rec = nullptr;
  int ka = 0, kb = 0, kc = 0;
  // Zeroed-per-launch device counters for sweep stages with more blocks than SMs (merged
  // batches): their tasks are sorted largest first and taken by persistent CTAs.
  unsigned int *queue_base = nullptr;
  int nqueue = 0, max_queue = 0;
  void key(int a, int b) {
    ka = a;
    kb = b;
    kc = 0;
  }
  Phase &next(int kind) {
    Phase &ph = (*rec)[PhaseKey{ka, kb, kc++}];
    ph.kind = kind;
    return ph;
  }
  void op(std::function<int(char *)> f) {
    if (rec) next(0).ops.push_back(f);
    else ops.push_back(f);
  }
  int run(spike_ctx *c) {
    if (!ar.h.empty()) {
      SP_TRY(ensure(&c->dargs, &c->dargs_bytes, ar.h.size(), c->stream));
      SP_CUDA(cudaMemcpyAsync(c->dargs, ar.h.data(), ar.h.size(), cudaMemcpyHostToDevice, c->stream));
    }
    return run_ops(c->dargs);
  }
  int run_ops(char *base) {
    for (auto &o : ops) {
      const int rc = o(base);
      if (rc != 0) {
        g_cuda_err = std::string("kernel launch: ") + cudaGetErrorString((cudaError_t)rc);
        return SPIKE_ECUDA;
      }
    }
    return 0;
  }
  void gemm(GemmBatch &b) {
    if (rec) {
      next(2).g = b;
      return;
    }
    if (b.d.empty()) return;
    b.finalize(device_sms());
    const size_t off = ar.put(b.d);
    const int nd = (int)b.d.size(), tiles = b.tiles, tsz = b.tsz;
    cudaStream_t s = st;
    ops.push_back([=](char *base) { return launch_gemm((GemmDesc *)(base + off), nd, tiles, tsz, s); });
  }
  // One stage = per leaf a first and a second sweep (a[i], b[i]; empty slots have
  // ncols == 0), run by the leaf's CTA back to back in a single launch.  Pivoted
  // L / L^T sweeps (interleaved row swaps, a_piv / b_piv = LN or LT, -1 = none) use
  // their own kernel and launch.  Descriptors carry their leaf's ldf / dofs; the
  // arguments are those of the pivoted kernel.
  void stage(std::vector<SweepDesc> &a, std::vector<SweepDesc> &b, int a_piv, int b_piv, int ldf, int dofs,
             int k) {
    if (rec) {
      Phase &ph = next(1);
      ph.a = a;
      ph.b = b;
      ph.a_piv = a_piv;
      ph.b_piv = b_piv;
      ph.k = k;
      return;
    }
    cudaStream_t s = st;
    const int nl = (int)a.size();
    auto used = [](const std::vector<SweepDesc> &v) {
      for (auto &d : v)
        if (d.ncols > 0) return true;
      return false;
    };
    const bool ua = used(a), ub = used(b);
    const int fp = f32;
    const int sms = device_sms();
    if (a_piv < 0 && b_piv < 0 && ua && ub) {
      std::vector<int> order(nl);
      for (int i = 0; i < nl; ++i) order[i] = i;
      unsigned int *q = nullptr;
      if (queue_base && nl > sms && nqueue < max_queue) {
        q = queue_base + nqueue++;
        auto cost = [](const SweepDesc &d) {
          return d.ncols > 0 ? (double)(d.r1 - d.r0) * d.ncols * (d.kw + NB) : 0.0;
        };
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return cost(a[x]) + cost(b[x]) > cost(a[y]) + cost(b[y]); });
        ops.push_back([=](char *) { return (int)cudaMemsetAsync(q, 0, sizeof(unsigned int), s); });
      }
      std::vector<SweepDesc> ab;
      for (int i : order) {
        ab.push_back(a[i]);
        ab.push_back(b[i]);
      }
      const size_t off = ar.put(ab);
      ops.push_back([=](char *base) {
        return launch_sweeps((SweepDesc *)(base + off), nl, 2, ldf, dofs, s, fp, q, sms);
      });
      return;
    }
    for (int pass = 0; pass < 2; ++pass) {
      std::vector<SweepDesc> &v = pass ? b : a;
      const int pk = pass ? b_piv : a_piv;
      if (!(pass ? ub : ua)) continue;
      const size_t off = ar.put(v);
      ops.push_back([=](char *base) {
        return pk >= 0 ? launch_piv_sweep(pk, (SweepDesc *)(base + off), nl, k, ldf, dofs, s)
                       : launch_sweeps((SweepDesc *)(base + off), nl, 1, ldf, dofs, s, fp);
      });
    }
  }
  void trs(TrsBatch &b) {
    if (rec) {
      next(3).t = b;
      return;
    }
    if (b.d.empty()) return;
    b.finalize(device_sms());
    const size_t off = ar.put(b.d);
    const int nd = (int)b.d.size(), tiles = b.tiles, maxn = b.maxn, cols = b.cols;
    cudaStream_t s = st;
    ops.push_back([=](char *base) { return launch_getrs((TrsDesc *)(base + off), nd, tiles, maxn, cols, s); });
  }
  void sums(const std::vector<SumDesc> &v, int64_t maxe) {
    if (rec) {
      Phase &ph = next(4);
      ph.sums = v;
      ph.maxe = maxe;
      return;
    }
    if (v.empty()) return;
    const size_t so = ar.put(v);
    const int nd = (int)v.size();
    cudaStream_t s = st;
    ops.push_back([=](char *base) { return launch_sum_blocks((SumDesc *)(base + so), nd, maxe, s); });
  }
  // Add a recorded phase (possibly merged from several systems) as launches.
  void emit(Phase &ph) {
    switch (ph.kind) {
      case 0:
        for (auto &o : ph.ops) ops.push_back(o);
        break;
      case 1: {
        bool any = false;
        for (auto &d : ph.a) any = any || d.ncols > 0;
        for (auto &d : ph.b) any = any || d.ncols > 0;
        if (any) stage(ph.a, ph.b, ph.a_piv, ph.b_piv, 0, 0, ph.k);
        break;
      }
      case 2:
        gemm(ph.g);
        break;
      case 3:
        trs(ph.t);
        break;
      case 4:
        sums(ph.sums, ph.maxe);
        break;
    }
  }
};

// Merge phase `src` of one system into the phase with the same key of the batch.
static void merge_phase(Phase &dst, const Phase &src) {
  dst.kind = src.kind;
  for (auto &o : src.ops) dst.ops.push_back(o);
  dst.a.insert(dst.a.end(), src.a.begin(), src.a.end());
  dst.b.insert(dst.b.end(), src.b.begin(), src.b.end());
  dst.a_piv = src.a_piv;
  dst.b_piv = src.b_piv;
  dst.k = std::max(dst.k, src.k);
  for (auto &d : src.g.d) dst.g.d.push_back(d);
  for (auto &d : src.t.d) dst.t.d.push_back(d);
  dst.t.maxn = std::max(dst.t.maxn, src.t.maxn);
  dst.sums.insert(dst.sums.end(), src.sums.begin(), src.sums.end());
  dst.maxe = std::max(dst.maxe, src.maxe);
}

// ============================================================== factor
static int factor_reduced_level(spike_ctx *c, int lv, char *tmp, size_t tmp_bytes);

// The launches of one merge level of the reduced system, for one or several systems.
struct LevelBatch {
  GemmBatch gA, gB, gC;
  std::vector<LuDesc> lus;
  TrsBatch tr;
  int maxn = 0;
  std::vector<std::function<int(char *)>> copies;
};

// Device memory of one factorization: the persistent block (owned by the handle) and
// the scratch that spike_factor uses and frees before returning.  Offsets are 256-byte
// aligned carvings of one allocation each.
struct FactorLayout {
  int k = 0, dofs = 0, ldf = 0;
  int64_t zacc = 0, maxlen = 0, nmerge = 0;
  size_t o_fb = 0, o_dinv = 0, o_b64 = 0, o_ipiv = 0, o_cpl = 0, o_spk = 0, o_mlu = 0, o_mpiv = 0, o_id = 0,
         o_st = 0, mem = 0;
  bool split = false;
  size_t o_sfrag[2] = {0, 0}, o_srexp[2] = {0, 0}, o_snorm = 0;
  size_t band_stage = 0, s_z = 0, s_zoff = 0, s_leaf = 0, s_tmp = 0, tmp_bytes = 0, scr = 0;
  std::vector<int64_t> zoff;
};

// borrow: a mixed-precision handle reads the caller's device band for its residuals
// (SPIKE_FLAG_BORROW_BAND) instead of keeping a copy.
// Mixed-precision handles form their refinement residuals on the tensor cores (resid_split.cu)
// unless SPIKE_FLAG_FP64_RESIDUAL asks for FP64 FMAs or the band is too wide for its tiles.
static bool use_split_residual(const Plan &pl, int f32, int flags) {
  return f32 && !(flags & SPIKE_FLAG_FP64_RESIDUAL) && split_supported(pl.kl, pl.ku);
}

static void factor_layout(const Plan &pl, int pivot, int f32, int64_t ldab, bool band_dev, bool borrow,
                          FactorLayout &L, int flags) {
  const int64_t n = pl.n;
  const int k = pl.k, nlv = pl.nleaves;
  const size_t es = f32 ? sizeof(float) : sizeof(double);
  const int64_t kk = (int64_t)k * k;
  L.k = k;
  L.dofs = pivot ? 2 * k : k;
  L.ldf = (L.dofs + k + 1 + 1) & ~1;
  L.zoff.assign(nlv, 0);
  L.zacc = 0;
  L.maxlen = 0;
  for (int i = 0; i < nlv; ++i) {
    L.zoff[i] = L.zacc;
    L.zacc += pl.leaves[i].len * 2 * (int64_t)k;
    L.maxlen = std::max(L.maxlen, pl.leaves[i].len);
  }
  L.nmerge = 0;
  size_t maxm = 1;
  for (auto &lv : pl.levels) {
    L.nmerge += (int64_t)lv.size();
    maxm = std::max(maxm, lv.size());
  }
  const int nspk = std::max((int)pl.levels.size(), 1);
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    size_t o = off;
    off = (off + bytes + 255) & ~size_t(255);
    return o;
  };
  L.o_fb = carve(es * (size_t)n * L.ldf);
  L.o_dinv = carve(es * (size_t)n);
  L.o_b64 = (f32 && !(borrow && band_dev)) ? carve(sizeof(double) * (size_t)n * ldab) : 0;
  L.o_ipiv = pivot ? carve(sizeof(int) * (size_t)n) : 0;
  L.o_cpl = carve(sizeof(double) * (size_t)nlv * 2 * kk);
  L.o_spk = carve(sizeof(double) * (size_t)nspk * 2 * nlv * 2 * kk);
  L.o_mlu = carve(sizeof(double) * (size_t)std::max<int64_t>(L.nmerge, 1) * 4 * kk);
  L.o_mpiv = carve(sizeof(int) * (size_t)std::max<int64_t>(L.nmerge, 1) * 2 * k);
  L.o_id = carve(sizeof(double) * (size_t)kk);
  L.o_st = carve(sizeof(unsigned long long) * 8);
  L.split = use_split_residual(pl, f32, flags);
  if (L.split) {
    for (int t = 0; t < 2; ++t) {
      L.o_sfrag[t] = carve(split_band_bytes(n, pl.kl, pl.ku));
      L.o_srexp[t] = carve(sizeof(int) * (size_t)n);
    }
    L.o_snorm = carve(sizeof(unsigned long long) * 2);
  }
  L.mem = off;
  off = 0;
  // a pageable host band is staged in an allocation of its own, freed once the setup kernels
  // have read it (a pinned one is read in place; mixed handles copy it into their FP64 band)
  L.band_stage = (band_dev || f32) ? 0 : sizeof(double) * (size_t)n * ldab;
  L.s_z = carve(es * (size_t)L.zacc);
  L.s_zoff = carve(sizeof(int64_t) * (size_t)nlv);
  L.s_leaf = carve(sizeof(LeafDev) * (size_t)nlv);
  L.tmp_bytes = sizeof(double) * maxm * 5 * kk;
  L.s_tmp = carve(L.tmp_bytes);
  L.scr = off;
}

// The partition ratio requested by opt, with the pivoting default (spike_options.R13).
static double plan_r13(const spike_options *opt, int pivot) {
  const double r13 = opt ? opt->R13 : 0.0;
  if (r13 > 0.0 || !pivot || (opt && (opt->flags & SPIKE_FLAG_STAGE_BALANCE))) return r13;
  return SPIKE_PIVOT_R13;
}

extern "C" int spike_factor_bytes(int64_t n, int kl, int ku, int p, int pivot, const spike_options *opt,
                                  int host_band, int64_t *resident, int64_t *transient) {
  if (!resident) return -8;
  if (!transient) return -9;
  if (pivot != 0 && pivot != 1) return -5;
  Plan pl;
  const int rc = make_plan(n, kl, ku, p, opt ? opt->K : 0.0, opt ? opt->nrhs_hint : 0, opt ? opt->flags : 0,
                           plan_r13(opt, pivot), pl);
  if (rc != 0) return rc;
  const int f32 = (opt && (opt->flags & SPIKE_FLAG_MIXED)) ? 1 : 0;
  if (f32 && pivot) return SPIKE_ENOTSUP;
  FactorLayout L;
  factor_layout(pl, pivot, f32, (int64_t)kl + ku + 1, host_band == 0,
                (opt && (opt->flags & SPIKE_FLAG_BORROW_BAND)) != 0, L, opt ? opt->flags : 0);
  *resident = (int64_t)L.mem;
  *transient = (int64_t)(L.scr + L.band_stage);
  return 0;
}

// A rank's part of a sharded factorization: `band` holds global band columns from col0 on.
struct ShardSpec {
  int rank, nranks;
  int64_t col0;
};

// A factorization stopped before its block LU (spike_factor_batch): the block tasks go to a
// launch shared with other systems; the rest continues from this state.
struct FactorCont {
  char *fscr = nullptr;
  LeafDev *dleaf = nullptr;
  char *zbuf = nullptr;
  int64_t *dzoff = nullptr;
  char *tmp = nullptr;
  size_t tmp_bytes = 0;
};

static int factor_impl(const double *band, int64_t ldab, int64_t n, int kl, int ku, int p, int pivot,
                       const spike_options *opt, spike_handle *out, const ShardSpec *sh,
                       std::vector<FactorTask> *tasks = nullptr, FactorCont *cont = nullptr);

extern "C" int spike_factor_ex(const double *band, int64_t ldab, int64_t n, int kl, int ku, int p, int pivot,
                               const spike_options *opt, spike_handle *out) {
  return factor_impl(band, ldab, n, kl, ku, p, pivot, opt, out, nullptr);
}

static int factor_impl(const double *band, int64_t ldab, int64_t n, int kl, int ku, int p, int pivot,
                       const spike_options *opt, spike_handle *out, const ShardSpec *sh,
                       std::vector<FactorTask> *tasks, FactorCont *cont) {
  if (!out) return -9;
  *out = nullptr;
  if (!band) return -1;
  if (n < 1) return -3;
  if (kl < 0) return -4;
  if (ku < 0) return -5;
  if (ldab < (int64_t)kl + ku + 1) return -2;
  if (p < 1) return -6;
  if (pivot != 0 && pivot != 1) return -7;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return SPIKE_ENOGPU;
  }
  Plan pl;
  int rc = make_plan(n, kl, ku, p, opt ? opt->K : 0.0, opt ? opt->nrhs_hint : 0, opt ? opt->flags : 0,
                     plan_r13(opt, pivot), pl);
  if (rc != 0) return map_plan_rc(rc);
  pl.pivot = pivot;

  spike_ctx *c = new spike_ctx();
  c->pl = pl;
  c->stream = opt ? (cudaStream_t)opt->stream : nullptr;
  c->k = pl.k;
  c->pivot = pivot;
  c->nleaves = pl.nleaves;
  c->NL = (int)pl.levels.size();
  c->timing = opt && (opt->flags & SPIKE_FLAG_TIMING);
  c->f32 = (opt && (opt->flags & SPIKE_FLAG_MIXED)) ? 1 : 0;
  c->invariant = (opt && (opt->flags & SPIKE_FLAG_BATCH_INVARIANT)) ? 1 : 0;
  c->graphs = (opt && (opt->flags & SPIKE_FLAG_GRAPHS)) ? 1 : 0;
  if (opt && opt->refine_tol > 0.0) c->refine_tol = opt->refine_tol;
  c->es = c->f32 ? sizeof(float) : sizeof(double);
  if (c->f32 && pivot) {
    delete c;
    return SPIKE_ENOTSUP;
  }
  if (c->timing) {
    for (auto &e : c->fev) cudaEventCreate(&e);
    for (auto &e : c->nev) cudaEventCreate(&e);
    for (auto &e : c->tev) cudaEventCreate(&e);
  }
  const int k = c->k, nlv = c->nleaves;
  const int64_t kk = (int64_t)k * k;
  cudaStream_t s = c->stream;

  auto fail = [&](int code) {
    spike_free(c);
    return code;
  };

  const bool band_dev = is_device_ptr(band);
  // sharded: this rank's leaves and rows; the other leaves are given no rows, so every kernel
  // over the blocks skips them, and the band is addressed by global column
  Plan plx = pl;
  if (sh) {
    if (pivot || c->f32 || !band_dev) {
      delete c;
      return SPIKE_ENOTSUP;
    }
    if (shard_ranges(pl, sh->nranks, c->leaf_first, c->lvl) != 0 || sh->rank < 0 || sh->rank >= sh->nranks) {
      delete c;
      return -9;
    }
    c->shard = 1;
    c->rank = sh->rank;
    c->nranks = sh->nranks;
    c->l0 = c->leaf_first[sh->rank];
    c->l1 = c->leaf_first[sh->rank + 1];
    c->row0 = pl.leaves[c->l0].start;
    c->nrow = ((c->l1 < pl.nleaves) ? pl.leaves[c->l1].start : n) - c->row0;
    if (sh->col0 < 0 || sh->col0 > std::max<int64_t>(0, c->row0 - pl.k)) {
      delete c;
      return -3;
    }
    for (int i = 0; i < pl.nleaves; ++i)
      if (i < c->l0 || i >= c->l1) {
        plx.leaves[i].len = 0;
        plx.leaves[i].has_prev = plx.leaves[i].has_next = 0;
        plx.leaves[i].start = c->row0;
      }
    plx.n = c->nrow;
    band = (const double *)((const char *)band - (ptrdiff_t)(sh->col0 * ldab * (int64_t)sizeof(double)));
  }
  FactorLayout FL;
  const bool borrow = c->f32 && band_dev && opt && (opt->flags & SPIKE_FLAG_BORROW_BAND);
  factor_layout(plx, pivot, c->f32, ldab, band_dev, borrow, FL, opt ? opt->flags : 0);
  c->dofs = FL.dofs;
  c->ldf = FL.ldf;
  const std::vector<int64_t> &zoff = FL.zoff;
  const int64_t zacc = FL.zacc, maxlen = FL.maxlen;
  // leaves
  c->hl.resize(nlv);
  for (int i = 0; i < nlv; ++i) {
    const Leaf &L = plx.leaves[i];
    LeafDev d;
    d.start = L.start;
    d.len = L.len;
    d.rev = L.rev;
    d.top_nbr = L.rev ? L.has_next : L.has_prev;
    d.bot_nbr = L.rev ? L.has_prev : L.has_next;
    d.pad = 0;
    c->hl[i] = d;
  }
  int64_t nmerge = 0;
  c->merge_off.resize(c->NL + 1);
  for (int lv = 0; lv < c->NL; ++lv) {
    c->merge_off[lv] = nmerge;
    nmerge += (int64_t)pl.levels[lv].size();
  }
  c->merge_off[c->NL] = nmerge;
  c->total_merges = (int)nmerge;
  c->schur.assign(c->NL, {});

  // persistent memory (layout in factor_layout)
  const int nspk = std::max(c->NL, 1);
  const size_t o_fb = FL.o_fb, o_dinv = FL.o_dinv, o_b64 = FL.o_b64, o_ipiv = FL.o_ipiv, o_cpl = FL.o_cpl,
               o_spk = FL.o_spk, o_mlu = FL.o_mlu, o_mpiv = FL.o_mpiv, o_id = FL.o_id, o_st = FL.o_st;
  c->mem_bytes = FL.mem;
  {
    cudaError_t e = dev_alloc((void **)&c->mem, c->mem_bytes, s);
    if (e != cudaSuccess) {
      g_cuda_err = std::string("cudaMallocAsync: ") + cudaGetErrorString(e);
      c->mem = nullptr;
      return fail(SPIKE_ENOMEM);
    }
  }
  // (sharded: offset by -row0 so that the kernels index the rank's rows by global row)
  c->fbc = c->mem + o_fb - (ptrdiff_t)(c->row0 * c->ldf * (int64_t)c->es);
  c->dinvc = c->mem + o_dinv - (ptrdiff_t)(c->row0 * (int64_t)c->es);
  if (c->f32) {
    c->band64 = borrow ? const_cast<double *>(band) : (double *)(c->mem + o_b64);
    c->ldab64 = ldab;
  }
  c->ipiv = pivot ? (int *)(c->mem + o_ipiv) : nullptr;
  c->couple = (double *)(c->mem + o_cpl);
  c->spk = (double *)(c->mem + o_spk);
  c->mlu = (double *)(c->mem + o_mlu);
  c->mpiv = (int *)(c->mem + o_mpiv);
  c->ident = (double *)(c->mem + o_id);
  c->status = (unsigned long long *)(c->mem + o_st);
  if (FL.split) {
    for (int t = 0; t < 2; ++t) {
      c->sfrag[t] = c->mem + FL.o_sfrag[t];
      c->srexp[t] = (int *)(c->mem + FL.o_srexp[t]);
    }
    c->snorm = (unsigned long long *)(c->mem + FL.o_snorm);
  }

  // factor-time scratch: staged band (host input), Z, per-merge temporaries
  const size_t s_z = FL.s_z, s_zoff = FL.s_zoff, s_leaf = FL.s_leaf, s_tmp = FL.s_tmp;
  const size_t tmp_bytes = FL.tmp_bytes, soff = FL.scr;
  char *fscr = nullptr;
  {
    cudaError_t e = dev_alloc((void **)&fscr, soff, s);
    if (e != cudaSuccess) {
      g_cuda_err = std::string("cudaMallocAsync: ") + cudaGetErrorString(e);
      return fail(SPIKE_ENOMEM);
    }
  }
  double *bstage = nullptr;  // staged host band
  auto fail2 = [&](int code) {
    cudaFreeAsync(fscr, s);
    if (bstage) cudaFreeAsync(bstage, s);
    return fail(code);
  };
  // Where the setup kernels read the band: device memory as given; a mixed handle's FP64 copy
  // (filled straight from host memory); pinned host memory in place, through its mapped device
  // address (the repack streams it over the host link once, with no staging buffer); otherwise
  // a staged device copy.
  const double *dband = band;
  bool band_in_b64 = false;
  if (!band_dev && c->f32) {
    if (cudaMemcpyAsync(c->band64, band, sizeof(double) * (size_t)n * ldab, cudaMemcpyHostToDevice, s) !=
        cudaSuccess) {
      g_cuda_err = "cudaMemcpyAsync band";
      return fail2(SPIKE_ECUDA);
    }
    dband = c->band64;
    band_in_b64 = true;
  } else if (!band_dev) {
    dband = (const double *)mapped_host_ptr(band);
  }
  if (!band_dev && !dband) {
    cudaError_t e = dev_alloc((void **)&bstage, sizeof(double) * (size_t)n * ldab, s);
    if (e != cudaSuccess) {
      g_cuda_err = std::string("cudaMallocAsync: ") + cudaGetErrorString(e);
      bstage = nullptr;
      return fail2(SPIKE_ENOMEM);
    }
    if (cudaMemcpyAsync(bstage, band, sizeof(double) * (size_t)n * ldab, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      g_cuda_err = "cudaMemcpyAsync band";
      return fail2(SPIKE_ECUDA);
    }
    dband = bstage;
  }
  char *zbuf = fscr + s_z;  // element size es
  int64_t *dzoff = (int64_t *)(fscr + s_zoff);
  LeafDev *dleaf = (LeafDev *)(fscr + s_leaf);
  char *tmp = fscr + s_tmp;

  // identity and status init
  {
    std::vector<double> id((size_t)kk, 0.0);
    for (int i = 0; i < k; ++i) id[(size_t)i * k + i] = 1.0;
    unsigned long long st[8] = {0, ULLONG_MAX, 0, 0, 0, 0, 0, 0};
    if (cudaMemcpyAsync(c->ident, id.data(), sizeof(double) * kk, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(c->status, st, sizeof(st), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dzoff, zoff.data(), sizeof(int64_t) * nlv, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dleaf, c->hl.data(), sizeof(LeafDev) * nlv, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(zbuf, 0, c->es * (size_t)zacc, s) != cudaSuccess ||
        cudaMemsetAsync(c->spk, 0, sizeof(double) * (size_t)nspk * 2 * nlv * 2 * kk, s) != cudaSuccess) {
      g_cuda_err = "initialisation copies";
      return fail2(SPIKE_ECUDA);
    }
  }
  if (c->timing) cudaEventRecord(c->fev[0], s);
  // 1. repack the band into per-leaf LU storage; couplings; Z right-hand sides
  if (c->f32 && !borrow && !band_in_b64 &&
      cudaMemcpyAsync(c->band64, dband, sizeof(double) * (size_t)n * ldab, cudaMemcpyDeviceToDevice, s) !=
                    cudaSuccess) {
    g_cuda_err = "band copy";
    return fail2(SPIKE_ECUDA);
  }
  // mixed: the digit fragments of A and A^T for the tensor-core refinement residual
  for (int t = 0; t < 2 && c->sfrag[0]; ++t) {
    if ((rc = launch_split_band(c->band64, ldab, n, kl, ku, t, c->srexp[t], c->snorm + t, c->sfrag[t], s)) != 0) {
      g_cuda_err = std::string("split kernels: ") + cudaGetErrorString((cudaError_t)rc);
      return fail2(SPIKE_ECUDA);
    }
  }
  if ((rc = launch_repack(dband, ldab, kl, ku, n, k, c->ldf, c->dofs, dleaf, nlv, c->fbc, &c->status[3], s, maxlen,
                          c->f32)) != 0 ||
      (rc = launch_couplings(dband, ldab, kl, ku, n, k, dleaf, nlv, c->couple, s)) != 0 ||
      (rc = launch_zinit(dleaf, nlv, k, c->couple, zbuf, dzoff, c->f32, s)) != 0) {
    g_cuda_err = std::string("setup kernels: ") + cudaGetErrorString((cudaError_t)rc);
    return fail2(SPIKE_ECUDA);
  }
  if (bstage) {  // the setup kernels were the band's last readers (stream order frees it after them)
    cudaFreeAsync(bstage, s);
    bstage = nullptr;
  }
  if (c->timing) cudaEventRecord(c->fev[1], s);
  // 2. block factorizations and spike sweeps (Sec. 2.3): truncated sweeps for the
  // first/last blocks, three full sweeps for middle ones (the L-sweep of the top spike
  // is fused into the non-pivoting LU; the others run in the same CTA after it).
  {
    std::vector<SweepDesc> ltop(nlv, empty_sweep()), lbot(nlv, empty_sweep()), ub(nlv, empty_sweep());
    View none{nullptr, 0, 0};
    for (int i = 0; i < nlv; ++i) {
      const LeafDev &L = c->hl[i];
      const int nl = (int)L.len;
      const bool mid = L.top_nbr && L.bot_nbr;
      View zt{(double *)(zbuf + zoff[i] * (int64_t)c->es), 1, L.len},
          zb{(double *)(zbuf + (zoff[i] + (int64_t)k * L.len) * (int64_t)c->es), 1, L.len};
      if (pivot && mid) ltop[i] = sdesc(c, i, LN, 0, nl, k, zt, nullptr, none, 0.0, zt);
      if (L.bot_nbr) lbot[i] = sdesc(c, i, LN, pivot ? nl - 2 * k : nl - k, nl, k, zb, nullptr, none, 0.0, zb);
      if (mid) ub[i] = sdesc(c, i, UN, 0, nl, 2 * k, zt, nullptr, none, 0.0, zt);
      else if (L.bot_nbr) ub[i] = sdesc(c, i, UN, nl - k, nl, k, zb, nullptr, none, 0.0, zb);
    }
    if (tasks) {
      // several systems: this one's blocks join the shared launch (spike_factor_batch)
      for (int i = 0; i < nlv; ++i) {
        FactorTask t;
        memset(&t, 0, sizeof(t));
        t.leaf = c->hl[i];
        t.k = k;
        t.ldf = c->ldf;
        t.fb_all = c->fbc;
        t.dinv_all = c->dinvc;
        t.Z = zbuf + zoff[i] * (int64_t)c->es;
        t.amax_bits = &c->status[3];
        t.status = c->status;
        t.sw[0] = lbot[i];
        t.sw[1] = ub[i];
        tasks->push_back(t);
      }
      cont->fscr = fscr;
      cont->dleaf = dleaf;
      cont->zbuf = zbuf;
      cont->dzoff = dzoff;
      cont->tmp = tmp;
      cont->tmp_bytes = tmp_bytes;
      *out = c;
      return 0;
    }
    std::vector<SweepDesc> pairs;
    for (int i = 0; i < nlv; ++i) {
      if (pivot) pairs.push_back(ltop[i]);
      pairs.push_back(lbot[i]);
      pairs.push_back(ub[i]);
    }
    if (!pivot) {
      Arena ar;
      const size_t off = ar.put(pairs);
      if ((rc = ensure(&c->dargs, &c->dargs_bytes, ar.h.size(), s)) != 0) return fail2(rc);
      if (cudaMemcpyAsync(c->dargs, ar.h.data(), ar.h.size(), cudaMemcpyHostToDevice, s) != cudaSuccess) {
        g_cuda_err = "sweep descriptors";
        return fail2(SPIKE_ECUDA);
      }
      rc = launch_factor_nopiv(dleaf, nlv, k, c->ldf, c->fbc, c->dinvc, zbuf, dzoff, &c->status[3], kBoostEps,
                               c->status, (const SweepDesc *)(c->dargs + off), s, c->f32);
      if (rc != 0) {
        g_cuda_err = std::string("factor kernel: ") + cudaGetErrorString((cudaError_t)rc);
        return fail2(SPIKE_ECUDA);
      }
      if (c->timing) cudaEventRecord(c->fev[2], s);
    } else {
      // block GEPP, then the block's pivoted L sweeps and U sweep, in one launch
      Arena ar;
      const size_t off = ar.put(pairs);
      if ((rc = ensure(&c->dargs, &c->dargs_bytes, ar.h.size(), s)) != 0) return fail2(rc);
      if (cudaMemcpyAsync(c->dargs, ar.h.data(), ar.h.size(), cudaMemcpyHostToDevice, s) != cudaSuccess) {
        g_cuda_err = "sweep descriptors";
        return fail2(SPIKE_ECUDA);
      }
      rc = launch_factor_piv(dleaf, nlv, k, c->ldf, (double *)c->fbc, (double *)c->dinvc, c->ipiv, c->status,
                             (const SweepDesc *)(c->dargs + off), s);
      if (rc != 0) {
        g_cuda_err = std::string("factor kernel: ") + cudaGetErrorString((cudaError_t)rc);
        return fail2(SPIKE_ECUDA);
      }
      if (c->timing) cudaEventRecord(c->fev[2], s);
    }
  }
  if ((rc = launch_tips0(dleaf, nlv, k, zbuf, dzoff, c->spk, s, c->f32)) != 0) {
    g_cuda_err = std::string("tips kernel: ") + cudaGetErrorString((cudaError_t)rc);
    return fail2(SPIKE_ECUDA);
  }
  if (c->timing) cudaEventRecord(c->fev[3], s);
  // 4. recursive reduced system factorization (sharded: the levels inside the rank; the others
  // follow the exchanges of spike_shard_import)
  for (int lv = 0; lv < (c->shard ? c->lvl : c->NL); ++lv) {
    if ((rc = factor_reduced_level(c, lv, tmp, tmp_bytes)) != 0) return fail2(rc);
  }
  if (c->timing) {
    cudaEventRecord(c->fev[4], s);
    c->fdone = true;
  }
  // 5. status
  unsigned long long st[8];
  if (cudaMemcpyAsync(st, c->status, sizeof(st), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    g_cuda_err = std::string("factor: ") + cudaGetErrorString(cudaGetLastError());
    return fail2(SPIKE_ECUDA);
  }
  if (c->shard && c->lvl < c->NL) {
    c->sh_fscr = fscr;  // the per-merge temporaries of the coarse levels
    c->sh_tmp_off = s_tmp;
    c->sh_tmp_bytes = tmp_bytes;
    c->sh_op = 1;
    c->sh_level = c->lvl;
  } else {
    cudaFreeAsync(fscr, s);
  }
  c->boosts = (int64_t)st[0];
  c->zero_col = (st[1] == ULLONG_MAX) ? 0 : (int64_t)st[1];
  c->nan_flag = (int)st[2];
  *out = c;
  if (pivot && c->zero_col) return (int)std::min<int64_t>(c->zero_col, INT_MAX);
  return 0;
}

extern "C" int spike_factor(const double *band, int64_t n, int kl, int ku, int p, int pivot, spike_handle *out) {
  return spike_factor_ex(band, (int64_t)kl + ku + 1, n, kl, ku, p, pivot, nullptr, out);
}

static int factor_reduced_level(spike_ctx *c, int lv, char *tmp, size_t tmp_bytes);
static void reduced_level_build(spike_ctx *c, int lv, char *tmp, LevelBatch &LB);
static void reduced_level_emit(LevelBatch &LB, Pipeline &pp);
static int reduced_level_flags(const std::vector<spike_ctx *> &cs, int lv, cudaStream_t s, spike_ctx *args);

extern "C" int spike_factor_batch(const double *const *bands, const int64_t *ldab, const int64_t *n, const int *kl,
                                  const int *ku, const int *p, int count, const spike_options *opt,
                                  spike_handle *out) {
  if (!bands) return -1;
  if (!ldab) return -2;
  if (!n) return -3;
  if (!kl) return -4;
  if (!ku) return -5;
  if (!p) return -6;
  if (count < 0) return -7;
  if (!out) return -9;
  for (int i = 0; i < count; ++i) out[i] = nullptr;
  if (count == 0) return 0;
  if (opt && (opt->flags & (SPIKE_FLAG_MIXED | SPIKE_FLAG_TIMING))) return SPIKE_ENOTSUP;
  for (int i = 0; i < count; ++i)
    if (!bands[i] || !is_device_ptr(bands[i])) return SPIKE_ENOTSUP;
  std::vector<spike_ctx *> cs;
  std::vector<FactorCont> conts((size_t)count);
  std::vector<FactorTask> tasks;
  int maxk = 1;
  auto fail = [&](int code) {
    for (size_t i = 0; i < cs.size(); ++i) {
      if (conts[i].fscr) cudaFreeAsync(conts[i].fscr, cs[i]->stream);
      spike_free(cs[i]);
    }
    for (int i = 0; i < count; ++i) out[i] = nullptr;
    return code;
  };
  // 1. every system's plan, memory and setup kernels, up to its block LU
  for (int i = 0; i < count; ++i) {
    spike_handle h = nullptr;
    const int rc = factor_impl(bands[i], ldab[i], n[i], kl[i], ku[i], p[i], 0, opt, &h, nullptr, &tasks, &conts[i]);
    if (rc != 0 || !h) return fail(rc != 0 ? rc : SPIKE_ECUDA);
    cs.push_back(h);
    maxk = std::max(maxk, h->k);
  }
  spike_ctx *c0 = cs[0];
  cudaStream_t s = c0->stream;
  // 2. all blocks of all systems in one launch, largest first, from a work queue
  std::stable_sort(tasks.begin(), tasks.end(), [](const FactorTask &a, const FactorTask &b) {
    return (double)a.leaf.len * a.k * a.k > (double)b.leaf.len * b.k * b.k;
  });
  {
    Arena ar;
    const size_t ot = ar.put(tasks);
    const size_t oq = ar.put(std::vector<unsigned>(1, 0u));
    int rc = ensure(&c0->dargs, &c0->dargs_bytes, ar.h.size(), s);
    if (rc != 0) return fail(rc);
    if (cudaMemcpyAsync(c0->dargs, ar.h.data(), ar.h.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
      return fail(SPIKE_ECUDA);
    rc = launch_factor_tasks((const FactorTask *)(c0->dargs + ot), (int)tasks.size(), maxk,
                             (unsigned *)(c0->dargs + oq), s);
    if (rc != 0) {
      g_cuda_err = std::string("factor tasks: ") + cudaGetErrorString((cudaError_t)rc);
      return fail(SPIKE_ECUDA);
    }
  }
  // 3. tips of every system
  for (size_t i = 0; i < cs.size(); ++i) {
    spike_ctx *c = cs[i];
    const int rc = launch_tips0(conts[i].dleaf, c->nleaves, c->k, conts[i].zbuf, conts[i].dzoff, c->spk, s, 0);
    if (rc != 0) return fail(SPIKE_ECUDA);
  }
  // 4. the reduced systems, one merge level of every system per round (levels aligned from the
  // bottom), one flag round trip and one set of batched launches per level
  int maxnl = 0;
  for (auto *c : cs) maxnl = std::max(maxnl, c->NL);
  for (int lv = 0; lv < maxnl; ++lv) {
    std::vector<spike_ctx *> at;
    std::vector<size_t> idx;
    for (size_t i = 0; i < cs.size(); ++i)
      if (lv < cs[i]->NL) {
        at.push_back(cs[i]);
        idx.push_back(i);
      }
    int rc = reduced_level_flags(at, lv, s, c0);
    if (rc != 0) return fail(rc);
    LevelBatch LB;
    for (size_t j = 0; j < at.size(); ++j) reduced_level_build(at[j], lv, conts[idx[j]].tmp, LB);
    Pipeline pp;
    pp.st = s;
    reduced_level_emit(LB, pp);
    if ((rc = pp.run(c0)) != 0) return fail(rc);
  }
  // 5. status of every system
  std::vector<unsigned long long> st((size_t)8 * cs.size());
  for (size_t i = 0; i < cs.size(); ++i)
    if (cudaMemcpyAsync(&st[8 * i], cs[i]->status, sizeof(unsigned long long) * 8, cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
      return fail(SPIKE_ECUDA);
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(SPIKE_ECUDA);
  for (size_t i = 0; i < cs.size(); ++i) {
    spike_ctx *c = cs[i];
    cudaFreeAsync(conts[i].fscr, s);
    c->boosts = (int64_t)st[8 * i];
    c->zero_col = (st[8 * i + 1] == ULLONG_MAX) ? 0 : (int64_t)st[8 * i + 1];
    c->nan_flag = (int)st[8 * i + 2];
    out[i] = c;
  }
  return 0;
}

// One merge level of the reduced system (Sec. 2.2): for each pair of adjacent
// groups L = [a,b), R = [b,c) factor the 2k x 2k interface
//   M = [ I  V_{b-1,bot} ; W_{b,top}  I ]
// and form the merged group's spikes (Eqs. RED_SYS_RECB / RED_SYS_W):
//   [alpha; beta] = M^{-1} [0; V_{b,top}],  [gamma; delta] = M^{-1} [W_{b-1,bot}; 0]
//   V'_L = -V_L beta,   V'_R = V_R - W_R alpha,   W'_L = W_L - V_L delta,   W'_R = -W_R gamma
// (interface tips V'_{b,top} = beta, W'_{b,top} = delta come from the 2k solve).
// When |W_{b,top}| <= 1 the pivoted LU of M keeps the identity rows for the first k
// columns, so M = [I 0; W I][I V; 0 S] with S = I - W V: only S is LU-factored
// (same pivot decisions as partial pivoting on M), otherwise M itself is.
static void reduced_level_build(spike_ctx *c, int lv, char *tmp, LevelBatch &LB) {
  const Plan &pl = c->pl;
  const auto &ms = pl.levels[lv];
  const int nm = (int)ms.size();
  const int k = c->k;
  const int64_t kk = (int64_t)k * k;
  const std::vector<int> &sc = c->schur[lv];
  const bool last = (lv + 1 >= c->NL);
  GemmBatch &gA = LB.gA, &gB = LB.gB, &gC = LB.gC;
  std::vector<LuDesc> &lus = LB.lus;
  TrsBatch &tr = LB.tr;
  int &maxn = LB.maxn;
  for (int m = 0; m < nm; ++m) {
    const Merge &mg = ms[m];
    // a rank forms the merges inside its leaves and, above them, the one merge containing them
    const bool inside = !c->shard || (mg.a >= c->l0 && mg.c <= c->l1);
    const bool mine = c->shard && mg.a <= c->l0 && c->l1 <= mg.c;
    if (!inside && !mine) continue;
    const int64_t gm = c->merge_off[lv] + m;
    double *lu = c->mlu + gm * 4 * kk;
    int *piv = c->mpiv + gm * 2 * k;
    double *slot = (double *)tmp + (int64_t)m * 5 * kk;  // [alpha; beta; gamma; delta; T]
    double *al = slot, *be = slot + kk, *ga = slot + 2 * kk, *de = slot + 3 * kk, *Tm = slot + 4 * kk;
    const double *Vlb = TIP(c, lv, 0, mg.b - 1, 1), *Wrt = TIP(c, lv, 1, mg.b, 0);
    const double *Vrt = TIP(c, lv, 0, mg.b, 0), *Wlb = TIP(c, lv, 1, mg.b - 1, 1);
    LuDesc L;
    memset(&L, 0, sizeof(L));
    L.a = lu;
    L.ipiv = piv;
    L.active = 1;
    L.status = c->status;
    if (sc[m]) {
      gA.add(gd(Wrt, k, 1, Vlb, k, 1, c->ident, k, 1, lu, k, 1, k, k, k, -1.0, 1.0));  // S = I - W V
      if (mg.hasW) gA.add(gd(Wrt, k, 1, Wlb, k, 1, nullptr, 0, 0, Tm, k, 1, k, k, k, 1.0, 0.0));
      if (mg.hasV) gA.add(gd(nullptr, 0, 0, nullptr, 0, 0, Vrt, k, 1, be, k, 1, k, k, 0, 0.0, 1.0));
      L.n = k;
      L.lda = k;
      if (mg.hasV) tr.add(lu, piv, k, k, be, k, k, 0, 1.0);
      if (mg.hasW) tr.add(lu, piv, k, k, Tm, k, k, 0, -1.0);  // delta = -S^{-1} W_rt W_lb
      if (mg.hasV) gB.add(gd(Vlb, k, 1, be, k, 1, nullptr, 0, 0, al, k, 1, k, k, k, -1.0, 0.0));
      if (mg.hasW) {
        gB.add(gd(Vlb, k, 1, Tm, k, 1, Wlb, k, 1, ga, k, 1, k, k, k, -1.0, 1.0));
        gB.add(gd(nullptr, 0, 0, nullptr, 0, 0, Tm, k, 1, de, k, 1, k, k, 0, 0.0, 1.0));
      }
    } else {
      const int n2 = 2 * k;
      gA.add(gd(nullptr, 0, 0, nullptr, 0, 0, c->ident, k, 1, lu, n2, 1, k, k, 0, 0.0, 1.0));
      gA.add(gd(nullptr, 0, 0, nullptr, 0, 0, Vlb, k, 1, lu + k, n2, 1, k, k, 0, 0.0, 1.0));
      gA.add(gd(nullptr, 0, 0, nullptr, 0, 0, Wrt, k, 1, lu + (int64_t)k * n2, n2, 1, k, k, 0, 0.0, 1.0));
      gA.add(gd(nullptr, 0, 0, nullptr, 0, 0, c->ident, k, 1, lu + (int64_t)k * n2 + k, n2, 1, k, k, 0, 0.0, 1.0));
      if (mg.hasV) {
        gA.add(gd(nullptr, 0, 0, nullptr, 0, 0, nullptr, 0, 0, al, k, 1, k, k, 0, 0.0, 0.0));
        gA.add(gd(nullptr, 0, 0, nullptr, 0, 0, Vrt, k, 1, be, k, 1, k, k, 0, 0.0, 1.0));
        tr.add(lu, piv, n2, n2, al, k, k, 0, 1.0);
      }
      if (mg.hasW) {
        gA.add(gd(nullptr, 0, 0, nullptr, 0, 0, Wlb, k, 1, ga, k, 1, k, k, 0, 0.0, 1.0));
        gA.add(gd(nullptr, 0, 0, nullptr, 0, 0, nullptr, 0, 0, de, k, 1, k, k, 0, 0.0, 0.0));
        tr.add(lu, piv, n2, n2, ga, k, k, 0, 1.0);
      }
      L.n = n2;
      L.lda = n2;
    }
    maxn = std::max(maxn, L.n);
    lus.push_back(L);
    if (!last && !inside) {
      // merge over several ranks: update this rank's leaves only.  L-side leaves [la, lb),
      // R-side leaves [ra, rb); the interface tips (b-1, bottom) and (b, top) come from the
      // 2k solve when the rank holds them (the formulas below give the same values).
      const int b = mg.b;
      const int la = std::max(mg.a, c->l0), lb = std::min(b, c->l1);
      const int ra = std::max(b, c->l0), rb = std::min(mg.c, c->l1);
      auto zero = [&](int sp, int i0, int rows) {
        gC.add(gd(nullptr, 0, 0, nullptr, 0, 0, nullptr, 0, 0, TIP(c, lv + 1, sp, i0, 0), k, 1, rows, k, 0, 0.0, 0.0));
      };
      if (lb > la) {
        const int ML = 2 * (lb - la) * k;
        if (mg.hasV)
          gC.add(gd(TIP(c, lv, 0, la, 0), k, 1, be, k, 1, nullptr, 0, 0, TIP(c, lv + 1, 0, la, 0), k, 1, ML, k, k, -1.0,
                    0.0));
        else
          zero(0, la, ML);
        if (mg.hasW)
          gC.add(gd(TIP(c, lv, 0, la, 0), k, 1, de, k, 1, TIP(c, lv, 1, la, 0), k, 1, TIP(c, lv + 1, 1, la, 0), k, 1, ML,
                    k, k, -1.0, 1.0));
        else
          zero(1, la, ML);
      }
      if (rb > ra) {
        const int t0 = (ra == b) ? 1 : 0;  // holding b: its top tip comes from the solve
        const int MR = (2 * (rb - ra) - t0) * k;
        if (mg.hasV) {
          gC.add(gd(TIP(c, lv, 1, ra, t0), k, 1, al, k, 1, TIP(c, lv, 0, ra, t0), k, 1, TIP(c, lv + 1, 0, ra, t0), k, 1,
                    MR, k, k, -1.0, 1.0));
          if (t0) gC.add(gd(nullptr, 0, 0, nullptr, 0, 0, be, k, 1, TIP(c, lv + 1, 0, b, 0), k, 1, k, k, 0, 0.0, 1.0));
        } else {
          zero(0, ra, 2 * (rb - ra) * k);
        }
        if (mg.hasW) {
          gC.add(gd(TIP(c, lv, 1, ra, t0), k, 1, ga, k, 1, nullptr, 0, 0, TIP(c, lv + 1, 1, ra, t0), k, 1, MR, k, k,
                    -1.0, 0.0));
          if (t0) gC.add(gd(nullptr, 0, 0, nullptr, 0, 0, de, k, 1, TIP(c, lv + 1, 1, b, 0), k, 1, k, k, 0, 0.0, 1.0));
        } else {
          zero(1, ra, 2 * (rb - ra) * k);
        }
      }
    } else if (!last) {
      const int a = mg.a, b = mg.b, cc = mg.c;
      const int ML = 2 * (b - a) * k, MR = (2 * (cc - b) - 1) * k, MA = 2 * (cc - a) * k;
      if (mg.hasV) {
        gC.add(gd(TIP(c, lv, 0, a, 0), k, 1, be, k, 1, nullptr, 0, 0, TIP(c, lv + 1, 0, a, 0), k, 1, ML, k, k, -1.0,
                  0.0));
        gC.add(gd(TIP(c, lv, 1, b, 1), k, 1, al, k, 1, TIP(c, lv, 0, b, 1), k, 1, TIP(c, lv + 1, 0, b, 1), k, 1, MR,
                  k, k, -1.0, 1.0));
        gC.add(gd(nullptr, 0, 0, nullptr, 0, 0, be, k, 1, TIP(c, lv + 1, 0, b, 0), k, 1, k, k, 0, 0.0, 1.0));
      } else {
        gC.add(gd(nullptr, 0, 0, nullptr, 0, 0, nullptr, 0, 0, TIP(c, lv + 1, 0, a, 0), k, 1, MA, k, 0, 0.0, 0.0));
      }
      if (mg.hasW) {
        gC.add(gd(TIP(c, lv, 0, a, 0), k, 1, de, k, 1, TIP(c, lv, 1, a, 0), k, 1, TIP(c, lv + 1, 1, a, 0), k, 1, ML,
                  k, k, -1.0, 1.0));
        gC.add(gd(TIP(c, lv, 1, b, 1), k, 1, ga, k, 1, nullptr, 0, 0, TIP(c, lv + 1, 1, b, 1), k, 1, MR, k, k, -1.0,
                  0.0));
        gC.add(gd(nullptr, 0, 0, nullptr, 0, 0, de, k, 1, TIP(c, lv + 1, 1, b, 0), k, 1, k, k, 0, 0.0, 1.0));
      } else {
        gC.add(gd(nullptr, 0, 0, nullptr, 0, 0, nullptr, 0, 0, TIP(c, lv + 1, 1, a, 0), k, 1, MA, k, 0, 0.0, 0.0));
      }
    }
  }
  if (!last) {
    // untouched groups of this level keep their spikes: copy the whole level first
    double *src = TIP(c, lv, 0, 0, 0), *dst = TIP(c, lv + 1, 0, 0, 0);
    const size_t bytes = sizeof(double) * (size_t)2 * c->nleaves * 2 * kk;
    cudaStream_t s = c->stream;
    LB.copies.push_back([=](char *) { return (int)cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s); });
  }
}

// Launch a level's batches (one system's or several systems'): interface LUs, the 2k solves,
// then the level's spike copy and the merged-spike products.
static void reduced_level_emit(LevelBatch &LB, Pipeline &pp) {
  cudaStream_t s = pp.st;
  pp.gemm(LB.gA);
  if (!LB.lus.empty()) {
    const size_t off = pp.ar.put(LB.lus);
    const int nd = (int)LB.lus.size(), maxn = LB.maxn;
    pp.ops.push_back([=](char *base) { return launch_getrf((LuDesc *)(base + off), nd, maxn, nullptr, s); });
  }
  pp.trs(LB.tr);
  pp.gemm(LB.gB);
  for (auto &o : LB.copies) pp.ops.push_back(o);
  pp.gemm(LB.gC);
}

// The Schur-path flags of level lv of several systems (one flag per merge, Sec. 2.2 reading 12)
// with one device round trip, into each system's schur[lv].
static int reduced_level_flags(const std::vector<spike_ctx *> &cs, int lv, cudaStream_t s, spike_ctx *args) {
  std::vector<const double *> w;
  std::vector<int> cnt;
  for (spike_ctx *c : cs) {
    const auto &ms = c->pl.levels[lv];
    for (auto &mg : ms) w.push_back(TIP(c, lv, 1, mg.b, 0));
    cnt.push_back((int)ms.size());
  }
  const int nm = (int)w.size();
  std::vector<int> f(nm, 0);
  if (nm > 0) {
    Arena ar;
    const size_t ow = ar.put(w);
    const size_t of = ar.put(f);
    SP_TRY(ensure(&args->dargs, &args->dargs_bytes, ar.h.size(), s));
    SP_CUDA(cudaMemcpyAsync(args->dargs, ar.h.data(), ar.h.size(), cudaMemcpyHostToDevice, s));
    // one launch per system (each with its own k x k tips), one read-back for all of them
    int pos = 0;
    for (size_t i = 0; i < cs.size(); ++i) {
      if (cnt[i] > 0) {
        const int rc = launch_noswap_flags((const double *const *)(args->dargs + ow) + pos, cs[i]->k, cnt[i],
                                           (int *)(args->dargs + of) + pos, s);
        if (rc != 0) {
          g_cuda_err = std::string("noswap: ") + cudaGetErrorString((cudaError_t)rc);
          return SPIKE_ECUDA;
        }
      }
      pos += cnt[i];
    }
    SP_CUDA(cudaMemcpyAsync(f.data(), args->dargs + of, sizeof(int) * nm, cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaStreamSynchronize(s));
  }
  int pos = 0;
  for (size_t i = 0; i < cs.size(); ++i) {
    cs[i]->schur[lv].assign(f.begin() + pos, f.begin() + pos + cnt[i]);
    pos += cnt[i];
  }
  return 0;
}

static int factor_reduced_level(spike_ctx *c, int lv, char *tmp, size_t tmp_bytes) {
  (void)tmp_bytes;
  SP_TRY(reduced_level_flags({c}, lv, c->stream, c));
  LevelBatch LB;
  reduced_level_build(c, lv, tmp, LB);
  Pipeline pp;
  pp.st = c->stream;
  reduced_level_emit(LB, pp);
  return pp.run(c);
}

// ================================================================ solve
// Scratch of one solve pipeline (element size es for the work arrays W and H).
struct SolveBufs {
  void *W;     // row-major n x m work array (RHS in, solution out), element size es
  void *H;     // row-major n x m scratch, element size es
  double *Y;   // reduced unknowns: leaves x {top, bottom} x k x m, row-major blocks
  double *TM;  // per-merge temporaries, 2 k x m each
  double *PP;  // per-leaf partial products (transposed reduced system), k x m each
};

// Record the SPIKE solve of op(A) X = W (Sec. 2.1-2.3 for N, Sec. 4 for T) on the
// row-major work array W, in place.  f32: W and H are FP32 and the leaf sweeps run
// in FP32 (mixed-precision handles); the reduced system is always FP64.
// Which parts of a solve to record: the first stage (head: D stage for N, S^T stage for T),
// the merge levels [lv_lo, lv_hi) of the reduced system, the last stage (tail: retrieval for
// N, D^T stage for T).  A sharded handle records only its own blocks and the merges inside
// them; the merges over several ranks are run by the exchange steps.
struct SolveRange {
  bool head = true, tail = true;
  int lv_lo = 0, lv_hi = INT_MAX;
};

static void build_solve_body(spike_ctx *c, Pipeline &pp, const SolveBufs &B, int m, int tr, bool marks,
                             const SolveRange &rg);
static void build_solve(spike_ctx *c, Pipeline &pp, const SolveBufs &B, int m, int tr, bool marks,
                        const SolveRange &rg = SolveRange()) {
  c->in_solve = 1;
  build_solve_body(c, pp, B, m, tr, marks, rg);
  c->in_solve = 0;
}

static void build_solve_body(spike_ctx *c, Pipeline &pp, const SolveBufs &B, int m, int tr, bool marks,
                             const SolveRange &rg) {
  const int64_t n = c->pl.n;
  const int k = c->k, nlv = c->nleaves;
  const int64_t kk = (int64_t)k * k, km = (int64_t)k * m;
  const size_t es = c->es;
  const int f32 = c->f32;
  cudaStream_t s = pp.st;
  double *Y = B.Y, *TM = B.TM, *PP = B.PP;
  auto eptr = [es](void *base, int64_t idx) { return (double *)((char *)base + idx * (int64_t)es); };
  auto YB = [&](int i, int t) { return Y + ((int64_t)i * 2 + t) * km; };
  auto rview = [&](const LeafDev &L, void *base) {
    if (L.rev) return View{eptr(base, (L.start + L.len - 1) * (int64_t)m), -(int64_t)m, 1};
    return View{eptr(base, L.start * (int64_t)m), (int64_t)m, 1};
  };
  auto rows = [&](void *base, int64_t row0) { return eptr(base, row0 * (int64_t)m); };
  // GEMM operand type flags for the work arrays
  const int tA = f32 ? G_A32 : 0, tB = f32 ? G_B32 : 0, tC0 = f32 ? G_C032 : 0, tC = f32 ? G_C32 : 0;
  auto typed = [](GemmDesc g, int t) {
    g.types = t;
    return g;
  };
  (void)tA;
  void *W = B.W, *H = B.H;
  View none{nullptr, 0, 0};
  const bool piv = c->pivot != 0;
  auto memset_op = [&](void *p, size_t bytes) {
    pp.op([=](char *) { return (int)cudaMemsetAsync(p, 0, bytes, s); });
  };
  cudaEvent_t *evs = tr ? c->tev : c->nev;
  auto mark = [&](int i) {
    if (!marks || !c->timing) return;
    cudaEvent_t e = evs[i];
    pp.op([=](char *) { return (int)cudaEventRecord(e, s); });
  };
  auto own = [&](int i) { return !c->shard || (i >= c->l0 && i < c->l1); };
  auto inside = [&](const Merge &mg) { return !c->shard || (mg.a >= c->l0 && mg.c <= c->l1); };
  // the H rows this handle holds (all rows, or a rank's own rows)
  void *Hmem = c->shard ? (void *)eptr(H, c->row0 * (int64_t)m) : H;
  const size_t Hbytes = es * (size_t)(c->shard ? c->nrow : n) * m;
  const int lv_lo = std::max(0, rg.lv_lo), lv_hi = std::min(c->NL, rg.lv_hi);
  pp.key(0, 0);
  if (rg.head) {
    memset_op(Hmem, Hbytes);
    memset_op(Y, sizeof(double) * (size_t)nlv * 2 * km);
  }

  if (tr == 0) {
    pp.key(1, 0);
    if (rg.head) {
    // ---------------- D stage (Eq. Dstage) with the sweep savings of Sec. 2.3
    std::vector<SweepDesc> sa(nlv, empty_sweep()), sb(nlv, empty_sweep());
    for (int i = 0; i < nlv; ++i) {
      if (!own(i)) continue;
      const LeafDev &L = c->hl[i];
      const int nl = (int)L.len;
      const View fv = rview(L, W), hv = rview(L, H);
      sa[i] = sdesc(c, i, LN, 0, nl, m, fv, nullptr, none, 0, fv);  // W <- L^{-1} W
      if (L.top_nbr && L.bot_nbr) sb[i] = sdesc(c, i, UN, 0, nl, m, fv, nullptr, none, 0, hv);
      else if (L.bot_nbr) sb[i] = sdesc(c, i, UN, nl - k, nl, m, fv, nullptr, none, 0, hv);
    }
    pp.stage(sa, sb, piv ? LN : -1, -1, c->ldf, c->dofs, k);
    // gather Y tips (global rows) from H
    GemmBatch g0;
    for (int i = 0; i < nlv; ++i) {
      if (!own(i)) continue;
      const LeafDev &L = c->hl[i];
      if (i > 0)
        g0.add(typed(gd(nullptr, 0, 0, nullptr, 0, 0, rows(H, L.start), m, 1, YB(i, 0), m, 1, k, m, 0, 0.0, 1.0), tC0));
      if (i + 1 < nlv)
        g0.add(typed(gd(nullptr, 0, 0, nullptr, 0, 0, rows(H, L.start + L.len - k), m, 1, YB(i, 1), m, 1, k, m, 0,
                        0.0, 1.0),
                     tC0));
    }
    pp.gemm(g0);
    mark(1);
    }
    // ---------------- reduced system, levels ascending: D^[1]^-1 ... (Eqs. D1Inverse, S2Inverse)
    for (int lv = lv_lo; lv < lv_hi; ++lv) {
      pp.key(2, lv);
      const auto &ms = c->pl.levels[lv];
      GemmBatch g1, g2, g3;
      TrsBatch ts;
      for (int mi = 0; mi < (int)ms.size(); ++mi) {
        const Merge &mg = ms[mi];
        if (!inside(mg)) continue;
        const int64_t gm = c->merge_off[lv] + mi;
        const double *lu = c->mlu + gm * 4 * kk;
        const int *pv = c->mpiv + gm * 2 * k;
        double *ta = TM + (int64_t)mi * 2 * km, *tb = ta + km;  // [a; b]
        const double *Vlb = TIP(c, lv, 0, mg.b - 1, 1), *Wrt = TIP(c, lv, 1, mg.b, 0);
        if (c->schur[lv][mi]) {
          // b = S^{-1} (y_{b,top} - W y_{b-1,bot});  a = y_{b-1,bot} - V b
          g1.add(gd(Wrt, k, 1, YB(mg.b - 1, 1), m, 1, YB(mg.b, 0), m, 1, tb, m, 1, k, m, k, -1.0, 1.0));
          ts.add(lu, pv, k, k, tb, m, m, 0, 1.0);
          g2.add(gd(Vlb, k, 1, tb, m, 1, YB(mg.b - 1, 1), m, 1, ta, m, 1, k, m, k, -1.0, 1.0));
        } else {
          g1.add(gd(nullptr, 0, 0, nullptr, 0, 0, YB(mg.b - 1, 1), m, 1, ta, m, 1, k, m, 0, 0.0, 1.0));
          g1.add(gd(nullptr, 0, 0, nullptr, 0, 0, YB(mg.b, 0), m, 1, tb, m, 1, k, m, 0, 0.0, 1.0));
          ts.add(lu, pv, 2 * k, 2 * k, ta, m, m, 0, 1.0);
        }
        // updates: y_L -= V_L b (all L tips but (b-1,bot)), y_R -= W_R a (all R tips but (b,top))
        const int ML = (2 * (mg.b - mg.a) - 1) * k, MR = (2 * (mg.c - mg.b) - 1) * k;
        g3.add(gd(TIP(c, lv, 0, mg.a, 0), k, 1, tb, m, 1, YB(mg.a, 0), m, 1, YB(mg.a, 0), m, 1, ML, m, k, -1.0, 1.0));
        g3.add(gd(TIP(c, lv, 1, mg.b, 1), k, 1, ta, m, 1, YB(mg.b, 1), m, 1, YB(mg.b, 1), m, 1, MR, m, k, -1.0, 1.0));
        g3.add(gd(nullptr, 0, 0, nullptr, 0, 0, ta, m, 1, YB(mg.b - 1, 1), m, 1, k, m, 0, 0.0, 1.0));
        g3.add(gd(nullptr, 0, 0, nullptr, 0, 0, tb, m, 1, YB(mg.b, 0), m, 1, k, m, 0, 0.0, 1.0));
      }
      pp.gemm(g1);
      pp.trs(ts);
      pp.gemm(g2);
      pp.gemm(g3);
    }
    mark(2);
    if (!rg.tail) return;
    // ---------------- retrieval (Eqs. one/two/three): X_i = U^{-1}(L^{-1}F - L^{-1}[R_top x_top; 0; R_bot x_bot])
    pp.key(3, 0);
    memset_op(Hmem, Hbytes);
    GemmBatch gc;
    std::vector<SweepDesc> sc(nlv, empty_sweep()), sd(nlv, empty_sweep());
    for (int i = 0; i < nlv; ++i) {
      if (!own(i)) continue;
      const LeafDev &L = c->hl[i];
      const int nl = (int)L.len;
      const View fv = rview(L, W), hv = rview(L, H);
      const double *Rt = c->couple + (int64_t)i * 2 * kk, *Rb = Rt + kk;
      if (L.top_nbr) {
        const double *xn = L.rev ? YB(i + 1, 0) : YB(i - 1, 1);
        gc.add(typed(gd(Rt, k, 1, xn, m, 1, nullptr, 0, 0, hv.p, hv.rs, hv.cs, k, m, k, 1.0, 0.0), tC));
      }
      if (L.bot_nbr) {
        const double *xn = L.rev ? YB(i - 1, 1) : YB(i + 1, 0);
        gc.add(typed(gd(Rb, k, 1, xn, m, 1, nullptr, 0, 0, (double *)((char *)hv.p + (int64_t)(nl - k) * hv.rs * (int64_t)es),
                        hv.rs, hv.cs, k, m, k, 1.0, 0.0),
                     tC));
      }
      if (L.top_nbr && L.bot_nbr) sc[i] = sdesc(c, i, LN, 0, nl, m, hv, nullptr, none, 0, hv);
      else if (L.bot_nbr) sc[i] = sdesc(c, i, LN, piv ? nl - 2 * k : nl - k, nl, m, hv, nullptr, none, 0, hv);
      sd[i] = sdesc(c, i, UN, 0, nl, m, fv, hv.p, hv, -1.0, fv);
    }
    pp.gemm(gc);
    pp.stage(sc, sd, piv ? LN : -1, -1, c->ldf, c->dofs, k);
  } else {
    // ---------------- transpose: S^T Y = F then D^T X = Y (Sec. 4.1, 4.2)
    pp.key(1, 0);
    if (rg.head) {
    GemmBatch g0, gz;
    for (int i = 0; i < nlv; ++i) {
      if (!own(i)) continue;
      const LeafDev &L = c->hl[i];
      if (i > 0) {
        double *v = rows(W, L.start);
        g0.add(typed(gd(nullptr, 0, 0, nullptr, 0, 0, v, m, 1, YB(i, 0), m, 1, k, m, 0, 0.0, 1.0), tC0));
        gz.add(typed(gd(nullptr, 0, 0, nullptr, 0, 0, nullptr, 0, 0, v, m, 1, k, m, 0, 0.0, 0.0), tC));
      }
      if (i + 1 < nlv) {
        double *v = rows(W, L.start + L.len - k);
        g0.add(typed(gd(nullptr, 0, 0, nullptr, 0, 0, v, m, 1, YB(i, 1), m, 1, k, m, 0, 0.0, 1.0), tC0));
        gz.add(typed(gd(nullptr, 0, 0, nullptr, 0, 0, nullptr, 0, 0, v, m, 1, k, m, 0, 0.0, 0.0), tC));
      }
    }
    pp.gemm(g0);
    pp.gemm(gz);
    std::vector<SweepDesc> sa(nlv, empty_sweep()), sb(nlv, empty_sweep()), e0(nlv, empty_sweep());
    for (int i = 0; i < nlv; ++i) {
      if (!own(i)) continue;
      const LeafDev &L = c->hl[i];
      const int nl = (int)L.len;
      const View fv = rview(L, W), hv = rview(L, H);
      sa[i] = sdesc(c, i, UT, 0, nl, m, fv, nullptr, none, 0, fv);  // w = U^{-T} [0; F~; 0]
      const int r0 = (L.top_nbr && L.bot_nbr) ? 0 : (piv ? nl - 2 * k : nl - k);
      if (L.bot_nbr) sb[i] = sdesc(c, i, LT, r0, nl, m, piv ? hv : fv, nullptr, none, 0, hv);
    }
    if (piv) {
      // the pivoted L^T sweep runs in place: copy w into H first
      pp.stage(sa, e0, -1, -1, c->ldf, c->dofs, k);
      const size_t bytes = es * (size_t)n * m;
      pp.op([=](char *) { return (int)cudaMemcpyAsync(H, W, bytes, cudaMemcpyDeviceToDevice, s); });
      pp.stage(sb, e0, LT, -1, c->ldf, c->dofs, k);
    } else {
      pp.stage(sa, sb, -1, -1, c->ldf, c->dofs, k);
    }
    // G tips: y_{j+1,top} -= Bhat_j^T z_{j,bot}, y_{j-1,bot} -= Chat_j^T z_{j,top} (Eqs. G_in_transpose_1/2)
    GemmBatch gg;
    for (int j = 0; j < nlv; ++j) {
      if (!own(j)) continue;
      const LeafDev &L = c->hl[j];
      const int nl = (int)L.len;
      const View hv = rview(L, H);
      const double *Rt = c->couple + (int64_t)j * 2 * kk, *Rb = Rt + kk;
      if (L.top_nbr) {
        double *tgt = L.rev ? YB(j + 1, 0) : YB(j - 1, 1);
        gg.add(typed(gd(Rt, 1, k, hv.p, hv.rs, hv.cs, tgt, m, 1, tgt, m, 1, k, m, k, -1.0, 1.0), tB));
      }
      if (L.bot_nbr) {
        double *tgt = L.rev ? YB(j - 1, 1) : YB(j + 1, 0);
        gg.add(typed(gd(Rb, 1, k, (double *)((char *)hv.p + (int64_t)(nl - k) * hv.rs * (int64_t)es), hv.rs, hv.cs,
                        tgt, m, 1, tgt, m, 1, k, m, k, -1.0, 1.0),
                     tB));
      }
    }
    pp.gemm(gg);
    mark(1);
    }
    // ---------------- transposed reduced system, levels descending (Sec. 4.3)
    for (int lv = lv_hi - 1; lv >= lv_lo; --lv) {
      pp.key(2, -lv);  // levels descending: higher levels first in every system
      const auto &ms = c->pl.levels[lv];
      GemmBatch gpart, g2, g3, g4;
      std::vector<SumDesc> sums;
      TrsBatch ts;
      int64_t maxe = 0;
      for (int mi = 0; mi < (int)ms.size(); ++mi) {
        const Merge &mg = ms[mi];
        if (!inside(mg)) continue;
        const int64_t gm = c->merge_off[lv] + mi;
        const double *lu = c->mlu + gm * 4 * kk;
        const int *pv = c->mpiv + gm * 2 * k;
        double *s2 = TM + (int64_t)mi * 2 * km, *s1 = s2 + km;  // [g2; g1] -> [s2; s1]
        const double *Vlb = TIP(c, lv, 0, mg.b - 1, 1), *Wrt = TIP(c, lv, 1, mg.b, 0);
        // g1 = V_L^T y_L, g2 = W_R^T y_R: one partial product per leaf (both tips), then a
        // fixed-order sum over the group's leaves
        for (int i = mg.a; i < mg.c; ++i) {
          const int sp = (i < mg.b) ? 0 : 1;
          gpart.add(gd(TIP(c, lv, sp, i, 0), 1, k, YB(i, 0), m, 1, nullptr, 0, 0, PP + (int64_t)i * km, m, 1, k, m,
                       2 * k, 1.0, 0.0));
        }
        SumDesc d1{PP + (int64_t)mg.a * km, s1, km, km, mg.b - mg.a, 0};
        SumDesc d2{PP + (int64_t)mg.b * km, s2, km, km, mg.c - mg.b, 0};
        sums.push_back(d1);
        sums.push_back(d2);
        maxe = std::max<int64_t>(maxe, km);
        if (c->schur[lv][mi]) {
          // s1 = S^{-T} (g1 - V^T g2);  s2 = g2 - W^T s1
          g2.add(gd(Vlb, 1, k, s2, m, 1, s1, m, 1, s1, m, 1, k, m, k, -1.0, 1.0));
          ts.add(lu, pv, k, k, s1, m, m, 1, 1.0);
          g3.add(gd(Wrt, 1, k, s1, m, 1, s2, m, 1, s2, m, 1, k, m, k, -1.0, 1.0));
        } else {
          ts.add(lu, pv, 2 * k, 2 * k, s2, m, m, 1, 1.0);  // M^T [s2; s1] = [g2; g1]
        }
        // y_{b,top} -= s1;  y_{b-1,bot} -= s2
        g4.add(gd(c->ident, k, 1, s1, m, 1, YB(mg.b, 0), m, 1, YB(mg.b, 0), m, 1, k, m, k, -1.0, 1.0));
        g4.add(gd(c->ident, k, 1, s2, m, 1, YB(mg.b - 1, 1), m, 1, YB(mg.b - 1, 1), m, 1, k, m, k, -1.0, 1.0));
      }
      pp.gemm(gpart);
      pp.sums(sums, maxe);
      pp.gemm(g2);
      pp.trs(ts);
      pp.gemm(g3);
      pp.gemm(g4);
    }
    mark(2);
    if (!rg.tail) return;
    // ---------------- D^T stage (Eq. sweeps_in_D): X_i = L^{-T}(w + U^{-T}[y_top; 0; y_bot])
    pp.key(3, 0);
    memset_op(Hmem, Hbytes);
    GemmBatch gp;
    std::vector<SweepDesc> sc(nlv, empty_sweep()), sd(nlv, empty_sweep());
    for (int i = 0; i < nlv; ++i) {
      if (!own(i)) continue;
      const LeafDev &L = c->hl[i];
      const int nl = (int)L.len;
      const View fv = rview(L, W), hv = rview(L, H);
      if (i > 0)
        gp.add(typed(gd(nullptr, 0, 0, nullptr, 0, 0, YB(i, 0), m, 1, rows(H, L.start), m, 1, k, m, 0, 0.0, 1.0), tC));
      if (i + 1 < nlv)
        gp.add(typed(gd(nullptr, 0, 0, nullptr, 0, 0, YB(i, 1), m, 1, rows(H, L.start + L.len - k), m, 1, k, m, 0,
                        0.0, 1.0),
                     tC));
      if (L.top_nbr && L.bot_nbr) sc[i] = sdesc(c, i, UT, 0, nl, m, hv, nullptr, none, 0, hv);
      else if (L.bot_nbr) sc[i] = sdesc(c, i, UT, nl - k, nl, m, hv, nullptr, none, 0, hv);
      SweepDesc d = sdesc(c, i, LT, 0, nl, m, fv, nullptr, none, 0, fv);
      if (!piv) {
        d.gb = hv.p;
        d.gb_rs = hv.rs;
        d.gb_cs = hv.cs;
        d.gb_scale = 1.0;
      }
      sd[i] = d;
    }
    pp.gemm(gp);
    if (piv) {
      // W += H, then the pivoted L^T sweep in place
      std::vector<SweepDesc> e0 = e0_dummy(nlv);
      pp.stage(sc, e0, -1, -1, c->ldf, c->dofs, k);
      const int64_t cnt = n * (int64_t)m;
      double *Wd = (double *)W, *Hd = (double *)H;
      pp.op([=](char *) { return launch_axpy(Wd, Hd, 1.0, cnt, s); });
      std::vector<SweepDesc> e1 = e0_dummy(nlv);
      pp.stage(sd, e1, LT, -1, c->ldf, c->dofs, k);
    } else {
      pp.stage(sc, sd, -1, -1, c->ldf, c->dofs, k);
    }
  }
}

constexpr size_t kGraphCache = 16;

static void drop_graph(GraphEntry &g, cudaStream_t s) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.args) cudaFreeAsync(g.args, s);
  g.exec = nullptr;
  g.args = nullptr;
}

// Capture the recorded launches of a solve into a CUDA graph with its own descriptor
// buffer, keep it in the handle's cache (least recently used one replaced) and launch it.
static int capture_solve(spike_ctx *c, Pipeline &pp, cudaStream_t s, int m, int tr, const double *F, int64_t ld,
                         const char *scratch) {
  GraphEntry g;
  g.m = m;
  g.tr = tr;
  g.F = F;
  g.ld = ld;
  g.scratch = scratch;
  if (!pp.ar.h.empty()) {
    SP_CUDA(dev_alloc((void **)&g.args, pp.ar.h.size(), s));
    SP_CUDA(cudaMemcpyAsync(g.args, pp.ar.h.data(), pp.ar.h.size(), cudaMemcpyHostToDevice, s));
  }
  cudaGraph_t graph = nullptr;
  SP_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  const int rc = pp.run_ops(g.args);
  const cudaError_t ec = cudaStreamEndCapture(s, &graph);
  if (rc != 0 || ec != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    if (g.args) cudaFreeAsync(g.args, s);
    if (rc != 0) return rc;
    g_cuda_err = std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ec);
    return SPIKE_ECUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    if (g.args) cudaFreeAsync(g.args, s);
    g_cuda_err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei);
    return SPIKE_ECUDA;
  }
  g.last = ++c->gtick;
  ++c->graph_captures;
  if (c->gcache.size() >= kGraphCache) {
    auto lru = std::min_element(c->gcache.begin(), c->gcache.end(),
                                [](const GraphEntry &a, const GraphEntry &b) { return a.last < b.last; });
    drop_graph(*lru, s);
    c->gcache.erase(lru);
  }
  c->gcache.push_back(g);
  SP_CUDA(cudaGraphLaunch(g.exec, s));
  return 0;
}

// The solve.  Scratch comes from `ws` (ws_bytes) when given, else from the handle's own
// buffer (grown on demand).  With need != nullptr only the scratch size is computed
// (F may then be null; host_f says whether F would be host memory).
static int solve_impl(spike_handle h, double *F, int64_t ldf, int nrhs, char trans, char *ws, int64_t ws_bytes,
                      int64_t *need, bool host_f) {
  if (need) *need = 0;
  if (!valid(h)) return SPIKE_EHANDLE;
  if (!F && !need) return -2;
  spike_ctx *c = h;
  if (c->shard) return SPIKE_ENOTSUP;  // a rank's part: spike_shard_solve
  const int64_t n = c->pl.n;
  if (ldf < n) return -3;
  if (nrhs < 0) return -4;
  const int tr = (trans == 'N' || trans == 'n') ? 0 : ((trans == 'T' || trans == 't' || trans == 'C' || trans == 'c') ? 1 : -1);
  if (tr < 0) return -5;
  if (c->pivot && c->zero_col) return (int)std::min<int64_t>(c->zero_col, INT_MAX);
  if (nrhs == 0) return 0;
  const int k = c->k, nlv = c->nleaves, m = nrhs;
  const int64_t km = (int64_t)k * m;
  const size_t es = c->es;
  cudaStream_t s = c->stream;

  // Work layout: the sweeps run on a ROW-major copy W of F (row r holds the m
  // right-hand-side entries contiguously), so a block row and its window rows
  // touch a few contiguous lines instead of m lines n*8 bytes apart.
  const bool fdev = need ? !host_f : is_device_ptr(F);
  const bool mixed = c->f32 != 0;
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    size_t o = off;
    off = (off + bytes + 255) & ~size_t(255);
    return o;
  };
  const size_t nm8 = sizeof(double) * (size_t)n * m;
  const size_t o_f = fdev ? 0 : carve(nm8);
  const size_t o_w = (m > 1 || mixed) ? carve(es * (size_t)n * m) : 0;
  const size_t o_h = carve(es * (size_t)n * m);
  const size_t o_y = carve(sizeof(double) * (size_t)nlv * 2 * km);
  size_t maxm = 1;
  for (auto &lvv : c->pl.levels) maxm = std::max(maxm, lvv.size());
  const size_t o_t = carve(sizeof(double) * maxm * 2 * km);
  const size_t o_p = carve(sizeof(double) * (size_t)nlv * km);
  // mixed precision: F0 (the right-hand side), X (FP64 solution), R (residual), norms
  const size_t o_f0 = mixed ? carve(nm8) : 0;
  const size_t o_x = mixed ? carve(nm8) : 0;
  const size_t o_r = mixed ? carve(nm8) : 0;
  const size_t o_nrm = mixed ? carve(sizeof(unsigned long long) * (1 + 2 * (size_t)m)) : 0;
  const size_t o_act = mixed ? carve(sizeof(int) * (size_t)m) : 0;
  // tensor-core residual: the digit planes of X (for 8 or more columns; fewer take the FP64 kernel,
  // except on batch-invariant handles, whose columns must get the same bits in any solve: the
  // tensor-core residual computes each column exactly from its own digits whatever the count)
  const bool split = mixed && c->sfrag[0] != nullptr && (m >= 8 || c->invariant);
  const size_t xdig_bytes = split ? split_x_bytes(n, c->pl.kl, c->pl.ku, m) : 0;
  const size_t o_xd = split ? carve(xdig_bytes) : 0;
  if (need) {
    *need = (int64_t)off;
    return 0;
  }
  char *base;
  if (ws) {
    if (ws_bytes < (int64_t)off) return -7;
    base = ws;
  } else {
    SP_TRY(ensure(&c->scr, &c->scr_bytes, off, s));
    base = c->scr;
  }
  double *Fd = F;
  int64_t ld = ldf;
  if (!fdev) {
    Fd = (double *)(base + o_f);
    ld = n;
    SP_CUDA(cudaMemcpy2DAsync(Fd, sizeof(double) * n, F, sizeof(double) * ldf, sizeof(double) * n, m,
                              cudaMemcpyHostToDevice, s));
  }
  SolveBufs B;
  B.W = (m > 1 || mixed) ? (void *)(base + o_w) : (void *)Fd;  // FP64, m == 1: column-major == row-major
  B.H = base + o_h;
  B.Y = (double *)(base + o_y);
  B.TM = (double *)(base + o_t);
  B.PP = (double *)(base + o_p);
  cudaEvent_t *evs = tr ? c->tev : c->nev;

  // SPIKE_FLAG_GRAPHS: FP64 solves of device buffers are replayed from a CUDA graph once the
  // same call has been seen before (the first run also sets every kernel attribute, so the
  // capture contains launches, memsets and device copies only)
  // (stream capture needs a stream other than the legacy default one)
  const bool use_graph = !mixed && c->graphs && fdev && !c->timing && s != nullptr && s != cudaStreamLegacy;
  GraphEntry *hit = nullptr;
  bool capture = false;
  if (use_graph) {
    auto same = [&](const GraphEntry &g) {
      return g.m == m && g.tr == tr && g.F == Fd && g.ld == ld && g.scratch == base;
    };
    for (auto &g : c->gcache)
      if (same(g)) hit = &g;
    if (hit) {
      hit->last = ++c->gtick;
      ++c->graph_replays;
      SP_CUDA(cudaGraphLaunch(hit->exec, s));
      return 0;
    }
    for (auto &g : c->gseen)
      if (same(g)) capture = true;
    if (!capture) {
      GraphEntry g;
      g.m = m;
      g.tr = tr;
      g.F = Fd;
      g.ld = ld;
      g.scratch = base;
      if (c->gseen.size() >= 16) c->gseen.erase(c->gseen.begin());
      c->gseen.push_back(g);
    }
  }
  if (!mixed) {
    Pipeline pp;
    pp.st = s;
    if (c->timing) {
      cudaEvent_t e = evs[0];
      pp.ops.push_back([=](char *) { return (int)cudaEventRecord(e, s); });
    }
    if (m > 1) {
      double *src = Fd, *dst = (double *)B.W;
      const int64_t ldx = ld;
      pp.ops.push_back([=](char *) { return launch_transpose(src, dst, n, m, ldx, 1, s); });
    }
    build_solve(c, pp, B, m, tr, true);
    if (m > 1) {
      double *src = (double *)B.W, *dst = Fd;
      const int64_t ldx = ld;
      pp.ops.push_back([=](char *) { return launch_transpose(src, dst, n, m, ldx, 0, s); });
    }
    if (c->timing) {
      cudaEvent_t e = evs[3];
      pp.ops.push_back([=](char *) { return (int)cudaEventRecord(e, s); });
    }
    if (capture) {
      SP_TRY(capture_solve(c, pp, s, m, tr, Fd, ld, base));
      return 0;
    }
    SP_TRY(pp.run(c));
    if (c->timing) (tr ? c->tdone : c->ndone) = true;
  } else {
    // FP64 iterative refinement around the FP32 SPIKE solve.  Each column stops
    // (its x is frozen) at the first step whose backward error is <= SPIKE_MIXED_TOL,
    // so a column's result does not depend on the other columns solved with it.
    double *F0 = (double *)(base + o_f0), *X = (double *)(base + o_x), *R = (double *)(base + o_r);
    unsigned long long *nrm = (unsigned long long *)(base + o_nrm);
    int *dact = (int *)(base + o_act);
    std::vector<int> act((size_t)m, 1);
    SP_CUDA(cudaMemcpyAsync(dact, act.data(), sizeof(int) * (size_t)m, cudaMemcpyHostToDevice, s));
    if (c->timing) SP_CUDA(cudaEventRecord(evs[0], s));
    SP_CUDA(cudaMemcpy2DAsync(F0, sizeof(double) * n, Fd, sizeof(double) * ld, sizeof(double) * n, m,
                              cudaMemcpyDeviceToDevice, s));
    SP_CUDA(cudaMemsetAsync(X, 0, nm8, s));
    void *xdig = split ? (void *)(base + o_xd) : nullptr;
    if (split) SP_CUDA(cudaMemsetAsync(xdig, 0x40, xdig_bytes, s));  // digit 0 around every column
    const double *rhs = F0;  // first step: x = 0, r = F
    int steps = 0;
    double worst = INFINITY;
    std::vector<unsigned long long> hn(1 + 2 * (size_t)m);
    for (;;) {
      Pipeline pp;
      pp.st = s;
      pp.f32 = 1;
      {
        const double *src = rhs;
        float *dst = (float *)B.W;
        pp.ops.push_back([=](char *) { return launch_to_work32(src, n, dst, n, m, s); });
      }
      build_solve(c, pp, B, m, tr, steps == 0);
      {
        const float *d = (const float *)B.W;
        pp.ops.push_back([=](char *) { return launch_add_work32(X, n, d, n, m, dact, s); });
      }
      // r = F - op(A) x (FP64-accurate, original band) and the per-column backward errors
      if (split) {
        const void *fr = c->sfrag[tr];
        const int *rx = c->srexp[tr];
        const unsigned long long *an = c->snorm + tr;
        const int kl = c->pl.kl, ku = c->pl.ku;
        pp.ops.push_back([=](char *) {
          return launch_resid_split(fr, rx, an, n, kl, ku, tr, X, F0, R, m, xdig, nrm, s);
        });
      } else {
        pp.ops.push_back([=](char *) { return (int)cudaMemsetAsync(nrm, 0, sizeof(unsigned long long) * (1 + 2 * (size_t)m), s); });
        const double *band = c->band64;
        const int64_t ldb = c->ldab64;
        const int kl = c->pl.kl, ku = c->pl.ku;
        pp.ops.push_back([=](char *) { return launch_residual(band, ldb, n, kl, ku, X, F0, R, m, tr, nrm, s); });
      }
      SP_TRY(pp.run(c));
      ++steps;
      SP_CUDA(cudaMemcpyAsync(hn.data(), nrm, sizeof(unsigned long long) * hn.size(), cudaMemcpyDeviceToHost, s));
      SP_CUDA(cudaStreamSynchronize(s));
      auto as_d = [](unsigned long long b) {
        double d;
        memcpy(&d, &b, sizeof(d));
        return d;
      };
      const double an = as_d(hn[0]);
      worst = 0.0;
      bool any = false, changed = false;
      for (int col = 0; col < m; ++col) {
        const double r = as_d(hn[1 + 2 * col]), x = as_d(hn[2 + 2 * col]);
        const double be = (an > 0 && x > 0) ? r / (an * x) : (r == 0 ? 0.0 : INFINITY);
        worst = std::max(worst, be);
        if (!act[col]) continue;
        if (be > c->refine_tol) {
          any = true;
        } else {
          act[col] = 0;
          changed = true;
        }
      }
      if (!any || steps >= SPIKE_MIXED_MAX_STEPS) break;
      if (changed) SP_CUDA(cudaMemcpyAsync(dact, act.data(), sizeof(int) * (size_t)m, cudaMemcpyHostToDevice, s));
      rhs = R;
    }
    c->last_iters = steps;
    c->last_berr = worst;
    SP_CUDA(cudaMemcpy2DAsync(Fd, sizeof(double) * ld, X, sizeof(double) * n, sizeof(double) * n, m,
                              cudaMemcpyDeviceToDevice, s));
    if (c->timing) {
      SP_CUDA(cudaEventRecord(evs[3], s));
      (tr ? c->tdone : c->ndone) = true;
    }
  }
  if (!fdev) {
    SP_CUDA(cudaMemcpy2DAsync(F, sizeof(double) * ldf, Fd, sizeof(double) * n, sizeof(double) * n, m,
                              cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaStreamSynchronize(s));
  }
  return 0;
}

// ============================================================ sharded solves
// Partition-range sharding over ranks (NEXT to Sec. 3's SPIKE-MPI remark; the recursion of
// Sec. 2.2 across ranks).  Each rank holds its own blocks and rows; the merge levels inside
// a rank run locally, and every level above them is one exchange: the caller all-gathers a
// fixed-size buffer from every rank (spike_shard_pending / _export), hands the gathered
// buffers back (spike_shard_import) and the handle runs that level for the merge that
// contains its blocks.  What a level needs from the other ranks is only the spike or
// right-hand-side tips at the rank boundaries (k x k per spike in the factorization, k x m
// in the solves), or, for the transposed solve, one k x m partial product per rank.
enum ShardOp { SH_NONE = 0, SH_FACTOR = 1, SH_N_LEVEL = 2, SH_N_FINAL = 3, SH_T_GTIPS = 4, SH_T_LEVEL = 5 };

// the merge of level lv that contains this rank's blocks (index in the level)
static int shard_merge(spike_ctx *c, int lv) {
  const auto &ms = c->pl.levels[lv];
  for (int mi = 0; mi < (int)ms.size(); ++mi)
    if (ms[mi].a <= c->l0 && c->l1 <= ms[mi].c) return mi;
  return -1;
}

// rank whose first block is `leaf` (merge boundaries above the local levels are rank boundaries)
static int shard_rank_at(spike_ctx *c, int leaf) {
  for (int g = 0; g <= c->nranks; ++g)
    if (c->leaf_first[g] == leaf) return g;
  return -1;
}

struct ShardBufs {
  double *Wm, *Hm;  // the rank's rows of the work arrays (row-major, nrow x m)
  SolveBufs B;      // the same with W, H offset by -row0 (global row indexing)
  double *XP;       // the transposed solve's partial product (k x m)
};

static ShardBufs shard_bufs(spike_ctx *c, int m, size_t *bytes) {
  size_t off = 0;
  auto carve = [&](size_t b) {
    size_t o = off;
    off = (off + b + 255) & ~size_t(255);
    return o;
  };
  const int64_t km = (int64_t)c->k * m;
  const size_t rows = sizeof(double) * (size_t)c->nrow * m;
  size_t maxm = 1;
  for (auto &lvv : c->pl.levels) maxm = std::max(maxm, lvv.size());
  const size_t ow = carve(rows), oh = carve(rows), oy = carve(sizeof(double) * (size_t)c->nleaves * 2 * km),
               ot = carve(sizeof(double) * maxm * 2 * km), op = carve(sizeof(double) * (size_t)c->nleaves * km),
               ox = carve(sizeof(double) * km);
  ShardBufs S;
  memset(&S, 0, sizeof(S));
  if (bytes) {
    *bytes = off;
    return S;
  }
  char *base = c->scr;
  if (!base) return S;  // no solve scratch yet (a factorization's exchanges)
  S.Wm = (double *)(base + ow);
  S.Hm = (double *)(base + oh);
  S.B.W = (char *)S.Wm - (ptrdiff_t)(c->row0 * m * (int64_t)sizeof(double));
  S.B.H = (char *)S.Hm - (ptrdiff_t)(c->row0 * m * (int64_t)sizeof(double));
  S.B.Y = (double *)(base + oy);
  S.B.TM = (double *)(base + ot);
  S.B.PP = (double *)(base + op);
  S.XP = (double *)(base + ox);
  return S;
}

// The transposed solve's partial product of level lv: sum over this rank's blocks (in block
// order) of V_i^T y_i (the rank is on the left of its merge) or W_i^T y_i (on the right).
static void shard_t_partial(spike_ctx *c, Pipeline &pp, const ShardBufs &S, int m, int lv) {
  const int k = c->k;
  const int64_t km = (int64_t)k * m;
  const Merge &mg = c->pl.levels[lv][shard_merge(c, lv)];
  const int sp = (c->l0 < mg.b) ? 0 : 1;
  GemmBatch gpart;
  for (int i = c->l0; i < c->l1; ++i)
    gpart.add(gd(TIP(c, lv, sp, i, 0), 1, k, S.B.Y + (int64_t)i * 2 * km, m, 1, nullptr, 0, 0,
                 S.B.PP + (int64_t)i * km, m, 1, k, m, 2 * k, 1.0, 0.0));
  pp.gemm(gpart);
  std::vector<SumDesc> sums{SumDesc{S.B.PP + (int64_t)c->l0 * km, S.XP, km, km, c->l1 - c->l0, 0}};
  pp.sums(sums, km);
}

// One merge level above the rank (N solve, Eqs. D1Inverse / S2Inverse): the 2k interface solve
// of the rank's merge from the gathered boundary tips, then the updates of this rank's tips.
static void shard_n_level(spike_ctx *c, Pipeline &pp, const ShardBufs &S, int m, int lv) {
  const int k = c->k;
  const int64_t kk = (int64_t)k * k, km = (int64_t)k * m;
  const int mi = shard_merge(c, lv);
  const Merge &mg = c->pl.levels[lv][mi];
  double *Y = S.B.Y;
  auto YB = [&](int i, int t) { return Y + ((int64_t)i * 2 + t) * km; };
  const int64_t gm = c->merge_off[lv] + mi;
  const double *lu = c->mlu + gm * 4 * kk;
  const int *pv = c->mpiv + gm * 2 * k;
  double *ta = S.B.TM, *tb = ta + km;
  const int b = mg.b;
  const double *Vlb = TIP(c, lv, 0, b - 1, 1), *Wrt = TIP(c, lv, 1, b, 0);
  GemmBatch g1, g2, g3;
  TrsBatch ts;
  if (c->schur[lv][mi]) {
    g1.add(gd(Wrt, k, 1, YB(b - 1, 1), m, 1, YB(b, 0), m, 1, tb, m, 1, k, m, k, -1.0, 1.0));
    ts.add(lu, pv, k, k, tb, m, m, 0, 1.0);
    g2.add(gd(Vlb, k, 1, tb, m, 1, YB(b - 1, 1), m, 1, ta, m, 1, k, m, k, -1.0, 1.0));
  } else {
    g1.add(gd(nullptr, 0, 0, nullptr, 0, 0, YB(b - 1, 1), m, 1, ta, m, 1, k, m, 0, 0.0, 1.0));
    g1.add(gd(nullptr, 0, 0, nullptr, 0, 0, YB(b, 0), m, 1, tb, m, 1, k, m, 0, 0.0, 1.0));
    ts.add(lu, pv, 2 * k, 2 * k, ta, m, m, 0, 1.0);
  }
  // y_L -= V_L b on this rank's left-side tips, y_R -= W_R a on its right-side tips; the
  // interface tips (b-1, bottom) and (b, top) are a and b themselves
  const int la = std::max(mg.a, c->l0), lb = std::min(b, c->l1);
  const int ra = std::max(b, c->l0), rb = std::min(mg.c, c->l1);
  if (lb > la) {
    const int last = (lb == b) ? 1 : 0;
    const int ML = (2 * (lb - la) - last) * k;
    g3.add(gd(TIP(c, lv, 0, la, 0), k, 1, tb, m, 1, YB(la, 0), m, 1, YB(la, 0), m, 1, ML, m, k, -1.0, 1.0));
    if (last) g3.add(gd(nullptr, 0, 0, nullptr, 0, 0, ta, m, 1, YB(b - 1, 1), m, 1, k, m, 0, 0.0, 1.0));
  }
  if (rb > ra) {
    const int first = (ra == b) ? 1 : 0;
    const int MR = (2 * (rb - ra) - first) * k;
    g3.add(gd(TIP(c, lv, 1, ra, first), k, 1, ta, m, 1, YB(ra, first), m, 1, YB(ra, first), m, 1, MR, m, k, -1.0,
              1.0));
    if (first) g3.add(gd(nullptr, 0, 0, nullptr, 0, 0, tb, m, 1, YB(b, 0), m, 1, k, m, 0, 0.0, 1.0));
  }
  pp.gemm(g1);
  pp.trs(ts);
  pp.gemm(g2);
  pp.gemm(g3);
}

// One merge level above the rank (transposed solve, Sec. 4.3): g1 / g2 are the sums of the
// gathered partial products of the left / right ranks (rank order), then the transposed
// interface solve and the updates of the interface tips this rank holds.
static void shard_t_level(spike_ctx *c, Pipeline &pp, const ShardBufs &S, int m, int lv, const double *recv) {
  const int k = c->k;
  const int64_t kk = (int64_t)k * k, km = (int64_t)k * m;
  const int mi = shard_merge(c, lv);
  const Merge &mg = c->pl.levels[lv][mi];
  double *Y = S.B.Y;
  auto YB = [&](int i, int t) { return Y + ((int64_t)i * 2 + t) * km; };
  const int64_t gm = c->merge_off[lv] + mi;
  const double *lu = c->mlu + gm * 4 * kk;
  const int *pv = c->mpiv + gm * 2 * k;
  double *s2 = S.B.TM, *s1 = s2 + km;  // [g2; g1] -> [s2; s1]
  const int gl0 = shard_rank_at(c, mg.a), gl1 = shard_rank_at(c, mg.b), gr1 = shard_rank_at(c, mg.c);
  std::vector<SumDesc> sums{SumDesc{recv + (int64_t)gl0 * km, s1, km, km, gl1 - gl0, 0},
                            SumDesc{recv + (int64_t)gl1 * km, s2, km, km, gr1 - gl1, 0}};
  pp.sums(sums, km);
  const int b = mg.b;
  const double *Vlb = TIP(c, lv, 0, b - 1, 1), *Wrt = TIP(c, lv, 1, b, 0);
  GemmBatch g2, g3, g4;
  TrsBatch ts;
  if (c->schur[lv][mi]) {
    g2.add(gd(Vlb, 1, k, s2, m, 1, s1, m, 1, s1, m, 1, k, m, k, -1.0, 1.0));
    ts.add(lu, pv, k, k, s1, m, m, 1, 1.0);
    g3.add(gd(Wrt, 1, k, s1, m, 1, s2, m, 1, s2, m, 1, k, m, k, -1.0, 1.0));
  } else {
    ts.add(lu, pv, 2 * k, 2 * k, s2, m, m, 1, 1.0);
  }
  if (b >= c->l0 && b < c->l1)
    g4.add(gd(c->ident, k, 1, s1, m, 1, YB(b, 0), m, 1, YB(b, 0), m, 1, k, m, k, -1.0, 1.0));
  if (b - 1 >= c->l0 && b - 1 < c->l1)
    g4.add(gd(c->ident, k, 1, s2, m, 1, YB(b - 1, 1), m, 1, YB(b - 1, 1), m, 1, k, m, k, -1.0, 1.0));
  pp.gemm(g2);
  pp.trs(ts);
  pp.gemm(g3);
  pp.gemm(g4);
}

// copy `rows` x m of the work array back to the caller's F (column-major)
static void shard_finish(spike_ctx *c, Pipeline &pp, const ShardBufs &S, int m) {
  double *src = S.Wm, *dst = c->sh_F;
  const int64_t rows = c->nrow, ld = c->sh_ld;
  cudaStream_t s = c->stream;
  pp.ops.push_back([=](char *) { return launch_transpose(src, dst, rows, m, ld, 0, s); });
}

extern "C" int spike_shard_factor(const double *band, int64_t ldab, int64_t col0, int64_t n, int kl, int ku, int p,
                                  int rank, int nranks, const spike_options *opt, spike_handle *out) {
  if (!out) return -11;
  *out = nullptr;
  if (!band) return -1;
  if (n < 1) return -4;
  if (kl < 0) return -5;
  if (ku < 0) return -6;
  if (ldab < (int64_t)kl + ku + 1) return -2;
  if (p < 1) return -7;
  if (nranks < 1) return -9;
  if (rank < 0 || rank >= nranks) return -8;
  if (col0 < 0) return -3;
  ShardSpec sh{rank, nranks, col0};
  const int rc = factor_impl(band, ldab, n, kl, ku, p, 0, opt, out, &sh);
  // factor_impl numbers arguments as spike_factor_ex (n, kl, ku, p = -3..-6); -3 and -9 here
  // are its shard checks (col0 past the rank's first column, a rank count the plan cannot take)
  switch (rc) {
    case -4: return -5;
    case -5: return -6;
    case -6: return -7;
    default: return rc;
  }
}

extern "C" int spike_shard_pending(spike_handle h, int64_t *count) {
  if (!valid(h)) return SPIKE_EHANDLE;
  if (!count) return -2;
  const int64_t k = h->k, m = h->sh_m;
  switch (h->sh_op) {
    case SH_FACTOR: *count = 4 * k * k; break;
    case SH_N_LEVEL:
    case SH_N_FINAL:
    case SH_T_GTIPS: *count = 2 * k * m; break;
    case SH_T_LEVEL: *count = k * m; break;
    default: *count = 0;
  }
  return 0;
}

extern "C" int spike_shard_export(spike_handle h, double *send) {
  if (!valid(h)) return SPIKE_EHANDLE;
  if (!send) return -2;
  spike_ctx *c = h;
  cudaStream_t s = c->stream;
  const int64_t kk = (int64_t)c->k * c->k, km = (int64_t)c->k * c->sh_m;
  auto cp = [&](double *dst, const double *src, int64_t cnt) {
    return cudaMemcpyAsync(dst, src, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, s);
  };
  const ShardBufs S = shard_bufs(c, std::max(1, c->sh_m), nullptr);
  auto YB = [&](int i, int t) { return S.B.Y + ((int64_t)i * 2 + t) * km; };
  const int lv = c->sh_level;
  switch (c->sh_op) {
    case SH_FACTOR:
      SP_CUDA(cp(send, TIP(c, lv, 0, c->l0, 0), kk));
      SP_CUDA(cp(send + kk, TIP(c, lv, 1, c->l0, 0), kk));
      SP_CUDA(cp(send + 2 * kk, TIP(c, lv, 0, c->l1 - 1, 1), kk));
      SP_CUDA(cp(send + 3 * kk, TIP(c, lv, 1, c->l1 - 1, 1), kk));
      break;
    case SH_N_LEVEL:
    case SH_N_FINAL:
      SP_CUDA(cp(send, YB(c->l0, 0), km));
      SP_CUDA(cp(send + km, YB(c->l1 - 1, 1), km));
      break;
    case SH_T_GTIPS:  // this rank's corrections of its neighbours' boundary tips (zero at the ends)
      if (c->l0 > 0) SP_CUDA(cp(send, YB(c->l0 - 1, 1), km));
      else SP_CUDA(cudaMemsetAsync(send, 0, sizeof(double) * km, s));
      if (c->l1 < c->nleaves) SP_CUDA(cp(send + km, YB(c->l1, 0), km));
      else SP_CUDA(cudaMemsetAsync(send + km, 0, sizeof(double) * km, s));
      break;
    case SH_T_LEVEL:
      SP_CUDA(cp(send, S.XP, km));
      break;
    default:
      return SPIKE_ENOTSUP;  // no exchange pending
  }
  SP_CUDA(cudaStreamSynchronize(s));
  return 0;
}

extern "C" int spike_shard_import(spike_handle h, const double *recv) {
  if (!valid(h)) return SPIKE_EHANDLE;
  if (!recv) return -2;
  spike_ctx *c = h;
  cudaStream_t s = c->stream;
  const int G = c->nranks, m = std::max(1, c->sh_m);
  const int64_t kk = (int64_t)c->k * c->k, km = (int64_t)c->k * m;
  auto cp = [&](double *dst, const double *src, int64_t cnt) {
    return cudaMemcpyAsync(dst, src, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, s);
  };
  const int lv = c->sh_level;
  if (c->sh_op == SH_FACTOR) {
    for (int g = 0; g < G; ++g) {
      if (g == c->rank) continue;
      const double *r = recv + (int64_t)g * 4 * kk;
      const int f = c->leaf_first[g], l = c->leaf_first[g + 1] - 1;
      SP_CUDA(cp(TIP(c, lv, 0, f, 0), r, kk));
      SP_CUDA(cp(TIP(c, lv, 1, f, 0), r + kk, kk));
      SP_CUDA(cp(TIP(c, lv, 0, l, 1), r + 2 * kk, kk));
      SP_CUDA(cp(TIP(c, lv, 1, l, 1), r + 3 * kk, kk));
    }
    SP_TRY(factor_reduced_level(c, lv, c->sh_fscr + c->sh_tmp_off, c->sh_tmp_bytes));
    c->sh_level = lv + 1;
    if (c->sh_level >= c->NL) {
      unsigned long long st[8];
      SP_CUDA(cudaMemcpyAsync(st, c->status, sizeof(st), cudaMemcpyDeviceToHost, s));
      SP_CUDA(cudaStreamSynchronize(s));
      c->nan_flag = (int)st[2];
      cudaFreeAsync(c->sh_fscr, s);
      c->sh_fscr = nullptr;
      c->sh_op = SH_NONE;
    }
    return 0;
  }
  const ShardBufs S = shard_bufs(c, m, nullptr);
  auto YB = [&](int i, int t) { return S.B.Y + ((int64_t)i * 2 + t) * km; };
  const int tr = (c->sh_op == SH_T_GTIPS || c->sh_op == SH_T_LEVEL) ? 1 : 0;
  Pipeline pp;
  pp.st = s;
  switch (c->sh_op) {
    case SH_N_LEVEL:
      for (int g = 0; g < G; ++g) {
        if (g == c->rank) continue;
        SP_CUDA(cp(YB(c->leaf_first[g], 0), recv + (int64_t)g * 2 * km, km));
        SP_CUDA(cp(YB(c->leaf_first[g + 1] - 1, 1), recv + (int64_t)g * 2 * km + km, km));
      }
      shard_n_level(c, pp, S, m, lv);
      c->sh_level = lv + 1;
      if (c->sh_level >= c->NL) c->sh_op = SH_N_FINAL;
      break;
    case SH_N_FINAL: {
      // the neighbours' boundary solution tips, then the retrieval of this rank's blocks
      if (c->rank > 0) SP_CUDA(cp(YB(c->l0 - 1, 1), recv + (int64_t)(c->rank - 1) * 2 * km + km, km));
      if (c->rank + 1 < G) SP_CUDA(cp(YB(c->l1, 0), recv + (int64_t)(c->rank + 1) * 2 * km, km));
      SolveRange rg;
      rg.head = false;
      rg.lv_lo = rg.lv_hi = c->NL;
      build_solve(c, pp, S.B, m, 0, false, rg);
      shard_finish(c, pp, S, m);
      c->sh_op = SH_NONE;
      break;
    }
    case SH_T_GTIPS: {
      GemmBatch ga;
      if (c->rank > 0)
        ga.add(gd(c->ident, c->k, 1, recv + (int64_t)(c->rank - 1) * 2 * km + km, m, 1, YB(c->l0, 0), m, 1,
                  YB(c->l0, 0), m, 1, c->k, m, c->k, 1.0, 1.0));
      if (c->rank + 1 < G)
        ga.add(gd(c->ident, c->k, 1, recv + (int64_t)(c->rank + 1) * 2 * km, m, 1, YB(c->l1 - 1, 1), m, 1,
                  YB(c->l1 - 1, 1), m, 1, c->k, m, c->k, 1.0, 1.0));
      pp.gemm(ga);
      c->sh_level = c->NL - 1;
      shard_t_partial(c, pp, S, m, c->sh_level);
      c->sh_op = SH_T_LEVEL;
      break;
    }
    case SH_T_LEVEL:
      shard_t_level(c, pp, S, m, lv, recv);
      if (lv - 1 >= c->lvl) {
        c->sh_level = lv - 1;
        shard_t_partial(c, pp, S, m, lv - 1);
      } else {
        SolveRange rg;
        rg.head = false;
        rg.lv_lo = 0;
        rg.lv_hi = c->lvl;
        build_solve(c, pp, S.B, m, 1, false, rg);
        shard_finish(c, pp, S, m);
        c->sh_op = SH_NONE;
      }
      break;
    default:
      return SPIKE_ENOTSUP;
  }
  (void)tr;
  return pp.run(c);
}

extern "C" int spike_shard_solve(spike_handle h, double *F, int64_t ldf, int nrhs, char trans) {
  if (!valid(h)) return SPIKE_EHANDLE;
  spike_ctx *c = h;
  if (!c->shard || c->f32 || c->pivot) return SPIKE_ENOTSUP;
  if (c->sh_op != SH_NONE) return SPIKE_ENOTSUP;  // the previous operation still has exchanges to run
  if (!F) return -2;
  if (ldf < c->nrow) return -3;
  if (nrhs < 1) return -4;
  const int tr = (trans == 'N' || trans == 'n') ? 0 : ((trans == 'T' || trans == 't') ? 1 : -1);
  if (tr < 0) return -5;
  if (!is_device_ptr(F)) return SPIKE_ENOTSUP;
  const int m = nrhs;
  cudaStream_t s = c->stream;
  size_t need = 0;
  shard_bufs(c, m, &need);
  SP_TRY(ensure(&c->scr, &c->scr_bytes, need, s));
  const ShardBufs S = shard_bufs(c, m, nullptr);
  c->sh_F = F;
  c->sh_ld = ldf;
  c->sh_m = m;
  Pipeline pp;
  pp.st = s;
  {
    double *src = F, *dst = S.Wm;
    const int64_t rows = c->nrow;
    pp.ops.push_back([=](char *) { return launch_transpose(src, dst, rows, m, ldf, 1, s); });
  }
  const bool alone = c->nranks == 1;
  SolveRange rg;
  rg.tail = alone;
  rg.lv_lo = 0;
  rg.lv_hi = (tr == 0 || alone) ? c->lvl : 0;  // T runs the local levels last (descending)
  build_solve(c, pp, S.B, m, tr, false, rg);
  if (alone) {
    shard_finish(c, pp, S, m);
    c->sh_op = SH_NONE;
  } else if (tr == 0) {
    c->sh_op = SH_N_LEVEL;
    c->sh_level = c->lvl;
  } else {
    c->sh_op = SH_T_GTIPS;
  }
  return pp.run(c);
}

extern "C" int spike_solve_ex(spike_handle h, double *F, int64_t ldf, int nrhs, char trans) {
  return solve_impl(h, F, ldf, nrhs, trans, nullptr, 0, nullptr, false);
}

extern "C" int spike_solve_workspace(spike_handle h, int nrhs, char trans, int host_f, int64_t *bytes) {
  if (!bytes) return -5;
  *bytes = 0;
  if (!valid(h)) return SPIKE_EHANDLE;
  if (nrhs < 0) return -2;
  if (trans != 'N' && trans != 'n' && trans != 'T' && trans != 't' && trans != 'C' && trans != 'c') return -3;
  return solve_impl(h, nullptr, h->pl.n, nrhs, trans, nullptr, 0, bytes, host_f != 0);
}

extern "C" int spike_solve_ws(spike_handle h, double *F, int64_t ldf, int nrhs, char trans, void *workspace,
                              int64_t ws_bytes) {
  if (!workspace) return -6;
  return solve_impl(h, F, ldf, nrhs, trans, (char *)workspace, ws_bytes, nullptr, false);
}

// ============================================================== batched solve
// Several systems solved together: each system's solve is recorded as keyed phases
// (Pipeline::rec), the phases with equal keys are merged, and every merged phase is one
// launch.  Scratch per system as in solve_impl (FP64, device F); the merged descriptor
// arena follows the systems' scratch in the workspace.
static int solve_batch_impl(const spike_handle *hs, double *const *F, const int *nrhs, int count, char trans,
                            cudaStream_t s, char *ws, int64_t ws_bytes, int64_t *need) {
  if (need) *need = 0;
  if (!hs) return -1;
  if (!F && !need) return -2;
  if (!nrhs) return -3;
  if (count < 0) return -4;
  const int tr = (trans == 'N' || trans == 'n') ? 0 : ((trans == 'T' || trans == 't' || trans == 'C' || trans == 'c') ? 1 : -1);
  if (tr < 0) return -5;
  auto align = [](size_t x) { return (x + 255) & ~size_t(255); };
  struct Sys {
    size_t off, o_w, o_h, o_y, o_t, o_p;
  };
  std::vector<Sys> sys((size_t)count);
  size_t total = 0;
  for (int i = 0; i < count; ++i) {
    spike_ctx *c = hs[i];
    if (!valid(c)) return SPIKE_EHANDLE;
    if (c->f32 || c->pivot || c->shard) return SPIKE_ENOTSUP;
    if (nrhs[i] < 0) return -3;
    const int64_t n = c->pl.n, m = nrhs[i], km = (int64_t)c->k * m;
    size_t maxm = 1;
    for (auto &lvv : c->pl.levels) maxm = std::max(maxm, lvv.size());
    Sys &S = sys[i];
    S.off = total;
    size_t o = 0;
    auto carve = [&](size_t bytes) {
      size_t r = o;
      o = align(o + bytes);
      return r;
    };
    S.o_w = m > 1 ? carve(sizeof(double) * (size_t)n * m) : 0;
    S.o_h = carve(sizeof(double) * (size_t)n * m);
    S.o_y = carve(sizeof(double) * (size_t)c->nleaves * 2 * km);
    S.o_t = carve(sizeof(double) * maxm * 2 * km);
    S.o_p = carve(sizeof(double) * (size_t)c->nleaves * km);
    total += m > 0 ? o : 0;
  }
  std::map<PhaseKey, Phase> merged;
  for (int i = 0; i < count; ++i) {
    spike_ctx *c = hs[i];
    const int m = nrhs[i];
    if (m == 0) continue;
    const int64_t n = c->pl.n;
    char *base = (ws ? ws : (char *)nullptr) + sys[i].off;  // sizing pass: pointers are never used
    double *Fi = F ? F[i] : nullptr;
    if (!need && !Fi) return -2;
    SolveBufs B;
    B.W = m > 1 ? (void *)(base + sys[i].o_w) : (void *)Fi;
    B.H = base + sys[i].o_h;
    B.Y = (double *)(base + sys[i].o_y);
    B.TM = (double *)(base + sys[i].o_t);
    B.PP = (double *)(base + sys[i].o_p);
    std::map<PhaseKey, Phase> ph;
    Pipeline pr;
    pr.st = s;
    pr.rec = &ph;
    if (m > 1) {
      double *src = Fi, *dst = (double *)B.W;
      pr.key(-1, 0);
      pr.op([=](char *) { return launch_transpose(src, dst, n, m, n, 1, s); });
    }
    build_solve(c, pr, B, m, tr, false);
    if (m > 1) {
      double *src = (double *)B.W, *dst = Fi;
      pr.key(9, 0);
      pr.op([=](char *) { return launch_transpose(src, dst, n, m, n, 0, s); });
    }
    for (auto &kv : ph) merge_phase(merged[kv.first], kv.second);
  }
  const size_t q_off = align(total), q_bytes = 4096;  // work-queue counters of the sweep stages
  const size_t args_off = q_off + q_bytes;
  Pipeline pp;
  pp.st = s;
  pp.queue_base = (unsigned int *)((ws ? ws : (char *)nullptr) + q_off);
  pp.max_queue = (int)(q_bytes / sizeof(unsigned int));
  for (auto &kv : merged) pp.emit(kv.second);
  const int64_t want = (int64_t)(args_off + pp.ar.h.size());
  if (need) {
    *need = want;
    return 0;
  }
  if (!ws) return -7;
  if (ws_bytes < want) return -8;
  char *args = ws + args_off;
  if (!pp.ar.h.empty()) SP_CUDA(cudaMemcpyAsync(args, pp.ar.h.data(), pp.ar.h.size(), cudaMemcpyHostToDevice, s));
  return pp.run_ops(args);
}

extern "C" int spike_solve_batch_workspace(const spike_handle *hs, const int *nrhs, int count, char trans,
                                           int64_t *bytes) {
  if (!bytes) return -5;
  const int rc = solve_batch_impl(hs, nullptr, nrhs, count, trans, nullptr, nullptr, 0, bytes);
  return rc == -3 ? -2 : (rc == -4 ? -3 : (rc == -5 ? -4 : rc));  // argument positions of this entry point
}

extern "C" int spike_solve_batch(const spike_handle *hs, double *const *F, const int *nrhs, int count, char trans,
                                 void *stream, void *workspace, int64_t ws_bytes) {
  return solve_batch_impl(hs, F, nrhs, count, trans, (cudaStream_t)stream, (char *)workspace, ws_bytes, nullptr);
}

extern "C" int spike_solve(spike_handle h, double *F, int nrhs, char trans) {
  if (!valid(h)) return SPIKE_EHANDLE;
  return spike_solve_ex(h, F, h->pl.n, nrhs, trans);
}

extern "C" int spike_set_stream(spike_handle h, void *stream) {
  if (!valid(h)) return SPIKE_EHANDLE;
  h->stream = (cudaStream_t)stream;
  return 0;
}

extern "C" int spike_get_info(spike_handle h, spike_info *out) {
  if (!valid(h)) return SPIKE_EHANDLE;
  if (!out) return -2;
  fill_info(h->pl, out);
  out->boosts = h->boosts;
  out->zero_pivot_col = h->zero_col;
  out->device_bytes = (int64_t)(h->mem_bytes + h->scr_bytes + h->dargs_bytes);
  out->mixed = h->f32;
  out->refine_steps = h->last_iters;
  out->refine_berr = h->last_berr;
  out->graph_captures = h->graph_captures;
  out->graph_replays = h->graph_replays;
  out->numerics = h->nan_flag;
  return 0;
}

extern "C" int spike_get_tips(spike_handle h, int level, double *host_dst) {
  if (!valid(h)) return SPIKE_EHANDLE;
  if (level < 0 || level >= std::max(h->NL, 1)) return -2;
  if (!host_dst) return -3;
  const int64_t kk = (int64_t)h->k * h->k;
  // device layout [V/W][leaf][top/bot]; host layout [leaf][Vt, Vb, Wt, Wb]
  std::vector<double> tmp((size_t)2 * h->nleaves * 2 * kk);
  SP_CUDA(cudaMemcpyAsync(tmp.data(), TIP(h, level, 0, 0, 0), sizeof(double) * tmp.size(), cudaMemcpyDeviceToHost,
                          h->stream));
  SP_CUDA(cudaStreamSynchronize(h->stream));
  for (int i = 0; i < h->nleaves; ++i)
    for (int sp = 0; sp < 2; ++sp)
      for (int t = 0; t < 2; ++t)
        memcpy(host_dst + ((int64_t)i * 4 + sp * 2 + t) * kk, tmp.data() + (((int64_t)sp * h->nleaves + i) * 2 + t) * kk,
               sizeof(double) * kk);
  return 0;
}

extern "C" int spike_backward_error(const double *band, int64_t ldab, int64_t n, int kl, int ku, const double *X,
                                    const double *F, int nrhs, char trans, void *stream, double *berr) {
  if (!band) return -1;
  if (ldab < (int64_t)kl + ku + 1) return -2;
  if (n < 1) return -3;
  if (kl < 0) return -4;
  if (ku < 0) return -5;
  if (!X) return -6;
  if (!F) return -7;
  if (nrhs < 1) return -8;
  if (trans != 'N' && trans != 'n' && trans != 'T' && trans != 't') return -9;
  if (!berr) return -11;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long *scr = nullptr;
  const size_t bytes = sizeof(unsigned long long) * (1 + 2 * (size_t)nrhs);
  SP_CUDA(dev_alloc((void **)&scr, bytes, s));
  SP_CUDA(cudaMemsetAsync(scr, 0, bytes, s));
  const int e = launch_berr(band, ldab, n, kl, ku, X, F, nrhs, (trans == 'T' || trans == 't') ? 1 : 0, scr, s);
  if (e) {
    cudaFreeAsync(scr, s);
    g_cuda_err = std::string("berr kernel: ") + cudaGetErrorString((cudaError_t)e);
    return SPIKE_ECUDA;
  }
  std::vector<unsigned long long> h(1 + 2 * (size_t)nrhs);
  SP_CUDA(cudaMemcpyAsync(h.data(), scr, bytes, cudaMemcpyDeviceToHost, s));
  SP_CUDA(cudaFreeAsync(scr, s));
  SP_CUDA(cudaStreamSynchronize(s));
  auto as_d = [](unsigned long long b) {
    double d;
    memcpy(&d, &b, sizeof(d));
    return d;
  };
  const double an = as_d(h[0]);
  for (int c = 0; c < nrhs; ++c) {
    const double r = as_d(h[1 + 2 * c]), x = as_d(h[2 + 2 * c]);
    berr[c] = (an > 0 && x > 0) ? r / (an * x) : (r == 0 ? 0.0 : INFINITY);
  }
  return 0;
}

extern "C" int spike_residual(spike_handle h, const double *X, const double *F, double *R, int nrhs, char trans,
                              double *berr) {
  if (!valid(h)) return SPIKE_EHANDLE;
  if (!X) return -2;
  if (!F) return -3;
  if (!R) return -4;
  if (nrhs < 1) return -5;
  const int tr = (trans == 'N' || trans == 'n') ? 0 : ((trans == 'T' || trans == 't') ? 1 : -1);
  if (tr < 0) return -6;
  if (!h->sfrag[0]) return SPIKE_ENOTSUP;
  if (!is_device_ptr(X) || !is_device_ptr(F) || !is_device_ptr(R)) return SPIKE_ENOTSUP;
  spike_ctx *c = h;
  const int64_t n = c->pl.n;
  cudaStream_t s = c->stream;
  const size_t xb = split_x_bytes(n, c->pl.kl, c->pl.ku, nrhs);
  const size_t nb = sizeof(unsigned long long) * (1 + 2 * (size_t)nrhs);
  char *scr = nullptr;
  SP_CUDA(dev_alloc((void **)&scr, xb + ((nb + 255) & ~size_t(255)), s));
  unsigned long long *nrm = (unsigned long long *)(scr + xb);
  int e = (int)cudaMemsetAsync(scr, 0x40, xb, s);
  if (!e) e = launch_resid_split(c->sfrag[tr], c->srexp[tr], c->snorm + tr, n, c->pl.kl, c->pl.ku, tr, X, F, R, nrhs,
                                 scr, nrm, s);
  std::vector<unsigned long long> hn(1 + 2 * (size_t)nrhs);
  if (!e) e = (int)cudaMemcpyAsync(hn.data(), nrm, nb, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(scr, s);
  if (!e) e = (int)cudaStreamSynchronize(s);
  if (e) {
    g_cuda_err = std::string("residual: ") + cudaGetErrorString((cudaError_t)e);
    return SPIKE_ECUDA;
  }
  if (berr) {
    auto as_d = [](unsigned long long b) {
      double d;
      memcpy(&d, &b, sizeof(d));
      return d;
    };
    const double an = as_d(hn[0]);
    for (int col = 0; col < nrhs; ++col) {
      const double r = as_d(hn[1 + 2 * col]), x = as_d(hn[2 + 2 * col]);
      berr[col] = (an > 0 && x > 0) ? r / (an * x) : (r == 0 ? 0.0 : INFINITY);
    }
  }
  return 0;
}

extern "C" int spike_get_timings(spike_handle h, double *ms, int count) {
  if (!valid(h)) return SPIKE_EHANDLE;
  if (!ms || count < 0) return -2;
  double t[SPIKE_T_COUNT];
  for (double &v : t) v = -1.0;
  if (h->timing) {
    SP_CUDA(cudaStreamSynchronize(h->stream));
    auto el = [](cudaEvent_t a, cudaEvent_t b) {
      float f = -1.0f;
      if (cudaEventElapsedTime(&f, a, b) != cudaSuccess) {
        cudaGetLastError();
        return -1.0;
      }
      return (double)f;
    };
    if (h->fdone) {
      t[SPIKE_T_FACTOR] = el(h->fev[0], h->fev[4]);
      t[SPIKE_T_SETUP] = el(h->fev[0], h->fev[1]);
      t[SPIKE_T_BLOCK_LU] = el(h->fev[1], h->fev[2]);
      t[SPIKE_T_SPIKES] = el(h->fev[2], h->fev[3]);
      t[SPIKE_T_REDUCED] = el(h->fev[3], h->fev[4]);
    }
    if (h->ndone) {
      t[SPIKE_T_SOLVE_N] = el(h->nev[0], h->nev[3]);
      t[SPIKE_T_SOLVE_N_D] = el(h->nev[0], h->nev[1]);
      t[SPIKE_T_SOLVE_N_RED] = el(h->nev[1], h->nev[2]);
      t[SPIKE_T_SOLVE_N_RET] = el(h->nev[2], h->nev[3]);
    }
    if (h->tdone) {
      t[SPIKE_T_SOLVE_T] = el(h->tev[0], h->tev[3]);
      t[SPIKE_T_SOLVE_T_S] = el(h->tev[0], h->tev[1]);
      t[SPIKE_T_SOLVE_T_RED] = el(h->tev[1], h->tev[2]);
      t[SPIKE_T_SOLVE_T_D] = el(h->tev[2], h->tev[3]);
    }
  }
  for (int i = 0; i < count; ++i) ms[i] = (i < SPIKE_T_COUNT) ? t[i] : -1.0;
  return 0;
}

extern "C" int64_t spike_kernel_launches(void) { return (int64_t)g_launches.load(); }

extern "C" void spike_free(spike_handle h) {
  if (!valid(h)) return;
  cudaStream_t s = h->stream;
  cudaStreamSynchronize(s);
  for (auto &g : h->gcache) drop_graph(g, s);
  h->gcache.clear();
  if (h->mem) cudaFreeAsync(h->mem, s);
  if (h->sh_fscr) cudaFreeAsync(h->sh_fscr, s);
  if (h->scr) cudaFreeAsync(h->scr, s);
  if (h->dargs) cudaFreeAsync(h->dargs, s);
  cudaStreamSynchronize(s);
  if (h->timing) {
    for (auto &e : h->fev) cudaEventDestroy(e);
    for (auto &e : h->nev) cudaEventDestroy(e);
    for (auto &e : h->tev) cudaEventDestroy(e);
  }
  h->magic = 0;
  delete h;
}

extern "C" const char *spike_strerror(int code) {
  if (code == 0) return "success";
  if (code > 0) return "zero pivot column: the matrix is singular";
  switch (code) {
    case SPIKE_ENOMEM: return "device or host allocation failed";
    case SPIKE_ECUDA: return "CUDA error (see spike_last_cuda_error)";
    case SPIKE_EHANDLE: return "invalid handle";
    case SPIKE_ENOTSUP: return "unsupported argument combination";
    case SPIKE_ENOGPU: return "no CUDA device available";
    case SPIKE_ELIMIT: return "size above the fixed limit of an entry point that allocates nothing";
    case SPIKE_ETIMEOUT: return "timeout (reserved: not returned by this library)";
    default: return "invalid argument";
  }
}

extern "C" const char *spike_last_cuda_error(void) { return g_cuda_err.c_str(); }
