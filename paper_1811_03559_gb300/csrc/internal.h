// Internal declarations shared by the host orchestration (api.cu, plan.cpp) and
// the device kernels (leaf.cu, dense.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/spike.h"

namespace spk {

constexpr int NB = 32;        // rows per block step in the factor and sweep kernels
constexpr int NTHREADS = 256; // threads per CTA of the leaf kernels
constexpr int CW = 256;       // RHS columns per sweep pass

// ------------------------------------------------------------------ planning

// One factored diagonal block ("leaf"): a whole partition, or one half of a
// partition run as a SPIKE 2x2 pair (Sec. 3.1/3.2).
struct Leaf {
  int64_t start, len;  // global rows [start, start+len)
  int rev;             // 1: UL factorization, done as LU of the reversed block Q A_i Q (Sec. 5.2)
  int has_prev, has_next;
  int part;            // partition index 0..P-1
  int half;            // 0 single, 1 top half of a 2x2 pair, 2 bottom half
};

// One pairwise merge of the recursive reduced system (Sec. 2.2, Eqs. RED_SYS_RECB/RED_SYS_W):
// left group = leaves [a, b), right group = leaves [b, c).
struct Merge {
  int a, b, c;
  int hasV;  // the merged group has a V spike (it does not contain the last leaf)
  int hasW;  // the merged group has a W spike (it does not contain the first leaf)
};

struct Plan {
  int64_t n = 0;
  int kl = 0, ku = 0, k = 0;
  int t_req = 0, t_eff = 0, m = 0, P = 0, r = 0, nleaves = 0;
  int pivot = 0;
  double K = 2.0, R12 = 0, R13 = 0;
  int64_t n1 = 0, n2 = 0, n3 = 0;
  std::vector<Leaf> leaves;
  std::vector<std::vector<Merge>> levels;  // merge levels, applied in order
};

// Returns 0 or -(argument index) on invalid input.  r13 > 0 overrides the partition ratio.
int make_plan(int64_t n, int kl, int ku, int t, double K, int nrhs_hint, int flags, double r13, Plan &out);

// Partition-range sharding: leaf_first (nranks + 1 entries) and the number of merge levels
// that stay inside one rank.  0, or -1 for an invalid rank count (see plan.cpp).
int shard_ranges(const Plan &pl, int nranks, std::vector<int> &leaf_first, int &local_levels);

// ------------------------------------------------------- device descriptors

// Leaf geometry as the kernels see it (local frame = reversed for UL leaves).
struct LeafDev {
  int64_t start, len;
  int rev;
  int top_nbr;  // the block has a neighbour coupled through its local top rows
  int bot_nbr;  // ... through its local bottom rows
  int pad;
};

// Triangular sweep kinds over the per-leaf LU band (local frame):
//   LN: unit lower L, forward         UN: upper U, backward
//   UT: U^T (lower), forward          LT: L^T (unit upper), backward
enum SweepKind { LN = 0, UN = 1, UT = 2, LT = 3 };

// One leaf's sweep: rows [r0, r1) of X = T^{-1} G, rows of X outside [r0, r1) taken as zero.
// G(r,c) = ga[r*ga_rs + c*ga_cs] + gb_scale * gb[r*gb_rs + c*gb_cs]  (gb may be null)
// X(r,c) = x[r*x_rs + c*x_cs]  (X may alias ga; it is also the source of the window rows)
struct SweepDesc {
  const double *fb;    // leaf factor band, local column 0
  const double *dinv;  // leaf diagonal reciprocals, local row 0
  const int *ipiv;     // leaf pivots (pivoting mode, local indices), local row 0
  int64_t nl;
  int r0, r1, ncols;   // ncols == 0: empty slot
  int kind;            // SweepKind
  int kw;              // off-diagonal width of the triangle (k, or 2k for U in pivoting mode)
  int fixed_split;     // 1: batch-invariant summation order of the window products
  int ldf, dofs;       // the leaf's factor storage: column stride and diagonal offset (leaf.cu)
  const double *ga;
  int64_t ga_rs, ga_cs;
  const double *gb;
  int64_t gb_rs, gb_cs;
  double gb_scale;
  double *x;
  int64_t x_rs, x_cs;
};

// Batched FP64 GEMM on strided operands: C = beta*C0 + alpha*A*B, with
// A(i,k) = A[i*a_rs + k*a_cs] (M x K), B(k,j) = B[k*b_rs + j*b_cs] (K x N),
// C(i,j) = C[i*c_rs + j*c_cs]; C0 likewise (not read when beta == 0).  Negative
// strides express reversed (Q) and transposed views.  K = 0 gives a scaled copy.
// `types` marks operands stored in FP32 (bit 1 A, 2 B, 4 C0, 8 C); arithmetic is FP64.
struct GemmDesc {
  const double *A, *B, *C0;
  double *C;
  int64_t a_rs, a_cs, b_rs, b_cs, c0_rs, c0_cs, c_rs, c_cs;
  int M, N, K, tiles_n;
  double alpha, beta;
  int tile0, types;
};
enum GemmTypes { G_A32 = 1, G_B32 = 2, G_C032 = 4, G_C32 = 8 };

// Batched dense LU with partial pivoting (first index of the largest |entry|).
struct LuDesc {
  double *a;   // row-major n x n, lda
  int *ipiv;   // n, 0-based row swapped with row j at step j
  int n, lda;
  int active;  // 0: skip
  int pad;
  unsigned long long *status;  // the matrix's system status words (null: the launch's)
};

// Batched solve with an LU of LuDesc: B <- alpha * op(M)^{-1} B (B row-major n x ncols).
struct TrsDesc {
  const double *lu;
  const int *ipiv;
  double *b;
  int64_t ldb;
  int n, lda, ncols, trans;
  double alpha;
  int tile0, pad;
};

// Fixed-order sum of `count` equally strided blocks: out[e] = sum_i in[i*stride + e].
struct SumDesc {
  const double *in;
  double *out;
  int64_t stride, elems;
  int count, pad;
};

// ------------------------------------------------------------ launchers
// Each returns cudaError_t as int (0 = success) and counts its kernel launches.
void count_launch(int n = 1);
// Stream-ordered allocation from the library's pool on the current device.  The pool keeps
// freed blocks (release threshold = max), so a factorization or solve that follows another
// reuses its memory instead of remapping it; spike_release_cached returns it.  Free with
// cudaFreeAsync.
cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t s);
// Raise a kernel's dynamic shared-memory limit to at least `bytes`, never lowering it.
// The limit is a process-wide attribute of the function: lowering it while another host
// thread launches the same kernel with a larger request would make that launch fail.
int smem_at_least(const void *func, size_t bytes);
// f32 != 0: the leaf storage (factors, spike columns, sweep operands) is FP32 (mixed-precision handles).
int launch_repack(const double *band, int64_t ldab, int kl, int ku, int64_t n, int k, int ldf, int dofs,
                  const LeafDev *leaves, int nleaves, void *fb, unsigned long long *amax_bits, void *stream,
                  int64_t max_leaf_len, int f32);
int launch_couplings(const double *band, int64_t ldab, int kl, int ku, int64_t n, int k, const LeafDev *leaves,
                     int nleaves, double *couple, void *stream);
int launch_zinit(const LeafDev *leaves, int nleaves, int k, const double *couple, void *zbuf,
                 const int64_t *zoff, int f32, void *stream);
// Block LU of every leaf followed, in the same CTA, by the leaf's spike sweeps
// (sweeps[2*leaf], sweeps[2*leaf+1]; empty slots have ncols == 0).
int launch_factor_nopiv(const LeafDev *leaves, int nleaves, int k, int ldf, void *fb, void *dinv, void *zbuf,
                        const int64_t *zoff, const unsigned long long *amax_bits, double boost_eps,
                        unsigned long long *status, const SweepDesc *sweeps, void *stream, int f32);
// sweeps: three per block (pivoted L sweep of the top spike, of the bottom spike, U sweep of both)
int launch_factor_piv(const LeafDev *leaves, int nleaves, int k, int ldf, double *fb, double *dinv, int *ipiv,
                      unsigned long long *status, const SweepDesc *sweeps, void *stream);
// One block of one system for the multi-system factorization (FP64, no pivoting): its geometry,
// the system's bandwidth and storage (ldf, factor and reciprocal bases, the block's Z columns),
// the system's max|a_ij| and status words, and the two spike sweeps that follow its LU.
struct FactorTask {
  LeafDev leaf;
  int k, ldf;
  void *fb_all, *dinv_all, *Z;
  const unsigned long long *amax_bits;
  unsigned long long *status;
  SweepDesc sw[2];
};
// Persistent CTAs over `ntasks` tasks from a zeroed counter (tasks listed largest first).
int launch_factor_tasks(const FactorTask *tasks, int ntasks, int maxk, unsigned *queue, void *stream);
// Runs per_cta consecutive descriptors per task (a leaf's sweep sequence), ncta tasks: one
// CTA per task, or, with queue (a zeroed device counter), `grid` persistent CTAs taking
// tasks in order.
int launch_sweeps(const SweepDesc *descs, int ncta, int per_cta, int ldf, int dofs, void *stream, int f32 = 0,
                  unsigned int *queue = nullptr, int grid = 0);
int launch_piv_sweep(int kind, const SweepDesc *descs, int ndesc, int k, int ldf, int dofs, void *stream);
int launch_tips0(const LeafDev *leaves, int nleaves, int k, const void *zbuf, const int64_t *zoff, double *spk,
                 void *stream, int f32);
// tile_size: 64, 32 or 16 (square tiles), or -1 / -4 / -8 (256 rows x that many columns);
// GemmDesc.tiles_n / tile0 computed for that shape
int launch_gemm(const GemmDesc *d, int ndesc, int total_tiles, int tile_size, void *stream);
int launch_getrf(const LuDesc *d, int ndesc, int maxn, unsigned long long *status, void *stream);
// cols: right-hand-side columns per CTA, 16 or 4 (TrsDesc.tile0 computed for that width)
int launch_getrs(const TrsDesc *d, int ndesc, int total_tiles, int maxn, int cols, void *stream);
// SMs of the current device (cached after the first call)
int device_sms();
int launch_noswap_flags(const double *const *w, int k, int nm, int *flags, void *stream);
int launch_assemble_M(const double *const *v, const double *const *w, int k, int nm, const int *flags, double *mbuf,
                      int64_t mstride, void *stream);
int launch_axpy(double *y, const double *x, double alpha, int64_t count, void *stream);
int launch_transpose(const double *in, double *out, int64_t rows, int cols, int64_t ld, int to_row_major,
                     void *stream);
// Column-major FP64 (rows x cols, ld) -> row-major FP32 work array.
int launch_to_work32(const double *in, int64_t ld, float *out, int64_t rows, int cols, void *stream);
// Column-major FP64 x (ld) += row-major FP32 correction d.
int launch_add_work32(double *x, int64_t ld, const float *d, int64_t rows, int cols, const int *active, void *stream);
// Residual for iterative refinement: R = F - op(A) X (all column-major FP64, ld = n) and, as bit
// patterns of non-negative doubles, norms[1+2c] = ||R_c||_inf, norms[2+2c] = ||X_c||_inf, norms[0] = ||op(A)||_inf.
int launch_residual(const double *band, int64_t ldab, int64_t n, int kl, int ku, const double *X, const double *F,
                    double *R, int nrhs, int trans, unsigned long long *norms, void *stream);
int launch_sum_blocks(const SumDesc *d, int ndesc, int64_t max_elems, void *stream);
// Backward-error reduction: scratch receives, as bit patterns of non-negative doubles,
// [0] ||op(A)||_inf, [1+2c] ||op(A)x_c - f_c||_inf, [2+2c] ||x_c||_inf.
int launch_berr(const double *band, int64_t ldab, int64_t n, int kl, int ku, const double *X, const double *F,
                int nrhs, int trans, unsigned long long *scratch, void *stream);

// FP64-accurate residual on the tensor cores (resid_split.cu): op(A) split once per
// factorization into int8 digit fragments (split_band_bytes per orientation, n int32 row
// exponents, one norm word), X split per call into split_x_bytes of scratch (zeroed by the
// caller before its first use: the zero rows around each column are never written).
bool split_supported(int kl, int ku);
size_t split_band_bytes(int64_t n, int kl, int ku);
size_t split_x_bytes(int64_t n, int kl, int ku, int nrhs);
int launch_split_band(const double *band, int64_t ldab, int64_t n, int kl, int ku, int trans, int *rexp,
                      unsigned long long *norm_bits, void *frag, void *stream);
// R = F - op(A) X; norms as launch_residual (all words written by the call)
int launch_resid_split(const void *frag, const int *rexp, const unsigned long long *anorm_bits, int64_t n, int kl,
                       int ku, int trans, const double *X, const double *F, double *R, int nrhs, void *xdig,
                       unsigned long long *norms, void *stream);

// spk tip storage index: level lv, spike s (0 = V, 1 = W), leaf i, tip t (0 = top, 1 = bottom)
inline int64_t tip_index(int lv, int s, int i, int t, int nleaves, int k) {
  return ((((int64_t)lv * 2 + s) * nleaves + i) * 2 + t) * (int64_t)k * k;
}

}  // namespace spk
