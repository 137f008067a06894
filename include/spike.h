/*
 * spike.h -- C ABI of libspike.so, a GB300-native recursive SPIKE banded solver.
 *
 * Problem (Sec. 2.1): find X in  A X = F  or  A^T X = F  (Sec. 4), where A is an
 * n x n band matrix with kl sub- and ku super-diagonals and F, X are n x nrhs.
 * A is partitioned into p diagonal blocks A_i with couplings B_i / C_i
 * (Sec. 2.1, Eq. "partitioning"), factored as A = D S (Eq. "spikes"), the
 * reduced system is solved recursively (Sec. 2.2) for any worker count p
 * (Sec. 3: 2^m partitions, r of them split in two and run as a SPIKE 2x2 pair),
 * and the factorization is reused for the transpose solve (Sec. 4).  Blocks are
 * factored without pivoting (LU, UL for the last block, with diagonal
 * boosting, Sec. 2.3) or with partial pivoting (Sec. 5.1, UL via Q A Q, Sec. 5.2).
 *
 * Storage conventions (all column-major, 0-based, FP64):
 *   band : A(i,j) at band[j*ldab + ku + i - j] for max(0,j-ku) <= i <= min(n-1,j+kl)
 *          (the LAPACK band layout; ldab >= kl+ku+1).  Other entries are ignored.
 *   F    : F(i,c) at F[c*ldf + i], ldf >= n.  Overwritten by X.
 * Pointers may be device memory or host memory (pageable or pinned); host
 * buffers are staged through device memory inside the call, except a pinned
 * (page-locked and mapped) FP64 band, which the factorization's setup kernels
 * read in place through its device address.
 *
 * Return codes: 0 on success.  -i: argument i is invalid (LAPACK info style,
 * arguments counted from 1).  SPIKE_E* (below): allocation, CUDA or internal
 * failures.  A positive value i from spike_factor in pivoting mode means the
 * pivot candidates of global column i-1 were all exactly zero (A singular);
 * the handle is still returned and spike_solve on it returns the same i.
 *
 * Threading: a handle may be used by one host thread at a time.  All GPU work
 * of a handle is issued on its stream (spike_set_stream / options.stream).
 */
#ifndef SPIKE_H_
#define SPIKE_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPIKE_OK 0
#define SPIKE_ENOMEM (-1001)   /* device or host allocation failed */
#define SPIKE_ECUDA (-1002)    /* a CUDA call failed (message via spike_last_cuda_error) */
#define SPIKE_EHANDLE (-1003)  /* NULL or freed handle */
#define SPIKE_ENOTSUP (-1004)  /* unsupported combination (e.g. bandwidth above the library limit) */
#define SPIKE_ENOGPU (-1005)   /* no CUDA device available */
#define SPIKE_ELIMIT (-1006)   /* size above the fixed limit of an entry point that allocates nothing */
#define SPIKE_ETIMEOUT (-1007) /* reserved: no kernel of this library waits on another (no spin-waits),
                                  so no call returns it */

#define SPIKE_FLAG_TIMING 1
/* Size partitions for stage-synchronised execution.  The reduced system puts a
 * device-wide synchronisation between the factorization and the solves, so each
 * stage costs the maximum over blocks of that stage alone.  The paper's combined
 * balance (Eq. R13_calculation: equal factor + solve work per partition) then
 * leaves the two end blocks idle in one stage and the inner ones in the other.
 * With this flag R13 is the paper's solve-stage limit 2 (Eq. ratios) when
 * nrhs_hint > 0, and its factorization limit 1 + 1.5K (Eq. ratiof) otherwise:
 * with few end blocks the inner blocks bound the factorization either way, and
 * R13 = 2 balances the solve stages exactly. */
#define SPIKE_FLAG_STAGE_BALANCE 2
/* Mixed precision: the block factorizations, spike sweeps and solve sweeps run in
 * FP32 (the FP32 FMA pipe is ~60x the FP64 one on GB300); the spike tips and the
 * whole reduced system stay FP64; spike_solve then refines in FP64: each step
 * forms r = F - op(A) x from an FP64 copy of the band kept by the handle, solves
 * with the FP32 factorization and adds the correction, until the backward error
 * of every column is <= SPIKE_MIXED_TOL (at most SPIKE_MIXED_MAX_STEPS steps;
 * spike_get_info reports the steps and the final backward error).  Non-pivoting
 * only (SPIKE_ENOTSUP with pivot = 1). */
#define SPIKE_FLAG_MIXED 4
/* Default partition ratio R13 of pivoting factorizations (see spike_options.R13): the
 * fastest of 1.5, 2, 2.5 and the formula for factor + N + T solve on the pivoting
 * workload (n = 262,144, k = 16 and 64, nrhs = 8, p = 148) on GB300. */
#define SPIKE_PIVOT_R13 1.5
/* Batch-invariant solves: every right-hand side of a solve gets the same bits whatever
 * the number of columns solved with it and its position among them.  The window
 * products of the triangular sweeps are then summed over a fixed set of sub-ranges
 * instead of a split that depends on the column count (a few percent slower on
 * wide solves); everything else on the solve path is column-independent already, and
 * mixed-precision refinement stops per column.  Lets independent requests be merged
 * into one solve without changing any result (the serving engine sets it). */
#define SPIKE_FLAG_BATCH_INVARIANT 8
/* Mixed-precision handles of a DEVICE band: read the caller's band for the FP64
 * residuals instead of keeping a copy (saves 8 n (kl+ku+1) bytes per handle).  The
 * band must then stay valid and unchanged until spike_free.  Ignored for host bands
 * and FP64 handles. */
#define SPIKE_FLAG_BORROW_BAND 16
/* CUDA graphs for repeated solves: an FP64 solve of device buffers is run directly the
 * first time a call (nrhs, trans, F pointer, ldf, scratch) is seen, captured as a CUDA
 * graph the second time, and replayed from then on (up to 16 graphs per handle, least
 * recently used replaced).  A replay launches the whole solve at once instead of a few
 * dozen separate launches; results are those of the direct launches.  The buffers a
 * graph was captured with must not be freed while it may be replayed (F is the caller's;
 * the scratch is the handle's own or the spike_solve_ws workspace).  Not used with
 * SPIKE_FLAG_TIMING, mixed precision, host F or the legacy default stream (NULL). */
#define SPIKE_FLAG_GRAPHS 32
/* Mixed precision: form the refinement residuals with FP64 FMAs instead of the tensor-core
 * residual (see spike_residual).  By default a mixed-precision handle splits op(A) once, at
 * factorization, into integer digit planes (about 16 n (kl + ku + 35) bytes for N and T
 * together, counted by spike_factor_bytes) and forms each residual of 8 or more columns on
 * the tensor cores, to FP64 accuracy; with fewer columns (except on SPIKE_FLAG_BATCH_INVARIANT
 * handles, which use it for every column count), or kl + ku above about 540, the FP64 kernel
 * is used. */
#define SPIKE_FLAG_FP64_RESIDUAL 64
#define SPIKE_MIXED_TOL 1e-14
#define SPIKE_MIXED_MAX_STEPS 10

/* Stage indices of spike_get_timings (milliseconds between CUDA events recorded
 * on the handle's stream; the last factorization and the last N / T solve). */
#define SPIKE_T_FACTOR 0         /* whole spike_factor GPU work */
#define SPIKE_T_SETUP 1          /* band repack, couplings, spike right-hand sides */
#define SPIKE_T_BLOCK_LU 2       /* block factorization kernel; without pivoting it also runs every
                                    spike sweep of the block in the same launch */
#define SPIKE_T_SPIKES 3         /* tip extraction (and, when pivoting, the spike sweeps) */
#define SPIKE_T_REDUCED 4        /* recursive reduced-system factorization */
#define SPIKE_T_SOLVE_N 5        /* whole N solve */
#define SPIKE_T_SOLVE_N_D 6      /*   D stage (L sweep, tip sweeps) */
#define SPIKE_T_SOLVE_N_RED 7    /*   reduced system */
#define SPIKE_T_SOLVE_N_RET 8    /*   retrieval */
#define SPIKE_T_SOLVE_T 9        /* whole T solve */
#define SPIKE_T_SOLVE_T_S 10     /*   S^T stage (sweeps, modified RHS) */
#define SPIKE_T_SOLVE_T_RED 11   /*   transposed reduced system */
#define SPIKE_T_SOLVE_T_D 12     /*   D^T stage */
#define SPIKE_T_COUNT 13

/* Largest half-bandwidth max(kl, ku) the kernels accept. */
#define SPIKE_MAX_K 512

typedef struct spike_ctx *spike_handle;

/* Options for spike_factor_ex / spike_plan.  Zero-initialise for defaults. */
typedef struct {
  /* Machine constant K = K2/K1 of the load-balancing model (Sec. 3.3, Eq.
   * R13_calculation): solve cost per row and RHS column over factor cost per row
   * and band column.  <= 0 selects 2.0, the value for kernels whose factor and
   * sweep steps run at the same FP64 rate (one k x k update per factored column
   * versus one k-wide update per column of a two-sweep solve). */
  double K;
  /* Expected nrhs used to size partitions (n_rhs/k in Eqs. R13/R12_calculation).
   * 0 selects the factorization-dominated limit n_rhs/k -> 0 (Eq. ratiof). */
  int32_t nrhs_hint;
  /* Bit flags: SPIKE_FLAG_TIMING records CUDA events around the pipeline stages
   * (read them with spike_get_timings). */
  int32_t flags;
  /* cudaStream_t for all work of the handle; NULL = the legacy default stream. */
  void *stream;
  /* > 0: use this partition ratio R13 = n1/n3 (R12 = R13/2) instead of the formula or
   * SPIKE_FLAG_STAGE_BALANCE -- for ratio sweeps and tuned configurations (Sec. 3.3).
   * Pivoting factorizations (pivot = 1) without this or SPIKE_FLAG_STAGE_BALANCE use
   * SPIKE_PIVOT_R13: the formula models the non-pivoting costs, whereas the pivoted end
   * blocks' GEPP costs several times a middle block's per row and the pivoted L sweeps of
   * a solve are a larger share.  spike_plan has no pivot argument: pass
   * R13 = SPIKE_PIVOT_R13 to it for the plan of a pivoting factorization. */
  double R13;
  /* SPIKE_FLAG_MIXED: stop refining a column once its FP64 backward error is <= this
   * (<= 0 selects SPIKE_MIXED_TOL). */
  double refine_tol;
  int64_t reserved[2];
} spike_options;

/* Description of a partition plan / factorization. */
typedef struct {
  int64_t n;
  int32_t kl, ku, k;        /* k = max(kl, ku): couplings are padded to k x k (Sec. 2.1) */
  int32_t p_requested;      /* worker count t asked for */
  int32_t p_effective;      /* t actually used (t = 2^(m+1)-1 runs as 2^(m+1)-2, Sec. 3.1; lowered
                               further if a block would be shorter than 2k rows) */
  int32_t m;                /* P = 2^m partitions (Sec. 3.1) */
  int32_t P;
  int32_t r;                /* partitions 2..r+1 (1-based) are split into a SPIKE 2x2 pair */
  int32_t leaves;           /* P + r blocks actually factored (one GPU CTA each) */
  int32_t levels;           /* merge levels of the reduced system (1 for the 2x2 pairs if r>0, plus m) */
  int32_t pivot;
  int64_t n1, n2, n3;       /* sizes of first/last, 2x2 and single inner partitions (Sec. 3.3) */
  double R12, R13;          /* balance ratios used (Eqs. R12/R13_calculation) */
  double K;                 /* balance constant used */
  int64_t boosts;           /* non-pivoting mode: number of boosted (near-zero) pivots (Sec. 2.3) */
  int64_t zero_pivot_col;   /* pivoting mode: 1-based global column of the first all-zero pivot column, 0 if none */
  int64_t device_bytes;     /* device memory held by the handle */
  int32_t mixed;            /* 1: SPIKE_FLAG_MIXED handle */
  int32_t refine_steps;     /* mixed: FP64 refinement steps of the last solve */
  double refine_berr;       /* mixed: max backward error over columns after the last solve */
  int64_t graph_captures;   /* SPIKE_FLAG_GRAPHS: solves captured as CUDA graphs */
  int64_t graph_replays;    /* SPIKE_FLAG_GRAPHS: solves replayed from a captured graph */
  int32_t numerics;         /* SPIKE_NUMERICS_* bits seen by the factorization (0: none).  As in
                               LAPACK, a NaN in A is not an error: the call succeeds and the results
                               carry NaN; this field says so without a pass over the output */
  int32_t reserved0;
} spike_info;

/* Bits of spike_info.numerics. */
#define SPIKE_NUMERICS_NAN_PIVOT 1         /* a block factorization met a NaN pivot (NaN or Inf in A) */
#define SPIKE_NUMERICS_SINGULAR_INTERFACE 2 /* an interface block of the reduced system (Sec. 2.2) had no
                                              nonzero pivot candidate: S is singular to working precision */

/* Compute the partition plan for (n, kl, ku, p) without touching a GPU (Sec. 3.1, 3.3).
 * leaf_offsets (may be NULL) receives leaves+1 entries: block b covers global rows
 * [leaf_offsets[b], leaf_offsets[b+1]).  leaf_flags (may be NULL) receives one int per
 * block: bit0 = factored as UL (reversed LU), bit1 = top half of a 2x2 pair,
 * bit2 = bottom half of a 2x2 pair.  Arrays must hold at least p+1 entries.
 * Returns 0 or -i for an invalid argument i. */
int spike_plan(int64_t n, int kl, int ku, int p, const spike_options *opt, spike_info *out,
               int64_t *leaf_offsets, int32_t *leaf_flags);

/* Factor A (Sec. 2.1-2.3, 3, 5).  band: device or host pointer, layout above with
 * ldab = kl+ku+1, read-only, owned by the caller, only read during the call.
 * p: worker count (>= 1).  pivot: 0 = non-pivoting LU/UL with diagonal boosting,
 * 1 = partial pivoting.  On success *out receives a new handle (free with
 * spike_free).  The call blocks until the factorization is complete. */
int spike_factor(const double *band, int64_t n, int kl, int ku, int p, int pivot, spike_handle *out);

/* As spike_factor with an explicit leading dimension ldab >= kl+ku+1 and options
 * (opt may be NULL). */
int spike_factor_ex(const double *band, int64_t ldab, int64_t n, int kl, int ku, int p, int pivot,
                    const spike_options *opt, spike_handle *out);

/* Overwrite F (n x nrhs, ldf = n) with X solving A X = F (trans 'N') or A^T X = F
 * (trans 'T'), reusing the factorization (Sec. 4).  F: device or host pointer owned
 * by the caller.  For device F the call is asynchronous on the handle's stream;
 * for host F it returns after X has been copied back. */
int spike_solve(spike_handle h, double *F, int nrhs, char trans);

/* As spike_solve with an explicit leading dimension ldf >= n. */
int spike_solve_ex(spike_handle h, double *F, int64_t ldf, int nrhs, char trans);

/* Device bytes that a factorization of (n, kl, ku, p, pivot, opt) will use, without
 * touching a GPU.  *resident: held by the handle until spike_free (block factors,
 * spike tips, reduced-system LUs and, with SPIKE_FLAG_MIXED, the FP64 band copy).
 * *transient: scratch that spike_factor allocates and frees inside the call (the
 * spike right-hand sides, plus, for FP64 handles, a staged copy of the band when
 * host_band != 0: the bound for a pageable band, as a pinned one is read in place
 * and a mixed handle copies a host band straight into its FP64 band).
 * Neither counts the handle's descriptor buffer (a few hundred KB at most) nor solve
 * scratch (see spike_solve_ws).  Returns 0, -i for an invalid argument i, or
 * SPIKE_ENOTSUP. */
int spike_factor_bytes(int64_t n, int kl, int ku, int p, int pivot, const spike_options *opt, int host_band,
                       int64_t *resident, int64_t *transient);

/* Device scratch bytes that spike_solve_ws needs for nrhs columns of the handle
 * (host_f != 0: F will be host memory and is staged in the workspace too). */
int spike_solve_workspace(spike_handle h, int nrhs, char trans, int host_f, int64_t *bytes);

/* spike_solve_ex on caller-provided device scratch: workspace (ws_bytes >= the
 * figure of spike_solve_workspace, else -7).  The handle then keeps no solve
 * scratch of its own, so many resident handles can share a few workspaces, one per
 * stream.  The workspace must not be reused until the solve's GPU work on the
 * handle's stream has completed.  Results are those of spike_solve_ex. */
int spike_solve_ws(spike_handle h, double *F, int64_t ldf, int nrhs, char trans, void *workspace, int64_t ws_bytes);

/* Solve `count` independent systems together (batching across matrices).  The same
 * stage of every system runs as one launch: all their blocks' sweeps in one grid, and
 * each merge level's reduced-system products, LU solves and sums as one batched launch
 * (levels aligned from the bottom for N, from the top for T).  Many systems of uneven
 * n, k and nrhs then fill the GPU together with a few dozen launches in all.
 *   hs[i]   FP64, non-pivoting handles (SPIKE_ENOTSUP for mixed-precision or pivoting
 *           ones); a handle may appear more than once.
 *   F[i]    device pointer, n_i x nrhs[i] with leading dimension n_i, overwritten by X_i.
 *   trans   one of 'N' / 'T' for all systems.
 *   workspace  device scratch of at least spike_solve_batch_workspace bytes (-8
 *           otherwise); it must not be reused until the work on `stream` is done.
 * Asynchronous on `stream`.  Every X_i is bitwise the result of spike_solve_ex on that
 * system alone (the merged launches keep each output's operation order).  The handles
 * must not be used by other threads during the call. */
int spike_solve_batch(const spike_handle *hs, double *const *F, const int *nrhs, int count, char trans,
                      void *stream, void *workspace, int64_t ws_bytes);

/* Factor `count` independent systems together (FP64, non-pivoting): system i is the band
 * bands[i] (device pointer, ldab[i]) of order n[i] with bandwidths kl[i], ku[i], split for
 * p[i] workers (Sec. 3).  Every system's blocks (Sec. 2.3: the LU and the spike sweeps of each
 * block) run in ONE launch, persistent CTAs taking the blocks of all systems from a work queue,
 * largest first, so many small uneven systems fill the GPU together; the reduced systems
 * (Sec. 2.2) run one merge level of every system per batched launch (levels aligned from the
 * bottom) with one device round trip per level.  out[i] receives system i's handle, exactly
 * the handle spike_factor_ex(bands[i], ldab[i], n[i], kl[i], ku[i], p[i], 0, opt) would return
 * (same factors, bit for bit).  opt (may be NULL) is shared; its stream carries all the work;
 * SPIKE_FLAG_MIXED and SPIKE_FLAG_TIMING are not supported (SPIKE_ENOTSUP), nor host bands.
 * Blocks until done.  On failure no handle is returned. */
int spike_factor_batch(const double *const *bands, const int64_t *ldab, const int64_t *n, const int *kl,
                       const int *ku, const int *p, int count, const spike_options *opt, spike_handle *out);

/* Device scratch bytes spike_solve_batch needs for these handles and column counts. */
int spike_solve_batch_workspace(const spike_handle *hs, const int *nrhs, int count, char trans, int64_t *bytes);

/* Set the cudaStream_t used by the handle (NULL = legacy default stream). */
int spike_set_stream(spike_handle h, void *stream);

/* Describe a handle (plan, boosts, zero pivot, memory). */
int spike_get_info(spike_handle h, spike_info *out);

/* Copy the k x k spike tips of merge level `level` (0 = the blocks' own spikes,
 * Eq. "spikes") to host memory: leaves x {V_t, V_b, W_t, W_b} x k x k, row-major
 * per tip.  Tips that the method never forms (V_t of the first block, W_b of the
 * last, and V / W of groups that contain the last / first block) read as zero.
 * For inspection and tests. */
int spike_get_tips(spike_handle h, int level, double *host_dst);

/* Backward error of a computed solution, on the GPU in FP64 from the ORIGINAL
 * band (device pointer, ldab >= kl+ku+1): for each column c,
 *   berr[c] = ||op(A) x_c - f_c||_inf / (||op(A)||_inf * ||x_c||_inf).
 * X, F: device pointers, n x nrhs with leading dimension n.  berr: host array of
 * nrhs doubles.  Uses the stream of `stream` (NULL = legacy default) and
 * synchronises it before returning.  Allocates a small device scratch buffer. */
int spike_backward_error(const double *band, int64_t ldab, int64_t n, int kl, int ku, const double *X,
                         const double *F, int nrhs, char trans, void *stream, double *berr);

/* R = F - op(A) X for a mixed-precision handle (SPIKE_FLAG_MIXED without
 * SPIKE_FLAG_FP64_RESIDUAL), with the kernel its iterative refinement uses (Sec. 5: the
 * residual of an approximate factorization is formed in the working precision, FP64):
 * every entry of op(A) (from the handle's FP64 band) and of X is written as a 56-bit
 * fixed-point number relative to a power of two of its row / column, split into 8 base-128
 * digits, and the digit products are accumulated exactly on the bf16 tensor cores; only the
 * two fixed-point roundings (2^-56 of the row and column scale), the final sum in FP64 and
 * f - Ax round.  X, F, R: device pointers, n x nrhs, leading dimension n (R may not alias
 * X).  berr (host, nrhs doubles, may be NULL) receives ||r_c||_inf / (||op(A)||_inf
 * ||x_c||_inf) per column.  Runs on the handle's stream and synchronises it; allocates its
 * scratch from the library's pool.  SPIKE_ENOTSUP for other handles or host pointers. */
int spike_residual(spike_handle h, const double *X, const double *F, double *R, int nrhs, char trans, double *berr);

/* Stage times of the last factorization and the last N and T solves of a handle
 * created with SPIKE_FLAG_TIMING (indices SPIKE_T_*; -1 for stages not run).
 * Synchronises the handle's stream.  ms must hold `count` doubles. */
int spike_get_timings(spike_handle h, double *ms, int count);

/* Measure the FP64 FMA throughput of the current device with a dependent-chain
 * DFMA loop on every SM (8 independent chains per thread, 2 CTAs of 512 threads
 * per SM), in TFLOP/s (2 flop per FMA).  The roofline denominator of the FP64
 * kernels.  Synchronises `stream`. */
int spike_measure_fp64_peak(void *stream, double *tflops);

/* Throughput probes of the arithmetic pipes the design choices rest on, on the current
 * device (2 CTAs of 512 threads per SM, 8 independent dependent chains per thread or warp,
 * each timed with CUDA events after a short untimed launch).  out[0..count) receives, in
 * this order (entries past 7 are left 0):
 *   0  DFMA, TFLOP/s (2 flop per FMA; the same loop as spike_measure_fp64_peak)
 *   1  FP64 mma.sync.m8n8k4 (DMMA), TFLOP/s
 *   2  FP32 FMA, TFLOP/s
 *   3  bf16 mma.sync.m16n8k16 with FP32 accumulation, TFLOP/s
 *   4  ms of the even warps running DFMA chains, odd warps idle
 *   5  ms of the odd warps running DMMA chains (the same FMA count), even warps idle
 *   6  ms of both at once in alternate warps: about max(4, 5) if DFMA and DMMA issue to
 *      separate pipes, about 4 + 5 if they share one.
 * Synchronises `stream`.  Returns 0, -2 (out NULL), -3 (count < 1), SPIKE_ENOMEM or
 * SPIKE_ECUDA. */
int spike_measure_pipes(void *stream, double *out, int count);

/* The machine constant K = K2/K1 of the load-balancing model (Sec. 3.3: solve cost per
 * row and right-hand side over factorization cost per row and band column), measured
 * as the paper prescribes: (solve time) / (factorization time) of one block with
 * nrhs = k, here the leading min(n, 65536) rows of `band` (device pointer) factored
 * as a single block (one CTA: block LU, then the two full sweeps of the solve).  The
 * run is repeated once and the second timing kept.  Synchronises `stream`. */
int spike_measure_K(const double *band, int64_t ldab, int64_t n, int kl, int ku, void *stream, double *K);

/* Result of spike_tune. */
typedef struct {
  double K_measured;    /* spike_measure_K on the same matrix */
  int32_t best_p;       /* fastest worker count among the candidates */
  int32_t best_mode;    /* 0: the paper's ratio with K_measured, 1: SPIKE_FLAG_STAGE_BALANCE, 2: explicit R13 */
  double best_R13;      /* partition ratio of the fastest configuration */
  double best_ms;       /* its factor + nsolves solves time */
  double default_ms;    /* p_candidates[0] with SPIKE_FLAG_STAGE_BALANCE */
  int32_t tried;        /* configurations timed */
  int32_t reserved;
} spike_tune_result;

/* Time factor + nsolves N solves of nrhs columns on the caller's matrix (device band,
 * non-pivoting) for every worker count in p_candidates and every sizing: the paper's
 * ratio with the measured K, stage balance, and each explicit R13 of r13_candidates
 * (nr entries, may be 0), after one untimed warm-up run.  table_ms (may be NULL)
 * receives np x (2 + nr) milliseconds, row-major.  The timings are CUDA events on
 * `stream` around the whole calls (factor's host round trips included).  Allocates
 * n x nrhs doubles of right-hand sides.  Synchronises `stream`. */
int spike_tune(const double *band, int64_t ldab, int64_t n, int kl, int ku, int nrhs, int nsolves,
               const int *p_candidates, int np, const double *r13_candidates, int nr, void *stream,
               double *table_ms, spike_tune_result *out);

/* Device memory: the library allocates stream-ordered from its own pool per device, which
 * keeps freed blocks cached (a factorization or solve that follows another reuses them
 * instead of remapping memory).  spike_release_cached synchronises every device the
 * library has used and returns the cached blocks that are not in use to the driver;
 * reserved_before / reserved_after (may be NULL) receive the pools' reserved bytes. */
int spike_release_cached(int64_t *reserved_before, int64_t *reserved_after);

/* Number of CUDA kernels this library has launched in the process so far. */
int64_t spike_kernel_launches(void);

/* Largest nrhs accepted by spike_backward_error_noalloc. */
#define SPIKE_NOALLOC_MAX_NRHS 1024

/* spike_backward_error for callers that cannot allocate memory.  (The paper has no
 * counterpart: this is a library-usage entry point.)  Some callers must not
 * allocate during the call: processes whose device memory is entirely held by
 * their own pool or caching allocator (a cudaMalloc would fail or fragment it),
 * and latency-bound loops that cannot absorb cudaFree, which synchronises the
 * whole device.  This entry point performs the same computation on the same
 * kernel as spike_backward_error and returns the same values, but calls no
 * cudaMalloc, cudaFree or other allocating routine, on the device or the host.
 * Its reduction scratch is a fixed array of (1 + 3*SPIKE_NOALLOC_MAX_NRHS)
 * 8-byte words (about 24 KB) in the library's device memory, held by every GPU
 * that loads the library until the process exits.
 *   - nrhs above SPIKE_NOALLOC_MAX_NRHS returns SPIKE_ELIMIT (nothing runs).
 *   - The first call on a device looks up that array's device address (once
 *     per device, with the device current); make that first call before any
 *     stream capture.  The address is cached for the life of the process: after
 *     cudaDeviceReset on a device, do not call this entry point on that device
 *     again in the same process.
 *   - `stream` must belong to the current device (the scratch used is the
 *     current device's copy of the array).
 *   - Every call shares the one array: calls whose GPU work overlaps (other
 *     streams, other host threads) race on it and must be serialised by the
 *     caller.  Each call clears the part it uses before using it.
 *   - On a CUDA failure it returns SPIKE_ECUDA without updating the text of
 *     spike_last_cuda_error (that text lives in a heap-allocated string).
 * Arguments, layout and synchronisation are those of spike_backward_error. */
int spike_backward_error_noalloc(const double *band, int64_t ldab, int64_t n, int kl, int ku, const double *X,
                                 const double *F, int nrhs, char trans, void *stream, double *berr);

/* ---------------------------------------------------------------------------------------
 * Partition-range sharding of one system over nranks GPUs (the SPIKE-MPI direction named in
 * Sec. 3, with the recursive reduced system of Sec. 2.2 carried across ranks).  Rank g owns
 * P / nranks consecutive partitions of the plan of (n, kl, ku, p): blocks
 * [leaf_first[g], leaf_first[g+1]) and rows [row_first[g], row_first[g+1]).  The pair level
 * and the first log2(P / nranks) power-of-two merge levels stay inside a rank; each of the
 * top log2(nranks) levels is one exchange, in which every rank contributes a fixed-size
 * buffer (the spike tips of its boundary blocks: 4 k x k in the factorization; its boundary
 * right-hand-side tips: 2 k x nrhs in the solves; one k x nrhs partial product per level in
 * the transposed solve) and receives all ranks' buffers (an all-gather, made by the caller
 * over NCCL, MPI or any transport).  Non-pivoting FP64 handles only.
 *
 * Protocol, per operation (spike_shard_factor, then any number of spike_shard_solve):
 *   while (spike_shard_pending(h, &count) == 0 && count > 0) {
 *     spike_shard_export(h, send);          // send: count doubles, device
 *     all-gather send over the ranks into recv (nranks x count doubles, rank-major, device)
 *     spike_shard_import(h, recv);
 *   }
 * Every rank runs the same number of exchanges with the same count.  A new operation may
 * start only when the previous one has no pending exchange (SPIKE_ENOTSUP otherwise).
 * ------------------------------------------------------------------------------------ */

/* The ranges of each rank (no GPU).  nranks must be a power of two between 1 and the plan's
 * partition count P (-5 otherwise).  row_first, leaf_first: nranks + 1 entries;
 * *local_levels: merge levels that stay inside one rank (the rest are exchanges). */
int spike_shard_plan(int64_t n, int kl, int ku, int p, int nranks, const spike_options *opt, int64_t *row_first,
                     int32_t *leaf_first, int32_t *local_levels);

/* Factor rank `rank`'s blocks (Sec. 2.3) and the merge levels inside them (Sec. 2.2).
 * band: device pointer to global band columns col0, col0 + 1, ... (LAPACK layout, ldab)
 * covering at least columns [max(0, r0 - k), min(n, r1 + k)) where [r0, r1) are the rank's
 * rows (spike_shard_plan) and k = max(kl, ku): the rank's rows and their couplings.  It is
 * read during the call only.  Other arguments as spike_factor_ex; the options' flags may not
 * include SPIKE_FLAG_MIXED.  -3: col0 is past the rank's first needed column; -9: a rank
 * count the plan cannot take.  The factorization is complete when no exchange is pending.
 * The diagonal boosting threshold (Sec. 2.3) is taken from the rank's own block entries. */
int spike_shard_factor(const double *band, int64_t ldab, int64_t col0, int64_t n, int kl, int ku, int p, int rank,
                       int nranks, const spike_options *opt, spike_handle *out);

/* Start a solve of A X = F (trans 'N') or A^T X = F ('T', Sec. 4) with the rank's rows of F:
 * F is a device pointer, (rows of the rank) x nrhs, leading dimension ldf; it is overwritten
 * with the rank's rows of X when the last exchange has been imported. */
int spike_shard_solve(spike_handle h, double *F, int64_t ldf, int nrhs, char trans);

/* Doubles each rank contributes to the pending exchange (0: the operation is complete). */
int spike_shard_pending(spike_handle h, int64_t *count);

/* Write this rank's contribution to the pending exchange to `send` (device, count doubles);
 * synchronises the handle's stream. */
int spike_shard_export(spike_handle h, double *send);

/* Run the pending level with the gathered contributions (recv: device, nranks x count
 * doubles, rank g's at recv + g * count; complete before the call).  Asynchronous on the
 * handle's stream, except the factorization's levels, which read a flag per merge back. */
int spike_shard_import(spike_handle h, const double *recv);

/* Release a handle and all its device memory.  NULL is ignored. */
void spike_free(spike_handle h);

/* Static description of a return code. */
const char *spike_strerror(int code);

/* Text of the last CUDA error seen by the calling thread inside the library. */
const char *spike_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SPIKE_H_ */
