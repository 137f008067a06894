/*
 * spike_serve.h -- serving engine of libspike.so: many banded systems kept factored
 * on one GPU, answering a stream of solve requests.
 *
 * The paper factors a matrix once and reuses the factorization for any number of
 * right-hand sides, with N and T alike (Sec. 4: the transpose solve needs no new
 * factorization).  A server holds a catalogue of matrices and keeps factorizations
 * resident in device memory under a byte budget, factoring a matrix on its first
 * request and evicting the least recently used factorizations when the budget is
 * full.  Requests for the same matrix, trans and precision that are waiting at the
 * same time are merged into one multi-column solve (continuous batching: whenever a
 * worker becomes free it takes the oldest waiting request whose matrix is not being
 * solved by another worker, plus every other waiting request with the same key, up
 * to max_batch_rhs columns).  With batch_systems > 1, FP64 requests of up to that many
 * matrices whose factorizations are resident are solved together with spike_solve_batch
 * (every stage of all of them in shared launches); this pays for many small systems, but
 * it keeps all those factorizations busy (not evictable) until the slowest finishes.
 * Each worker is one host thread driving one CUDA stream, so solves run concurrently.
 *
 * A request's result does not depend on what it was batched with: the solve kernels
 * give every right-hand side the same bits whatever the batch width or position
 * (and mixed-precision refinement stops per column), so a request served in a busy
 * mix returns exactly what it returns alone.
 *
 * Eviction: least recently used first by default; SPIKE_SERVE_EVICT_COST weighs each
 * factorization by how often it is used, how long it took to build and how many bytes it
 * holds (spike_server_config.evict_policy).
 *
 * Memory accounting: the budget covers resident factorizations (spike_factor_bytes'
 * resident figure, then the handle's actual device_bytes), the factorization scratch
 * while a factorization runs, and every worker's solve workspace and batch buffer.
 * Catalogue bands are the caller's memory and are not counted; mixed-precision
 * factorizations of device-resident bands read them for their FP64 residuals
 * (SPIKE_FLAG_BORROW_BAND) instead of keeping copies.
 *
 * Threading: all entry points may be called from any host thread.
 */
#ifndef SPIKE_SERVE_H_
#define SPIKE_SERVE_H_

#include <stdint.h>

#include "spike.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spike_server_s *spike_server;

/* Scheduler-only mode: no GPU is touched.  "Factorizations" hold their estimated
 * bytes, and a "solve" copies F to X (host memory) after sleeping the configured
 * times.  Exercises admission, eviction, batching and latency accounting. */
#define SPIKE_SERVE_DRYRUN 1
/* CUDA graphs per shape bucket: FP64 factorizations are made with SPIKE_FLAG_GRAPHS, and a
 * single-matrix FP64 solve of c merged columns runs as a solve of the next power of two
 * columns (the extra ones zero; results do not depend on them), on the worker's fixed
 * right-hand-side and workspace buffers, so each (matrix, trans, bucket) is captured once
 * and replayed afterwards. */
#define SPIKE_SERVE_GRAPHS 2
/* Tuned worker counts (with p = 0): the first factorization of each size class (floor(log2 n),
 * k) times factor + solve of nrhs_hint columns for a few worker counts around the default
 * rule (spike_tune, on that matrix's device band) and every later factorization of the class
 * uses the fastest.  The tuning runs on the worker that meets the class first and allocates
 * its own n x nrhs_hint right-hand sides outside the budget. */
#define SPIKE_SERVE_TUNED 4
/* Mixed-precision factorizations form their refinement residuals with FP64 FMAs
 * (SPIKE_FLAG_FP64_RESIDUAL): no digit planes of op(A), so a mixed handle takes about
 * 24 (kl + ku) bytes per row instead of about 56 (kl + ku), and more of them stay resident
 * under the budget; each residual then runs on the FP64 pipe. */
#define SPIKE_SERVE_FP64_RESIDUAL 8

typedef struct {
  int64_t budget_bytes;    /* device bytes for factorizations, their scratch and the workspaces (> 0) */
  int32_t streams;         /* workers (one host thread + one CUDA stream each), >= 1 */
  int32_t max_batch_rhs;   /* most right-hand sides merged into one solve, >= 1 */
  int32_t p;               /* worker count t of each factorization; 0: min(max(4, 2 SMs / streams), max(1, n / (16k))) */
  int32_t nrhs_hint;       /* expected columns per solve, for partition sizing (0: 16) */
  double K;                /* balance constant (<= 0: library default) */
  int32_t flags;           /* SPIKE_SERVE_* */
  int32_t dryrun_factor_us;  /* SPIKE_SERVE_DRYRUN: simulated factorization time */
  int32_t dryrun_solve_us;   /* SPIKE_SERVE_DRYRUN: simulated time per solve */
  int32_t batch_systems;     /* most matrices whose FP64 requests share one solve (0 or 1: one matrix) */
  int32_t evict_policy;      /* SPIKE_SERVE_EVICT_*: which idle factorization leaves first */
  int32_t reserved[5];
} spike_server_config;

/* Eviction policies.  LRU: the least recently used idle factorization.  COST: greedy-dual
 * size-frequency -- every resident factorization carries the priority
 *   L + (solves served since it was factored) x (its measured factorization time) / (its bytes),
 * the idle one with the lowest priority leaves first and L rises to its priority, so
 * factorizations that are used often, slow to rebuild or small stay resident, and L ages
 * out the ones that stopped being used. */
#define SPIKE_SERVE_EVICT_LRU 0
#define SPIKE_SERVE_EVICT_COST 1

typedef struct {
  int64_t submitted, completed, failed;
  int64_t batches;          /* solves run (each a merged batch of requests) */
  int64_t rhs;              /* right-hand sides solved */
  int64_t factorizations;   /* factorizations run (first use or after eviction) */
  int64_t evictions;
  int64_t admission_waits;  /* times a worker waited for budget held by running work */
  int64_t used_bytes;       /* device bytes currently counted against the budget */
  int64_t peak_bytes;       /* maximum of used_bytes */
  int32_t resident;         /* factorizations currently resident */
  int32_t max_batch;        /* most requests merged into one solve */
  int64_t multi_solves;     /* solves that covered more than one matrix (spike_solve_batch) */
  int32_t max_systems;      /* most matrices in one solve */
  int32_t tuned_classes;    /* SPIKE_SERVE_TUNED: size classes tuned so far */
  double p50_ms, p99_ms, max_ms, mean_ms;  /* latency: submit -> result in X */
  double span_s;            /* first submit -> last completion */
  double solves_per_s;      /* completed requests / span_s */
  double rhs_per_s;         /* right-hand sides / span_s */
  int64_t graph_replays;    /* SPIKE_SERVE_GRAPHS: solves replayed from captured graphs (resident handles) */
} spike_server_stats;

/* Create a server on the current CUDA device (dry-run: no device).  Returns 0, -1 for
 * an invalid config, SPIKE_ENOGPU, SPIKE_ECUDA. */
int spike_server_create(const spike_server_config *cfg, spike_server *out);

/* Register matrix `id` (any int64 not yet used): band in the layout of spike.h, host
 * or device memory, owned by the caller and left unchanged until
 * spike_server_destroy.  pivot: 0 or 1 as in spike_factor.  Returns 0 or -i. */
int spike_server_add_matrix(spike_server s, int64_t id, const double *band, int64_t ldab, int64_t n, int kl, int ku,
                            int pivot);

/* Queue a solve of op(A_id) X = F: F and X are n x nrhs, leading dimension n, host
 * (pinned is fastest) or device memory, owned by the caller until the request
 * completes; F is only read, X only written (they may be the same buffer).
 * trans 'N' or 'T'; precision 0 = FP64, 1 = mixed (FP32 factorization with FP64
 * refinement, SPIKE_FLAG_MIXED; not with pivot = 1).  Returns the request id (>= 0)
 * or -i / SPIKE_ENOTSUP.  Never blocks on GPU work. */
int64_t spike_server_submit(spike_server s, int64_t matrix_id, const double *F, double *X, int nrhs, char trans,
                            int precision);

/* Block until request `req` has completed.  Returns its status (0, or the error code of
 * the factorization or solve that served it); *latency_ms (may be NULL) receives
 * submit-to-completion time.  -2 for an unknown request id. */
int spike_server_wait(spike_server s, int64_t req, double *latency_ms);

/* Non-blocking: 0 and *latency_ms when request `req` has completed, 1 while it has not,
 * -2 for an unknown id. */
int spike_server_request_latency(spike_server s, int64_t req, double *latency_ms);

/* Block until every submitted request has completed. */
int spike_server_drain(spike_server s);

/* Counters and latency percentiles over the requests completed so far. */
int spike_server_stats_get(spike_server s, spike_server_stats *out);

/* Latencies (ms) of completed requests in completion order: copies min(cap, completed)
 * values, *count receives the number of completed requests. */
int spike_server_latencies(spike_server s, double *ms, int64_t cap, int64_t *count);

/* Text of the error of the last failed request (its return code and, for SPIKE_ECUDA,
 * the CUDA error seen by the worker thread); "" when none failed.  The pointer stays
 * valid until the calling thread calls this function again. */
const char *spike_server_last_error(spike_server s);

/* Finish queued requests, stop the workers and free every factorization and buffer. */
void spike_server_destroy(spike_server s);

#ifdef __cplusplus
}
#endif

#endif /* SPIKE_SERVE_H_ */
