// Partition tuning (Sec. 3.3): the machine constant K of the load-balancing model and a
// timed search over worker counts and partition ratios on the caller's matrix.
//
// The paper measures K = K2/K1 once per machine as (solve time) / (factorization time)
// for one block with as many right-hand sides as the bandwidth, and then sizes the
// partitions from K and n_rhs/k (Eqs. R13_calculation, R12_calculation).  Here the same
// measurement runs on a single GPU block (p = 1: one CTA, block LU then the two full
// sweeps of the solve), and spike_tune times whole factor + solve runs for the
// candidate configurations so the choice can be checked against a ratio sweep.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "spike.h"
#include "internal.h"

namespace {

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  Timer() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

// factor + nsolves N solves of F (n x nrhs zeros; the run time does not depend on the
// values), returns GPU milliseconds between events on `stream`, or a negative code.
int run_once(const double *band, int64_t ldab, int64_t n, int kl, int ku, int p, const spike_options &o, double *F,
             int nrhs, int nsolves, cudaStream_t st, double *ms) {
  Timer t;
  cudaEventRecord(t.a, st);
  spike_handle h = nullptr;
  int rc = spike_factor_ex(band, ldab, n, kl, ku, p, 0, &o, &h);
  if (rc != 0) {
    if (h) spike_free(h);
    return rc < 0 ? rc : SPIKE_ENOTSUP;
  }
  for (int s = 0; s < nsolves && rc == 0; ++s) rc = spike_solve_ex(h, F, n, nrhs, 'N');
  cudaEventRecord(t.b, st);
  if (cudaEventSynchronize(t.b) != cudaSuccess) rc = SPIKE_ECUDA;
  float f = 0.0f;
  cudaEventElapsedTime(&f, t.a, t.b);
  *ms = f;
  spike_free(h);
  return rc;
}

}  // namespace

extern "C" int spike_measure_K(const double *band, int64_t ldab, int64_t n, int kl, int ku, void *stream,
                               double *K) {
  if (!band) return -1;
  if (n < 1) return -3;
  if (!K) return -7;
  const cudaStream_t st = (cudaStream_t)stream;
  const int k = std::max(1, std::max(kl, ku));
  const int64_t n0 = std::min<int64_t>(n, 1 << 16);  // leading block: a band matrix with the same layout
  double *F = nullptr;
  const size_t fb = sizeof(double) * (size_t)n0 * k;
  if (spk::dev_alloc((void **)&F, fb, st) != cudaSuccess || cudaMemsetAsync(F, 0, fb, st) != cudaSuccess) {
    cudaGetLastError();
    if (F) cudaFreeAsync(F, st);
    return SPIKE_ENOMEM;
  }
  spike_options o;
  memset(&o, 0, sizeof(o));
  o.flags = SPIKE_FLAG_TIMING;
  o.stream = stream;
  double lu = 0.0, sv = 0.0;
  int rc = 0;
  for (int rep = 0; rep < 2 && rc == 0; ++rep) {  // the first run absorbs one-time costs
    spike_handle h = nullptr;
    rc = spike_factor_ex(band, ldab, n0, kl, ku, 1, 0, &o, &h);
    if (rc == 0) rc = spike_solve_ex(h, F, n0, k, 'N');
    double t[SPIKE_T_COUNT];
    if (rc == 0) rc = spike_get_timings(h, t, SPIKE_T_COUNT);
    if (rc == 0) {
      lu = t[SPIKE_T_BLOCK_LU];
      sv = t[SPIKE_T_SOLVE_N];
    }
    if (h) spike_free(h);
  }
  cudaFreeAsync(F, st);
  cudaStreamSynchronize(st);
  if (rc != 0) return rc;
  if (!(lu > 0.0) || !(sv > 0.0)) return SPIKE_ECUDA;
  *K = sv / lu;
  return 0;
}

extern "C" int spike_tune(const double *band, int64_t ldab, int64_t n, int kl, int ku, int nrhs, int nsolves,
                          const int *p_candidates, int np, const double *r13_candidates, int nr, void *stream,
                          double *table_ms, spike_tune_result *out) {
  if (!band) return -1;
  if (n < 1) return -3;
  if (nrhs < 1) return -6;
  if (nsolves < 0) return -7;
  if (!p_candidates || np < 1) return -8;
  if (nr < 0 || (nr > 0 && !r13_candidates)) return -10;
  if (!out) return -14;
  memset(out, 0, sizeof(*out));
  const cudaStream_t st = (cudaStream_t)stream;
  double K = 0.0;
  int rc = spike_measure_K(band, ldab, n, kl, ku, stream, &K);
  if (rc != 0) return rc;
  out->K_measured = K;
  double *F = nullptr;
  const size_t fb = sizeof(double) * (size_t)n * nrhs;
  if (spk::dev_alloc((void **)&F, fb, st) != cudaSuccess || cudaMemsetAsync(F, 0, fb, st) != cudaSuccess) {
    cudaGetLastError();
    if (F) cudaFreeAsync(F, st);
    return SPIKE_ENOMEM;
  }
  // columns of the table: 0 = the paper's ratio with the measured K, 1 = stage balance, 2.. = explicit R13
  const int ncol = 2 + nr;
  out->best_ms = -1.0;
  bool warmed = false;
  for (int i = 0; i < np && rc == 0; ++i) {
    for (int c = 0; c < ncol && rc == 0; ++c) {
      spike_options o;
      memset(&o, 0, sizeof(o));
      o.stream = stream;
      o.nrhs_hint = nrhs;
      if (c == 0) o.K = K;
      if (c == 1) o.flags = SPIKE_FLAG_STAGE_BALANCE;
      if (c >= 2) o.R13 = r13_candidates[c - 2];
      double ms = 0.0;
      if (!warmed) {
        rc = run_once(band, ldab, n, kl, ku, p_candidates[i], o, F, nrhs, nsolves, st, &ms);
        warmed = true;
        if (rc != 0) break;
      }
      rc = run_once(band, ldab, n, kl, ku, p_candidates[i], o, F, nrhs, nsolves, st, &ms);
      if (rc != 0) break;
      if (table_ms) table_ms[(size_t)i * ncol + c] = ms;
      ++out->tried;
      if (i == 0 && c == 1) out->default_ms = ms;
      if (out->best_ms < 0.0 || ms < out->best_ms) {
        spike_info info;
        out->best_ms = ms;
        out->best_p = p_candidates[i];
        out->best_mode = c < 2 ? c : 2;
        out->best_R13 = 0.0;
        if (spike_plan(n, kl, ku, p_candidates[i], &o, &info, nullptr, nullptr) == 0) out->best_R13 = info.R13;
      }
    }
  }
  cudaFreeAsync(F, st);
  cudaStreamSynchronize(st);
  return rc;
}
