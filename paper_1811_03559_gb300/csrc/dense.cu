// Batched dense FP64 kernels for the recursive reduced system (Sec. 2.2) and
// the transpose reduced system (Sec. 4.3): strided GEMM, LU with partial
// pivoting of the 2k x 2k interface blocks (or of their k x k Schur
// complement), LU solves with N or T, plus the FP64 banded residual used to
// report backward errors.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <mutex>
#include <unordered_map>

#include "internal.h"

namespace spk {

#define FULLMASK 0xffffffffu

int device_sms() {
  static std::atomic<int> cache[16];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) {
    cudaGetLastError();
    dev = 0;
  }
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
    cudaGetLastError();
    v = 152;
  }
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

int smem_at_least(const void *func, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void *, size_t> cur;
  std::lock_guard<std::mutex> g(mu);
  size_t &c = cur[func];
  if (c >= bytes) return 0;
  const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) c = bytes;
  return (int)e;
}

// --------------------------------------------------------------- GEMM
// TS x TS output tile per CTA (TS = 64, 32 or 16), 256 threads, each a (TS/16)^2
// sub-tile (rows ty+16u, columns tx+16v), K staged through shared memory 16 at a time.
// One SM retires only ~2 FP64 FMAs per clock, so a 64 x 64 x 128 tile is ~0.1 ms of
// work; batches with too few 64-tiles to fill the GPU use smaller tiles (host choice).
// Each output is accumulated in the same fixed order for every TS, so a row of C gets
// the same bits whatever batch or tile size it is computed in.
template <int TS>
__global__ void __launch_bounds__(256) k_gemm(const GemmDesc *descs, int ndesc) {
  constexpr int R = TS / 16;
  __shared__ double As[16][TS + 1];
  __shared__ double Bs[16][TS + 1];
  const int tile = blockIdx.x;
  int lo = 0, hi = ndesc - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (descs[mid].tile0 <= tile) lo = mid;
    else hi = mid - 1;
  }
  const GemmDesc D = descs[lo];
  const int t = tile - D.tile0;
  const int i0 = (t / D.tiles_n) * TS, j0 = (t % D.tiles_n) * TS;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[R][R];
#pragma unroll
  for (int u = 0; u < R; ++u)
#pragma unroll
    for (int v = 0; v < R; ++v) acc[u][v] = 0.0;
  const bool a_kfast = (D.a_cs == 1 || D.a_cs == -1);
  const bool b_jfast = (D.b_cs == 1 || D.b_cs == -1);
  for (int kk = 0; kk < D.K; kk += 16) {
    for (int idx = tid; idx < 16 * TS; idx += 256) {
      int i, kq;
      if (a_kfast) {
        kq = idx & 15;
        i = idx >> 4;
      } else {
        i = idx % TS;
        kq = idx / TS;
      }
      double v = 0.0;
      if (i0 + i < D.M && kk + kq < D.K) {
        const int64_t o = (int64_t)(i0 + i) * D.a_rs + (int64_t)(kk + kq) * D.a_cs;
        v = (D.types & G_A32) ? (double)((const float *)D.A)[o] : D.A[o];
      }
      As[kq][i] = v;
      int j, kb;
      if (b_jfast) {
        j = idx % TS;
        kb = idx / TS;
      } else {
        kb = idx & 15;
        j = idx >> 4;
      }
      double w = 0.0;
      if (j0 + j < D.N && kk + kb < D.K) {
        const int64_t o = (int64_t)(kk + kb) * D.b_rs + (int64_t)(j0 + j) * D.b_cs;
        w = (D.types & G_B32) ? (double)((const float *)D.B)[o] : D.B[o];
      }
      Bs[kb][j] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kq = 0; kq < 16; ++kq) {
      double a[R], b[R];
#pragma unroll
      for (int u = 0; u < R; ++u) a[u] = As[kq][ty + 16 * u];
#pragma unroll
      for (int v = 0; v < R; ++v) b[v] = Bs[kq][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < R; ++u)
#pragma unroll
        for (int v = 0; v < R; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int i = i0 + ty + 16 * u;
    if (i >= D.M) continue;
#pragma unroll
    for (int v = 0; v < R; ++v) {
      const int j = j0 + tx + 16 * v;
      if (j >= D.N) continue;
      double r = D.alpha * acc[u][v];
      if (D.beta != 0.0) {
        const int64_t o = (int64_t)i * D.c0_rs + (int64_t)j * D.c0_cs;
        r = fma(D.beta, (D.types & G_C032) ? (double)((const float *)D.C0)[o] : D.C0[o], r);
      }
      const int64_t oc = (int64_t)i * D.c_rs + (int64_t)j * D.c_cs;
      if (D.types & G_C32) ((float *)D.C)[oc] = (float)r;
      else D.C[oc] = r;
    }
  }
}

// Few columns (N <= 8, e.g. single right-hand sides): 256 rows x TN columns per CTA, one row
// per thread.  Same per-output K order as k_gemm, so the same bits.
template <int TN>
__global__ void __launch_bounds__(256) k_gemm_skinny(const GemmDesc *descs, int ndesc) {
  __shared__ double As[16][256 + 1];
  __shared__ double Bs[16][TN];
  const int tile = blockIdx.x;
  int lo = 0, hi = ndesc - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (descs[mid].tile0 <= tile) lo = mid;
    else hi = mid - 1;
  }
  const GemmDesc D = descs[lo];
  const int t = tile - D.tile0;
  const int i0 = (t / D.tiles_n) * 256, j0 = (t % D.tiles_n) * TN;
  const int tid = threadIdx.x;
  double acc[TN];
#pragma unroll
  for (int v = 0; v < TN; ++v) acc[v] = 0.0;
  const bool a_kfast = (D.a_cs == 1 || D.a_cs == -1);
  for (int kk = 0; kk < D.K; kk += 16) {
    for (int idx = tid; idx < 16 * 256; idx += 256) {
      int i, kq;
      if (a_kfast) {
        kq = idx & 15;
        i = idx >> 4;
      } else {
        i = idx & 255;
        kq = idx >> 8;
      }
      double v = 0.0;
      if (i0 + i < D.M && kk + kq < D.K) {
        const int64_t o = (int64_t)(i0 + i) * D.a_rs + (int64_t)(kk + kq) * D.a_cs;
        v = (D.types & G_A32) ? (double)((const float *)D.A)[o] : D.A[o];
      }
      As[kq][i] = v;
    }
    if (tid < 16 * TN) {
      const int kb = tid / TN, j = tid % TN;
      double w = 0.0;
      if (j0 + j < D.N && kk + kb < D.K) {
        const int64_t o = (int64_t)(kk + kb) * D.b_rs + (int64_t)(j0 + j) * D.b_cs;
        w = (D.types & G_B32) ? (double)((const float *)D.B)[o] : D.B[o];
      }
      Bs[kb][j] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kq = 0; kq < 16; ++kq) {
      const double a = As[kq][tid];
#pragma unroll
      for (int v = 0; v < TN; ++v) acc[v] = fma(a, Bs[kq][v], acc[v]);
    }
    __syncthreads();
  }
  const int i = i0 + tid;
  if (i >= D.M) return;
#pragma unroll
  for (int v = 0; v < TN; ++v) {
    const int j = j0 + v;
    if (j >= D.N) continue;
    double r = D.alpha * acc[v];
    if (D.beta != 0.0) {
      const int64_t o = (int64_t)i * D.c0_rs + (int64_t)j * D.c0_cs;
      r = fma(D.beta, (D.types & G_C032) ? (double)((const float *)D.C0)[o] : D.C0[o], r);
    }
    const int64_t oc = (int64_t)i * D.c_rs + (int64_t)j * D.c_cs;
    if (D.types & G_C32) ((float *)D.C)[oc] = (float)r;
    else D.C[oc] = r;
  }
}

int launch_gemm(const GemmDesc *d, int ndesc, int total_tiles, int tile_size, void *stream) {
  if (ndesc <= 0 || total_tiles <= 0) return 0;
  const cudaStream_t st = (cudaStream_t)stream;
  if (tile_size < 0) {  // skinny: 256 rows x (-tile_size) columns
    if (tile_size == -1) k_gemm_skinny<1><<<total_tiles, 256, 0, st>>>(d, ndesc);
    else if (tile_size == -4) k_gemm_skinny<4><<<total_tiles, 256, 0, st>>>(d, ndesc);
    else k_gemm_skinny<8><<<total_tiles, 256, 0, st>>>(d, ndesc);
  } else if (tile_size == 16) k_gemm<16><<<total_tiles, 256, 0, st>>>(d, ndesc);
  else if (tile_size == 32) k_gemm<32><<<total_tiles, 256, 0, st>>>(d, ndesc);
  else k_gemm<64><<<total_tiles, 256, 0, st>>>(d, ndesc);
  count_launch();
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------- GETRF
// One CTA per matrix: unblocked right-looking LU with partial pivoting, whole-row
// swaps (L stored permuted, as in dense LAPACK getrf).  The pivot is the first row
// holding the largest |entry| of the column.  In shared memory when it fits.
constexpr int GETRF_SMEM_BYTES = 160 * 1024;

// smem_bytes: the dynamic shared memory this launch has; a matrix is factored there
// only when it fits in it (the launch sizes it for the batch's largest matrix, or 0).
__global__ void __launch_bounds__(256) k_getrf(const LuDesc *descs, unsigned long long *status, size_t smem_bytes) {
  extern __shared__ double sh[];
  const LuDesc D = descs[blockIdx.x];
  if (!D.active) return;
  const int n = D.n;
  const bool insm = (size_t)n * (n + 1) * sizeof(double) <= smem_bytes;
  double *A = insm ? sh : D.a;
  const int lda = insm ? n + 1 : D.lda;  // padded rows: the 16 x 16 update grid spreads over banks
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ double s_v[8];
  __shared__ int s_i[8];
  __shared__ int s_p;
  if (insm) {
    for (int idx = tid; idx < n * n; idx += 256) sh[(idx / n) * lda + idx % n] = D.a[(int64_t)(idx / n) * D.lda + idx % n];
    __syncthreads();
  }
  for (int j = 0; j < n; ++j) {
    double best = -1.0;
    int bi = n;
    for (int i = j + tid; i < n; i += 256) {
      const double v = fabs(A[(int64_t)i * lda + j]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
    for (int o = 16; o; o >>= 1) {
      const double ov = __shfl_down_sync(FULLMASK, best, o);
      const int oi = __shfl_down_sync(FULLMASK, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      s_v[warp] = best;
      s_i[warp] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      double b = s_v[0];
      int p = s_i[0];
      for (int w = 1; w < 8; ++w)
        if (s_v[w] > b || (s_v[w] == b && s_i[w] < p)) {
          b = s_v[w];
          p = s_i[w];
        }
      if (!(b > 0.0)) {
        p = j;
        atomicOr(D.status ? &D.status[2] : &status[2], 2ull);  // singular interface block
      }
      s_p = p;
      D.ipiv[j] = p;
    }
    __syncthreads();
    const int p = s_p;
    if (p != j) {
      for (int c = tid; c < n; c += 256) {
        const double t = A[(int64_t)j * lda + c];
        A[(int64_t)j * lda + c] = A[(int64_t)p * lda + c];
        A[(int64_t)p * lda + c] = t;
      }
      __syncthreads();
    }
    const double piv = A[(int64_t)j * lda + j];
    if (piv != 0.0) {
      const double rinv = 1.0 / piv;
      for (int i = j + 1 + tid; i < n; i += 256) A[(int64_t)i * lda + j] *= rinv;
      __syncthreads();
      // rank-1 update of the trailing block: thread (ty, tx) of a 16 x 16 grid owns rows
      // j+1+ty (+16 ...) and columns j+1+tx (+16 ...)
      const int ty = tid >> 4, tx = tid & 15;
      const double *urow = A + (int64_t)j * lda;
      for (int i = j + 1 + ty; i < n; i += 16) {
        double *row = A + (int64_t)i * lda;
        const double l = row[j];
        for (int c = j + 1 + tx; c < n; c += 16) row[c] = fma(-l, urow[c], row[c]);
      }
    }
    __syncthreads();
  }
  if (insm) {
    for (int idx = tid; idx < n * n; idx += 256) D.a[(int64_t)(idx / n) * D.lda + idx % n] = sh[(idx / n) * lda + idx % n];
  }
}

int launch_getrf(const LuDesc *d, int ndesc, int maxn, unsigned long long *status, void *stream) {
  if (ndesc <= 0) return 0;
  size_t smem = (size_t)maxn * (maxn + 1) * sizeof(double);
  if (smem > (size_t)GETRF_SMEM_BYTES) smem = GETRF_SMEM_BYTES;  // the matrices that fit still use it
  if (smem > 48 * 1024) {
    cudaError_t e = (cudaError_t)smem_at_least((const void *)k_getrf, smem);
    if (e != cudaSuccess) return (int)e;
  }
  k_getrf<<<ndesc, 256, smem, (cudaStream_t)stream>>>(d, status, smem);
  count_launch();
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------- GETRS
// One CTA per (matrix, TRS_COLS-column tile of B): 16 columns, or 4 when 16-column tiles
// would leave most SMs idle (each solve is 2 n^2 FMAs per column on one SM).  trans 0: M x = b with P M = L U;
// trans 1: M^T x = b (U^T forward, L^T backward, swaps undone in reverse).

// SMEM_LU: the n x n factor is first copied to shared memory (row stride n + 1), so the
// column reads of every elimination step are shared-memory broadcasts instead of strided
// global loads; the arithmetic and its order are the same in both forms.
template <bool SMEM_LU, int TRS_COLS>
__global__ void __launch_bounds__(256) k_getrs(const TrsDesc *descs, int ndesc) {
  extern __shared__ double trs_sm[];  // [LU n x (n+1)] when SMEM_LU, then B n x TRS_COLS
  const int tile = blockIdx.x;
  int lo = 0, hi = ndesc - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (descs[mid].tile0 <= tile) lo = mid;
    else hi = mid - 1;
  }
  const TrsDesc D = descs[lo];
  const int col0 = (tile - D.tile0) * TRS_COLS;
  const int nc = min(TRS_COLS, D.ncols - col0);
  const int n = D.n;
  const int tid = threadIdx.x;
  const double *LU = D.lu;
  int lda = D.lda;
  double *Bs = trs_sm;
  if (SMEM_LU) {
    double *L = trs_sm;
    for (int idx = tid; idx < n * n; idx += 256) {
      const int i = idx / n, j = idx - i * n;
      L[i * (n + 1) + j] = D.lu[(int64_t)i * D.lda + j];
    }
    LU = L;
    lda = n + 1;
    Bs = trs_sm + (size_t)n * (n + 1);
  }
  for (int idx = tid; idx < n * TRS_COLS; idx += 256) {
    const int i = idx / TRS_COLS, c = idx % TRS_COLS;
    Bs[idx] = (c < nc) ? D.alpha * D.b[(int64_t)i * D.ldb + col0 + c] : 0.0;
  }
  __syncthreads();
  if (!D.trans) {
    if (tid < nc)
      for (int j = 0; j < n; ++j) {
        const int p = D.ipiv[j];
        if (p != j) {
          const double t = Bs[j * TRS_COLS + tid];
          Bs[j * TRS_COLS + tid] = Bs[p * TRS_COLS + tid];
          Bs[p * TRS_COLS + tid] = t;
        }
      }
    __syncthreads();
    for (int j = 0; j < n - 1; ++j) {
      for (int idx = tid; idx < (n - j - 1) * TRS_COLS; idx += 256) {
        const int i = j + 1 + idx / TRS_COLS, c = idx % TRS_COLS;
        Bs[i * TRS_COLS + c] = fma(-LU[(int64_t)i * lda + j], Bs[j * TRS_COLS + c], Bs[i * TRS_COLS + c]);
      }
      __syncthreads();
    }
    for (int j = n - 1; j >= 0; --j) {
      if (tid < TRS_COLS) Bs[j * TRS_COLS + tid] = Bs[j * TRS_COLS + tid] / LU[(int64_t)j * lda + j];
      __syncthreads();
      for (int idx = tid; idx < j * TRS_COLS; idx += 256) {
        const int i = idx / TRS_COLS, c = idx % TRS_COLS;
        Bs[i * TRS_COLS + c] = fma(-LU[(int64_t)i * lda + j], Bs[j * TRS_COLS + c], Bs[i * TRS_COLS + c]);
      }
      __syncthreads();
    }
  } else {
    for (int j = 0; j < n; ++j) {
      if (tid < TRS_COLS) Bs[j * TRS_COLS + tid] = Bs[j * TRS_COLS + tid] / LU[(int64_t)j * lda + j];
      __syncthreads();
      for (int idx = tid; idx < (n - j - 1) * TRS_COLS; idx += 256) {
        const int i = j + 1 + idx / TRS_COLS, c = idx % TRS_COLS;
        Bs[i * TRS_COLS + c] = fma(-LU[(int64_t)j * lda + i], Bs[j * TRS_COLS + c], Bs[i * TRS_COLS + c]);
      }
      __syncthreads();
    }
    for (int j = n - 1; j > 0; --j) {
      for (int idx = tid; idx < j * TRS_COLS; idx += 256) {
        const int i = idx / TRS_COLS, c = idx % TRS_COLS;
        Bs[i * TRS_COLS + c] = fma(-LU[(int64_t)j * lda + i], Bs[j * TRS_COLS + c], Bs[i * TRS_COLS + c]);
      }
      __syncthreads();
    }
    if (tid < nc)
      for (int j = n - 1; j >= 0; --j) {
        const int p = D.ipiv[j];
        if (p != j) {
          const double t = Bs[j * TRS_COLS + tid];
          Bs[j * TRS_COLS + tid] = Bs[p * TRS_COLS + tid];
          Bs[p * TRS_COLS + tid] = t;
        }
      }
    __syncthreads();
  }
  for (int idx = tid; idx < n * TRS_COLS; idx += 256) {
    const int i = idx / TRS_COLS, c = idx % TRS_COLS;
    if (c < nc) D.b[(int64_t)i * D.ldb + col0 + c] = Bs[idx];
  }
}

int launch_getrs(const TrsDesc *d, int ndesc, int total_tiles, int maxn, int cols, void *stream) {
  if (ndesc <= 0 || total_tiles <= 0) return 0;
  const size_t bsm = (size_t)maxn * cols * sizeof(double);
  const size_t lsm = (size_t)maxn * (maxn + 1) * sizeof(double);
  const cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (bsm + lsm <= 200 * 1024) {
    if (cols == 4) {
      e = (cudaError_t)smem_at_least((const void *)k_getrs<true, 4>, bsm + lsm);
      if (e != cudaSuccess) return (int)e;
      k_getrs<true, 4><<<total_tiles, 256, bsm + lsm, st>>>(d, ndesc);
    } else {
      e = (cudaError_t)smem_at_least((const void *)k_getrs<true, 16>, bsm + lsm);
      if (e != cudaSuccess) return (int)e;
      k_getrs<true, 16><<<total_tiles, 256, bsm + lsm, st>>>(d, ndesc);
    }
  } else {
    if (cols == 4) {
      if (bsm > 48 * 1024) {
        e = (cudaError_t)smem_at_least((const void *)k_getrs<false, 4>, bsm);
        if (e != cudaSuccess) return (int)e;
      }
      k_getrs<false, 4><<<total_tiles, 256, bsm, st>>>(d, ndesc);
    } else {
      if (bsm > 48 * 1024) {
        e = (cudaError_t)smem_at_least((const void *)k_getrs<false, 16>, bsm);
        if (e != cudaSuccess) return (int)e;
      }
      k_getrs<false, 16><<<total_tiles, 256, bsm, st>>>(d, ndesc);
    }
  }
  count_launch();
  return (int)cudaGetLastError();
}

// ------------------------------------------------------ no-swap test
// flags[m] = 1 when every |entry| of the k x k block W[m] is <= 1: then partial
// pivoting on [I V; W I] keeps the identity rows as pivots for the first k
// columns (ties go to the first row), so its LU is [I 0; W I][I V; 0 S] with
// S = I - W V, and only S needs a pivoted LU.
__global__ void k_noswap(const double *const *w, int k, int *flags) {
  const double *W = w[blockIdx.x];
  int ok = 1;
  for (int64_t idx = threadIdx.x; idx < (int64_t)k * k; idx += blockDim.x)
    if (!(fabs(W[idx]) <= 1.0)) ok = 0;
  ok = __syncthreads_and(ok);
  if (threadIdx.x == 0) flags[blockIdx.x] = ok;
}

int launch_noswap_flags(const double *const *w, int k, int nm, int *flags, void *stream) {
  if (nm <= 0) return 0;
  k_noswap<<<nm, 256, 0, (cudaStream_t)stream>>>(w, k, flags);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_assemble_M(const double *const *, const double *const *, int, int, const int *, double *, int64_t,
                      void *) {
  return 0;  // assembly is expressed as GEMM copies (K = 0)
}

// ------------------------------------------------------------- transpose
// Column-major (rows x cols, ld) <-> row-major (rows x cols, row stride cols), 32 x 32 tiles.
__global__ void k_transpose(const double *__restrict__ in, double *__restrict__ out, int64_t rows, int cols,
                            int64_t ld, int to_row_major) {
  __shared__ double t[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int q = ty; q < 32; q += 8) {
    if (to_row_major) {  // read column-major: rows contiguous
      const int64_t r = r0 + tx;
      const int c = c0 + q;
      t[q][tx] = (r < rows && c < cols) ? in[(int64_t)c * ld + r] : 0.0;
    } else {             // read row-major: columns contiguous
      const int64_t r = r0 + q;
      const int c = c0 + tx;
      t[tx][q] = (r < rows && c < cols) ? in[r * cols + c] : 0.0;
    }
  }
  __syncthreads();
  for (int q = ty; q < 32; q += 8) {
    if (to_row_major) {
      const int64_t r = r0 + q;
      const int c = c0 + tx;
      if (r < rows && c < cols) out[r * cols + c] = t[tx][q];
    } else {
      const int64_t r = r0 + tx;
      const int c = c0 + q;
      if (r < rows && c < cols) out[(int64_t)c * ld + r] = t[q][tx];
    }
  }
}

int launch_transpose(const double *in, double *out, int64_t rows, int cols, int64_t ld, int to_row_major,
                     void *stream) {
  if (rows <= 0 || cols <= 0) return 0;
  dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((cols + 31) / 32));
  k_transpose<<<grid, 256, 0, (cudaStream_t)stream>>>(in, out, rows, cols, ld, to_row_major);
  count_launch();
  return (int)cudaGetLastError();
}

// Column-major FP64 <-> row-major FP32 work array (mixed-precision refinement).
// add mode: x += d for the columns with active[c] != 0 (all when active is null).
__global__ void k_work32(const double *__restrict__ in, int64_t ld, float *__restrict__ w, double *x,
                         const float *__restrict__ d, int64_t rows, int cols, int add, const int *active) {
  __shared__ double t[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (!add) {
    for (int q = ty; q < 32; q += 8) {
      const int64_t r = r0 + tx;
      const int c = c0 + q;
      t[q][tx] = (r < rows && c < cols) ? in[(int64_t)c * ld + r] : 0.0;
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {
      const int64_t r = r0 + q;
      const int c = c0 + tx;
      if (r < rows && c < cols) w[r * cols + c] = (float)t[tx][q];
    }
  } else {
    for (int q = ty; q < 32; q += 8) {
      const int64_t r = r0 + q;
      const int c = c0 + tx;
      t[tx][q] = (r < rows && c < cols) ? (double)d[r * cols + c] : 0.0;
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {
      const int64_t r = r0 + tx;
      const int c = c0 + q;
      if (r < rows && c < cols && (!active || active[c])) x[(int64_t)c * ld + r] += t[q][tx];
    }
  }
}

int launch_to_work32(const double *in, int64_t ld, float *out, int64_t rows, int cols, void *stream) {
  if (rows <= 0 || cols <= 0) return 0;
  dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((cols + 31) / 32));
  k_work32<<<grid, 256, 0, (cudaStream_t)stream>>>(in, ld, out, nullptr, nullptr, rows, cols, 0, nullptr);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_add_work32(double *x, int64_t ld, const float *d, int64_t rows, int cols, const int *active,
                      void *stream) {
  if (rows <= 0 || cols <= 0) return 0;
  dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((cols + 31) / 32));
  k_work32<<<grid, 256, 0, (cudaStream_t)stream>>>(nullptr, ld, nullptr, x, d, rows, cols, 1, active);
  count_launch();
  return (int)cudaGetLastError();
}

// -------------------------------------------------------- block sums
// out[e] = sum_{i < count} in[i*stride + e], summed in index order (deterministic).
__global__ void k_sum_blocks(const SumDesc *d) {
  const SumDesc D = d[blockIdx.y];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < D.elems; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < D.count; ++i) s += D.in[(int64_t)i * D.stride + e];
    D.out[e] = s;
  }
}

int launch_sum_blocks(const SumDesc *d, int ndesc, int64_t max_elems, void *stream) {
  if (ndesc <= 0) return 0;
  dim3 grid((unsigned)std::min<int64_t>((max_elems + 255) / 256, 64), (unsigned)ndesc);
  k_sum_blocks<<<grid, 256, 0, (cudaStream_t)stream>>>(d);
  count_launch();
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------------ axpy
__global__ void k_axpy(double *y, const double *x, double alpha, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(alpha, x[i], y[i]);
}

int launch_axpy(double *y, const double *x, double alpha, int64_t count, void *stream) {
  if (count <= 0) return 0;
  int blocks = (int)((count + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_axpy<<<blocks, 256, 0, (cudaStream_t)stream>>>(y, x, alpha, count);
  count_launch();
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------- residual
// One thread per row of op(A) and per RHS column (grid.y).  Norms are reduced
// with atomicMax on the bit patterns of non-negative doubles (order-independent).
__global__ void __launch_bounds__(256) k_berr(const double *__restrict__ band, int64_t ldab, int64_t n, int kl, int ku,
                                              const double *X, const double *F, int trans,
                                              unsigned long long *scratch) {
  const int c = blockIdx.y;
  const double *x = X + (int64_t)c * n;
  const double *f = F + (int64_t)c * n;
  double rmax = 0.0, xmax = 0.0, amax = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0, a = 0.0;
    if (!trans) {
      const int64_t jlo = i - kl > 0 ? i - kl : 0, jhi = i + ku < n - 1 ? i + ku : n - 1;
      for (int64_t j = jlo; j <= jhi; ++j) {
        const double v = band[j * ldab + ku + i - j];
        s = fma(v, x[j], s);
        a += fabs(v);
      }
    } else {
      const int64_t jlo = i - ku > 0 ? i - ku : 0, jhi = i + kl < n - 1 ? i + kl : n - 1;
      for (int64_t j = jlo; j <= jhi; ++j) {
        const double v = band[i * ldab + ku + j - i];
        s = fma(v, x[j], s);
        a += fabs(v);
      }
    }
    rmax = fmax(rmax, fabs(f[i] - s));
    xmax = fmax(xmax, fabs(x[i]));
    amax = fmax(amax, a);
  }
  for (int o = 16; o; o >>= 1) {
    rmax = fmax(rmax, __shfl_xor_sync(FULLMASK, rmax, o));
    xmax = fmax(xmax, __shfl_xor_sync(FULLMASK, xmax, o));
    amax = fmax(amax, __shfl_xor_sync(FULLMASK, amax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&scratch[1 + 2 * c], (unsigned long long)__double_as_longlong(rmax));
    atomicMax(&scratch[2 + 2 * c], (unsigned long long)__double_as_longlong(xmax));
    if (c == 0) atomicMax(&scratch[0], (unsigned long long)__double_as_longlong(amax));
  }
}

// R = F - op(A) X for the refinement loop, with the same norm reductions as k_berr.
__global__ void __launch_bounds__(256) k_resid(const double *__restrict__ band, int64_t ldab, int64_t n, int kl,
                                               int ku, const double *X, const double *F, double *R, int trans,
                                               unsigned long long *norms) {
  const int c = blockIdx.y;
  const double *x = X + (int64_t)c * n;
  const double *f = F + (int64_t)c * n;
  double *rr = R + (int64_t)c * n;
  double rmax = 0.0, xmax = 0.0, amax = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0, a = 0.0;
    if (!trans) {
      const int64_t jlo = i - kl > 0 ? i - kl : 0, jhi = i + ku < n - 1 ? i + ku : n - 1;
      for (int64_t j = jlo; j <= jhi; ++j) {
        const double v = band[j * ldab + ku + i - j];
        s = fma(v, x[j], s);
        a += fabs(v);
      }
    } else {
      const int64_t jlo = i - ku > 0 ? i - ku : 0, jhi = i + kl < n - 1 ? i + kl : n - 1;
      for (int64_t j = jlo; j <= jhi; ++j) {
        const double v = band[i * ldab + ku + j - i];
        s = fma(v, x[j], s);
        a += fabs(v);
      }
    }
    const double r = f[i] - s;
    rr[i] = r;
    rmax = fmax(rmax, fabs(r));
    xmax = fmax(xmax, fabs(x[i]));
    amax = fmax(amax, a);
  }
  for (int o = 16; o; o >>= 1) {
    rmax = fmax(rmax, __shfl_xor_sync(FULLMASK, rmax, o));
    xmax = fmax(xmax, __shfl_xor_sync(FULLMASK, xmax, o));
    amax = fmax(amax, __shfl_xor_sync(FULLMASK, amax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&norms[1 + 2 * c], (unsigned long long)__double_as_longlong(rmax));
    atomicMax(&norms[2 + 2 * c], (unsigned long long)__double_as_longlong(xmax));
    if (c == 0) atomicMax(&norms[0], (unsigned long long)__double_as_longlong(amax));
  }
}

// Tiled form for many right-hand sides: one CTA owns RT consecutive rows of op(A).
// Row i of op(A) holds the entries at columns i - lo + d, d in [0, W), W = lo + hi + 1
// (lo = kl, hi = ku for N; swapped for T).  The CTA stages those RT x W entries once
// (as[li][d], row stride WP) and then, for each chunk of MC columns, the RT + W - 1
// rows of X the tile touches (xs[r][c], row stride MC + 1), so every global load is a
// contiguous run: band columns (N) or band rows (T), and X columns.  Thread (tr, tc)
// accumulates RPT consecutive rows of column tc in ascending d; results are staged
// in smem and written a column at a time, lanes over rows.
template <int RPT>
__global__ void __launch_bounds__(256) k_resid_tile(const double *__restrict__ band, int64_t ldab, int64_t n, int kl,
                                                    int ku, const double *__restrict__ X, const double *__restrict__ F,
                                                    double *R, int nrhs, int trans, int RT, int MC, int WP,
                                                    unsigned long long *norms) {
  extern __shared__ double smr[];
  const int lo = trans ? ku : kl, hi = trans ? kl : ku, W = lo + hi + 1;
  const int XT = RT + W - 1, XP = MC + 1;
  double *as = smr;                     // RT x WP
  double *xs = as + (size_t)RT * WP;    // XT x XP
  double *rs = xs + (size_t)XT * XP;    // RT x XP
  const int64_t i0 = (int64_t)blockIdx.x * RT;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // band tile, zero outside the matrix
  if (!trans) {
    // column j of A holds rows j-ku .. j+kl contiguously: band[j*ldab + ku + i - j]
    for (int jj = warp; jj < RT + W - 1; jj += 8) {
      const int64_t j = i0 - lo + jj;
      for (int li = lane; li < RT; li += 32) {
        const int64_t i = i0 + li;
        const int d = (int)(j - i) + lo;
        if (d < 0 || d >= W) continue;
        as[li * WP + d] = (i < n && j >= 0 && j < n) ? band[j * ldab + ku + i - j] : 0.0;
      }
    }
  } else {
    // row i of A^T is column i of A: band[i*ldab + d] with j = i - ku + d
    for (int idx = tid; idx < RT * W; idx += 256) {
      const int li = idx / W, d = idx - li * W;
      const int64_t i = i0 + li, j = i - lo + d;
      as[li * WP + d] = (i < n && j >= 0 && j < n) ? band[i * ldab + d] : 0.0;
    }
  }
  __syncthreads();
  if (tid < ((RT + 31) & ~31)) {  // whole warps: the reduction below shuffles
    double a = 0.0;
    if (tid < RT && i0 + tid < n)
      for (int d = 0; d < W; ++d) a += fabs(as[tid * WP + d]);
    for (int o = 16; o; o >>= 1) a = fmax(a, __shfl_xor_sync(FULLMASK, a, o));
    if (lane == 0) atomicMax(&norms[0], (unsigned long long)__double_as_longlong(a));
  }
  const int tc = tid % MC, tr = tid / MC;  // 256 / MC row lanes x RPT rows = RT
  for (int c0 = 0; c0 < nrhs; c0 += MC) {
    const int mc = min(MC, nrhs - c0);
    __syncthreads();
    for (int idx = tid; idx < XT * MC; idx += 256) {
      const int r = idx % XT, c = idx / XT;
      const int64_t j = i0 - lo + r;
      xs[r * XP + c] = (c < mc && j >= 0 && j < n) ? X[(int64_t)(c0 + c) * n + j] : 0.0;
    }
    __syncthreads();
    if (tr * RPT < RT) {
      double acc[RPT];
#pragma unroll
      for (int q = 0; q < RPT; ++q) acc[q] = 0.0;
      const double *ap = as + (size_t)(tr * RPT) * WP;
      const double *xp = xs + (size_t)(tr * RPT) * XP + tc;
      for (int d = 0; d < W; ++d) {
#pragma unroll
        for (int q = 0; q < RPT; ++q) acc[q] = fma(ap[q * WP + d], xp[(q + d) * XP], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < RPT; ++q) rs[(tr * RPT + q) * XP + tc] = acc[q];
    }
    __syncthreads();
    for (int c = warp; c < mc; c += 8) {
      const int64_t col = c0 + c;
      double rmax = 0.0, xmax = 0.0;
      for (int li = lane; li < RT; li += 32) {
        const int64_t i = i0 + li;
        if (i >= n) continue;
        const double r = F[col * n + i] - rs[li * XP + c];
        if (R) R[col * n + i] = r;
        rmax = fmax(rmax, fabs(r));
        xmax = fmax(xmax, fabs(xs[(li + lo) * XP + c]));
      }
      for (int o = 16; o; o >>= 1) {
        rmax = fmax(rmax, __shfl_xor_sync(FULLMASK, rmax, o));
        xmax = fmax(xmax, __shfl_xor_sync(FULLMASK, xmax, o));
      }
      if (lane == 0) {
        atomicMax(&norms[1 + 2 * col], (unsigned long long)__double_as_longlong(rmax));
        atomicMax(&norms[2 + 2 * col], (unsigned long long)__double_as_longlong(xmax));
      }
    }
  }
}

// Tile shape for k_resid_tile: MC columns per chunk (>= 8), RT rows, all in <= 200 KB
// of shared memory.  Returns false when no shape fits (very wide bands).
static bool resid_tile_shape(int kl, int ku, int nrhs, int *RT, int *MC, int *WP, int *RPT, size_t *smem) {
  const int W = kl + ku + 1;
  const int wp = (W % 2 == 1) ? W + 1 : W;  // WP - 1 odd: the column-wise band loads spread over banks
  for (int mc = (nrhs >= 32 ? 32 : (nrhs >= 16 ? 16 : 8)); mc >= 8; mc /= 2) {
    const int TR = 256 / mc;
    for (int rpt = 8; rpt >= 1; rpt /= 2) {
      const int rt = TR * rpt;
      if (rt > 64) continue;
      const size_t bytes = sizeof(double) * ((size_t)rt * wp + (size_t)(rt + W - 1) * (mc + 1) + (size_t)rt * (mc + 1));
      if (bytes <= 200 * 1024) {
        *RT = rt;
        *MC = mc;
        *WP = wp;
        *RPT = rpt;
        *smem = bytes;
        return true;
      }
    }
  }
  return false;
}

static int launch_resid_tile(const double *band, int64_t ldab, int64_t n, int kl, int ku, const double *X,
                             const double *F, double *R, int nrhs, int trans, unsigned long long *norms,
                             cudaStream_t st, bool *done) {
  *done = false;
  int RT, MC, WP, RPT;
  size_t smem;
  if (nrhs < 8 || !resid_tile_shape(kl, ku, nrhs, &RT, &MC, &WP, &RPT, &smem)) return 0;
  const unsigned grid = (unsigned)((n + RT - 1) / RT);
  cudaError_t e = cudaSuccess;
#define SPK_RESID(RP)                                                                                         \
  case RP:                                                                                                    \
    e = (cudaError_t)smem_at_least((const void *)k_resid_tile<RP>, smem);                                     \
    if (e != cudaSuccess) return (int)e;                                                                      \
    k_resid_tile<RP><<<grid, 256, smem, st>>>(band, ldab, n, kl, ku, X, F, R, nrhs, trans, RT, MC, WP, norms); \
    break;
  switch (RPT) {
    SPK_RESID(1)
    SPK_RESID(2)
    SPK_RESID(4)
    SPK_RESID(8)
    default: return 0;
  }
#undef SPK_RESID
  count_launch();
  *done = true;
  return (int)cudaGetLastError();
}

int launch_residual(const double *band, int64_t ldab, int64_t n, int kl, int ku, const double *X, const double *F,
                    double *R, int nrhs, int trans, unsigned long long *norms, void *stream) {
  bool done;
  const int e = launch_resid_tile(band, ldab, n, kl, ku, X, F, R, nrhs, trans, norms, (cudaStream_t)stream, &done);
  if (e || done) return e;
  int bx = (int)((n + 255) / 256);
  if (bx > 152 * 8) bx = 152 * 8;
  dim3 grid(bx, nrhs);
  k_resid<<<grid, 256, 0, (cudaStream_t)stream>>>(band, ldab, n, kl, ku, X, F, R, trans, norms);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_berr(const double *band, int64_t ldab, int64_t n, int kl, int ku, const double *X, const double *F,
                int nrhs, int trans, unsigned long long *scratch, void *stream) {
  bool done;
  const int e = launch_resid_tile(band, ldab, n, kl, ku, X, F, nullptr, nrhs, trans, scratch, (cudaStream_t)stream,
                                  &done);
  if (e || done) return e;
  int bx = (int)((n + 255) / 256);
  if (bx > 152 * 8) bx = 152 * 8;
  dim3 grid(bx, nrhs);
  k_berr<<<grid, 256, 0, (cudaStream_t)stream>>>(band, ldab, n, kl, ku, X, F, trans, scratch);
  count_launch();
  return (int)cudaGetLastError();
}

// -------------------------------------------------------- FP64 FMA probe
__global__ void __launch_bounds__(512) k_dfma_probe(double *out, int iters, double b, double c) {
  double a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// -------------------------------------------- backward error without allocation
// Fixed reduction scratch for spike_backward_error_noalloc:
//   [0]                         ||op(A)||_inf      (bit pattern, atomicMax)
//   [1 + 2c], [2 + 2c]          residual and ||x_c|| of column c
//   [1 + 2*MAX + c]             the finished berr[c] (as a double)
constexpr int NOALLOC_WORDS = 1 + 3 * SPIKE_NOALLOC_MAX_NRHS;
static __device__ __align__(256) unsigned long long g_noalloc_scratch[NOALLOC_WORDS];

// Host code must not pass g_noalloc_scratch itself to a kernel: on the host that name
// is a stand-in, not a device address.  The address is looked up once per device.
constexpr int NOALLOC_MAX_DEVICES = 64;
static std::atomic<unsigned long long *> g_noalloc_addr[NOALLOC_MAX_DEVICES];

static int noalloc_scratch(unsigned long long **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPIKE_ECUDA;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return SPIKE_ELIMIT;
  unsigned long long *p = g_noalloc_addr[dev].load(std::memory_order_acquire);
  if (!p) {
    void *addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || addr == nullptr) return SPIKE_ECUDA;
    p = (unsigned long long *)addr;
    g_noalloc_addr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return 0;
}

__global__ void k_berr_finish(unsigned long long *scr, int nrhs) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nrhs) return;
  const double an = __longlong_as_double((long long)scr[0]);
  const double r = __longlong_as_double((long long)scr[1 + 2 * c]);
  const double x = __longlong_as_double((long long)scr[2 + 2 * c]);
  const double b = (an > 0 && x > 0) ? r / (an * x) : (r == 0 ? 0.0 : INFINITY);
  scr[1 + 2 * SPIKE_NOALLOC_MAX_NRHS + c] = (unsigned long long)__double_as_longlong(b);
}

}  // namespace spk

extern "C" int spike_backward_error_noalloc(const double *band, int64_t ldab, int64_t n, int kl, int ku,
                                            const double *X, const double *F, int nrhs, char trans, void *stream,
                                            double *berr) {
  if (!band) return -1;
  if (ldab < (int64_t)kl + ku + 1) return -2;
  if (n < 1) return -3;
  if (kl < 0) return -4;
  if (ku < 0) return -5;
  if (!X) return -6;
  if (!F) return -7;
  if (nrhs < 1) return -8;
  if (nrhs > SPIKE_NOALLOC_MAX_NRHS) return SPIKE_ELIMIT;
  if (trans != 'N' && trans != 'n' && trans != 'T' && trans != 't') return -9;
  if (!berr) return -11;
  unsigned long long *scr = nullptr;
  const int rc = spk::noalloc_scratch(&scr);
  if (rc != 0) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  // the norms are max-reductions from zero: clear the words this call uses
  if (cudaMemsetAsync(scr, 0, sizeof(unsigned long long) * (1 + 2 * (size_t)nrhs), s) != cudaSuccess)
    return SPIKE_ECUDA;
  if (spk::launch_berr(band, ldab, n, kl, ku, X, F, nrhs, (trans == 'T' || trans == 't') ? 1 : 0, scr, s) != 0)
    return SPIKE_ECUDA;
  spk::k_berr_finish<<<(nrhs + 127) / 128, 128, 0, s>>>(scr, nrhs);
  spk::count_launch();
  if (cudaGetLastError() != cudaSuccess) return SPIKE_ECUDA;
  if (cudaMemcpyAsync(berr, scr + 1 + 2 * SPIKE_NOALLOC_MAX_NRHS, sizeof(double) * (size_t)nrhs,
                      cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return SPIKE_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SPIKE_ECUDA;
  return 0;
}

namespace spk {
// -------------------------------------------------------- pipe probes
// Throughput loops for spike_measure_pipes.  Each thread (or warp, for mma.sync) runs 8
// independent dependent chains; `sel` picks which warps run: bit 0 the even warps, bit 1
// the odd warps (3 = all), so one kernel gives the solo and the mixed runs.
__device__ __forceinline__ bool probe_runs(int sel) {
  const int w = threadIdx.x >> 5;
  return (w & 1) ? (sel & 2) != 0 : (sel & 1) != 0;
}

// DFMA chains (sel selects the warps) or, with dmma_sel, mma.sync.m8n8k4.f64 chains on the
// other selection: the shared-pipe experiment runs both in alternate warps.
__global__ void __launch_bounds__(512) k_pipe_fp64(double *out, int iters, int dfma_sel, int dmma_sel) {
  double r = 0.0;
  if (probe_runs(dfma_sel)) {
    double a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = threadIdx.x * 1e-3 + i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = fma(a[i], 1.0000001, 1e-9);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) r += a[i];
  } else if (probe_runs(dmma_sel)) {
    // per warp: 8 accumulator pairs of an 8x8 f64 tile, A and B fragments fixed
    const double fa = 1.0 + threadIdx.x * 1e-7, fb = 1e-3;
    double c[8][2];
#pragma unroll
    for (int i = 0; i < 8; ++i) c[i][0] = c[i][1] = i;
    // one mma.sync m8n8k4 = 256 FMAs per warp, 8 per lane: iters / 8 of them per chain give a
    // lane the DFMA loop's iters FMAs per chain
    const int n = iters / 8;
    for (int it = 0; it < n; ++it) {
#pragma unroll
      for (int i = 0; i < 8; ++i)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                     : "+d"(c[i][0]), "+d"(c[i][1])
                     : "d"(fa), "d"(fb));
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) r += c[i][0] + c[i][1];
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void __launch_bounds__(512) k_pipe_fp32(float *out, int iters) {
  float a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = threadIdx.x * 1e-3f + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fmaf(a[i], 1.0000001f, 1e-9f);
  }
  float r = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) r += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// mma.sync.m16n8k16 bf16 -> f32, 8 independent accumulator tiles per warp
__global__ void __launch_bounds__(512) k_pipe_bf16(float *out, int iters) {
  const uint32_t a0 = 0x3f803f80u, a1 = 0x3f003f00u, b0 = 0x3c003c00u;
  float c[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i) c[i][0] = c[i][1] = c[i][2] = c[i][3] = 0.f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                   "{%0,%1,%2,%3};\n"
                   : "+f"(c[i][0]), "+f"(c[i][1]), "+f"(c[i][2]), "+f"(c[i][3])
                   : "r"(a0), "r"(a1), "r"(a0), "r"(a1), "r"(b0), "r"(b0));
  }
  float r = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) r += c[i][0] + c[i][1] + c[i][2] + c[i][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

}  // namespace spk

extern "C" int spike_measure_fp64_peak(void *stream, double *tflops) {
  if (!tflops) return -2;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SPIKE_ECUDA;
  const int blocks = 2 * sms, threads = 512, iters = 8192;
  double *out = nullptr;
  if (spk::dev_alloc((void **)&out, sizeof(double) * blocks * threads, s) != cudaSuccess) return SPIKE_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  spk::k_dfma_probe<<<blocks, threads, 0, s>>>(out, iters / 8, 1.0000001, 1e-9);  // warm-up
  cudaEventRecord(e0, s);
  spk::k_dfma_probe<<<blocks, threads, 0, s>>>(out, iters, 1.0000001, 1e-9);
  cudaEventRecord(e1, s);
  spk::count_launch(2);
  float ms = 0.0f;
  const bool ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, s);
  if (!ok || ms <= 0.0f) return SPIKE_ECUDA;
  *tflops = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
  return 0;
}

extern "C" int spike_measure_pipes(void *stream, double *out, int count) {
  if (!out) return -2;
  if (count < 1) return -3;
  for (int i = 0; i < count; ++i) out[i] = 0.0;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SPIKE_ECUDA;
  const int blocks = 2 * sms, threads = 512, iters = 8192;
  const size_t nthr = (size_t)blocks * threads;
  double *buf = nullptr;
  if (spk::dev_alloc((void **)&buf, sizeof(double) * nthr, s) != cudaSuccess) return SPIKE_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  bool ok = true;
  // time one launch (after an untimed short one of the same kernel), in ms
  auto timed = [&](auto launch) {
    launch(iters / 8);
    cudaEventRecord(e0, s);
    launch(iters);
    cudaEventRecord(e1, s);
    spk::count_launch(2);
    float ms = 0.0f;
    ok = ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.0f;
    return (double)ms;
  };
  const double fma_flop = 2.0 * 8.0 * (double)iters * nthr;  // 8 chains x iters FMAs per thread
  auto fp64 = [&](int dsel, int msel) {
    return timed([&](int it) { spk::k_pipe_fp64<<<blocks, threads, 0, s>>>(buf, it, dsel, msel); });
  };
  // the DFMA rate from the peak probe's kernel (the roofline denominator), the rest from the
  // selectable kernel, which also runs the solo and mixed halves of the shared-pipe experiment
  const double t_dfma = timed([&](int it) { spk::k_dfma_probe<<<blocks, threads, 0, s>>>(buf, it, 1.0000001, 1e-9); });
  const double t_dmma = fp64(0, 3);
  const double t_even_dfma = fp64(1, 0), t_odd_dmma = fp64(0, 2), t_mix = fp64(1, 2);
  const double t_fp32 = timed([&](int it) { spk::k_pipe_fp32<<<blocks, threads, 0, s>>>((float *)buf, it); });
  const double t_bf16 = timed([&](int it) { spk::k_pipe_bf16<<<blocks, threads, 0, s>>>((float *)buf, it); });
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(buf, s);
  if (!ok || cudaGetLastError() != cudaSuccess) return SPIKE_ECUDA;
  // per warp: 8 chains of iters / 8 m8n8k4 MMAs of 256 FMAs (the same FMAs as the DFMA loop);
  // bf16: 8 chains of iters m16n8k16 MMAs of 2048 FMAs
  const double mma64_flop = 2.0 * 8.0 * (double)(iters / 8) * 256.0 * (nthr / 32);
  const double bf16_flop = 2.0 * 8.0 * (double)iters * 2048.0 * (nthr / 32);
  const double vals[7] = {fma_flop / (t_dfma * 1e-3) / 1e12,
                          mma64_flop / (t_dmma * 1e-3) / 1e12,
                          fma_flop / (t_fp32 * 1e-3) / 1e12,
                          bf16_flop / (t_bf16 * 1e-3) / 1e12,
                          t_even_dfma,
                          t_odd_dmma,
                          t_mix};
  for (int i = 0; i < count && i < 7; ++i) out[i] = vals[i];
  return 0;
}
