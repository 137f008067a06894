// Per-block ("leaf") kernels of the recursive SPIKE factorization and solves.
// One CTA owns one diagonal block A_i in its local frame (reversed for the UL
// blocks: UL(A_i) = Q LU(Q A_i Q) Q, Sec. 5.2), so every kernel here is an LU
// kernel.  All arithmetic is FP64 on the CUDA-core FMA pipe; on this part that
// pipe, not HBM, bounds every kernel, so the designs below aim at keeping
// four or more warps per SM issuing independent FMAs and at minimising the
// number of CTA-wide barriers per factored column.
//
// Storage (device, local frame, column-major):
//   fb   : column c of a leaf at fb + c*ldf; entry (r, c) of the combined LU
//          (unit L strictly below, U on/above the diagonal) at [dofs + r - c],
//          dofs = k (no pivoting) or 2k (partial pivoting: U gains kl extra
//          superdiagonals, Sec. 5.1).
//   dinv : 1 / U(r, r).
//   Z    : the two spike right-hand sides of a leaf, column-major with nl rows:
//          columns [0, k) = [R_top; 0] (coupling through the local top rows),
//          columns [k, 2k) = [0; R_bot] (coupling through the local bottom rows).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "internal.h"

namespace spk {

#define FULLMASK 0xffffffffu

constexpr int WCH = 256;  // sweep window rows per staged chunk
constexpr int SCW = 128;  // RHS columns per sweep pass: 8 warps x 16 accumulators
constexpr int WSPLIT = NTHREADS / 32;  // fixed sub-ranges of each window chunk (one per warp)
// two buffers of the block coefficients (window Tw, diagonal block Td, reciprocals) so the next
// block's are copied in while the current one computes, plus the right-hand-side block Gs
constexpr size_t SWEEP_SMEM = sizeof(double) * (2 * ((size_t)WCH * NB + NB * NB + NB) + (size_t)NB * (SCW + 1));

// ------------------------------------------------------------------ repack
// User band (LAPACK layout, global frame) -> per-leaf LU band (local frame),
// zero outside A_i's band, plus max|a_ij| for the boosting threshold.
template <typename T>
__global__ void __launch_bounds__(256) k_repack(const double *__restrict__ band, int64_t ldab, int kl, int ku,
                                                int64_t n, int k, int ldf, int dofs, const LeafDev *leaves,
                                                T *fb, unsigned long long *amax_bits) {
  const LeafDev L = leaves[blockIdx.y];
  const int64_t nl = L.len;
  const int64_t ncols_per_blk = 8;
  const int64_t c0 = (int64_t)blockIdx.x * ncols_per_blk;
  double lmax = 0.0;
  for (int64_t idx = threadIdx.x; idx < ncols_per_blk * ldf; idx += blockDim.x) {
    const int64_t c = c0 + idx / ldf;
    const int d = (int)(idx % ldf);
    if (c >= nl) break;
    const int64_t r = c + d - dofs;
    double v = 0.0;
    if (r >= 0 && r < nl && r - c <= k && c - r <= k) {
      const int64_t gi = L.rev ? (L.start + nl - 1 - r) : (L.start + r);
      const int64_t gj = L.rev ? (L.start + nl - 1 - c) : (L.start + c);
      const int64_t off = gi - gj;
      if (off >= -ku && off <= kl) v = band[gj * ldab + ku + off];
    }
    fb[(L.start + c) * ldf + d] = (T)v;
    lmax = fmax(lmax, fabs(v));
  }
  for (int o = 16; o; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(FULLMASK, lmax, o));
  if ((threadIdx.x & 31) == 0 && lmax > 0.0) atomicMax(amax_bits, (unsigned long long)__double_as_longlong(lmax));
}

int launch_repack(const double *band, int64_t ldab, int kl, int ku, int64_t n, int k, int ldf, int dofs,
                  const LeafDev *leaves, int nleaves, void *fb, unsigned long long *amax_bits, void *stream,
                  int64_t max_leaf_len, int f32) {
  dim3 grid((unsigned)((max_leaf_len + 7) / 8), (unsigned)nleaves);
  if (f32)
    k_repack<float><<<grid, 256, 0, (cudaStream_t)stream>>>(band, ldab, kl, ku, n, k, ldf, dofs, leaves, (float *)fb,
                                                            amax_bits);
  else
    k_repack<double><<<grid, 256, 0, (cudaStream_t)stream>>>(band, ldab, kl, ku, n, k, ldf, dofs, leaves,
                                                             (double *)fb, amax_bits);
  count_launch();
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------- couplings
// couple[leaf][0] = R_top (k x k, row-major, local row order): rows = local top k rows,
//   columns = the tip unknowns of the neighbour coupled through the top (global order):
//   forward leaf: C_i-hat (previous block's last k columns); reversed: Q_k B_i-hat (next block's first k).
// couple[leaf][1] = R_bot: rows = local bottom k rows; forward: B_i-hat; reversed: Q_k C_i-hat.
__global__ void k_couplings(const double *__restrict__ band, int64_t ldab, int kl, int ku, int64_t n, int k,
                            const LeafDev *leaves, double *couple) {
  const LeafDev L = leaves[blockIdx.x];
  const int64_t nl = L.len;
  const int64_t kk = (int64_t)k * k;
  double *Rt = couple + (int64_t)blockIdx.x * 2 * kk;
  double *Rb = Rt + kk;
  for (int64_t idx = threadIdx.x; idx < kk; idx += blockDim.x) {
    const int a = (int)(idx / k), b = (int)(idx % k);
    // top: local row a
    double vt = 0.0, vb = 0.0;
    {
      const int64_t gi = L.rev ? (L.start + nl - 1 - a) : (L.start + a);
      const int64_t gj = L.rev ? (L.start + nl + b) : (L.start - k + b);
      const int64_t off = gi - gj;
      if (L.top_nbr && gj >= 0 && gj < n && off >= -ku && off <= kl) vt = band[gj * ldab + ku + off];
    }
    {
      const int64_t r = nl - k + a;
      const int64_t gi = L.rev ? (L.start + nl - 1 - r) : (L.start + r);
      const int64_t gj = L.rev ? (L.start - k + b) : (L.start + nl + b);
      const int64_t off = gi - gj;
      if (L.bot_nbr && gj >= 0 && gj < n && off >= -ku && off <= kl) vb = band[gj * ldab + ku + off];
    }
    Rt[idx] = vt;
    Rb[idx] = vb;
  }
}

int launch_couplings(const double *band, int64_t ldab, int kl, int ku, int64_t n, int k, const LeafDev *leaves,
                     int nleaves, double *couple, void *stream) {
  k_couplings<<<nleaves, 256, 0, (cudaStream_t)stream>>>(band, ldab, kl, ku, n, k, leaves, couple);
  count_launch();
  return (int)cudaGetLastError();
}

// Z init (Z already zeroed): R_top into rows [0,k) of columns [0,k) for leaves that
// need the top spike (both neighbours), R_bot into rows [nl-k, nl) of columns [k, 2k).
template <typename T>
__global__ void k_zinit(const LeafDev *leaves, int k, const double *couple, T *zbuf, const int64_t *zoff) {
  const LeafDev L = leaves[blockIdx.x];
  const int64_t nl = L.len;
  const int64_t kk = (int64_t)k * k;
  const double *Rt = couple + (int64_t)blockIdx.x * 2 * kk;
  const double *Rb = Rt + kk;
  T *Z = zbuf + zoff[blockIdx.x];
  const bool mid = L.top_nbr && L.bot_nbr;
  for (int64_t idx = threadIdx.x; idx < kk; idx += blockDim.x) {
    const int a = (int)(idx % k), b = (int)(idx / k);  // row a fastest -> coalesced column-major writes
    if (mid) Z[(int64_t)b * nl + a] = (T)Rt[(int64_t)a * k + b];
    if (L.bot_nbr) Z[(int64_t)(k + b) * nl + (nl - k + a)] = (T)Rb[(int64_t)a * k + b];
  }
}

int launch_zinit(const LeafDev *leaves, int nleaves, int k, const double *couple, void *zbuf, const int64_t *zoff,
                 int f32, void *stream) {
  if (f32)
    k_zinit<float><<<nleaves, 256, 0, (cudaStream_t)stream>>>(leaves, k, couple, (float *)zbuf, zoff);
  else
    k_zinit<double><<<nleaves, 256, 0, (cudaStream_t)stream>>>(leaves, k, couple, (double *)zbuf, zoff);
  count_launch();
  return (int)cudaGetLastError();
}

template <typename T>
__device__ void sweep_run(const SweepDesc &D, int ldf, int dofs, T *sm);

// -------------------------------------------------- non-pivoting block LU
// Row stride of the U12 chunk in shared memory: odd for FP64 (conflict-free column access);
// a multiple of 4 for FP32, so a row's 16 columns are read as four 16-byte loads.
template <typename T>
constexpr int FACTOR_TLD = (sizeof(T) == 4) ? CW + 4 : CW + 1;

// v[0..15] = p[0..15] (p 16-byte aligned for FP32)
template <typename T>
__device__ __forceinline__ void load16(const T *p, T (&v)[16]) {
  if constexpr (sizeof(T) == 4) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 x = q[i];
      v[4 * i] = x.x;
      v[4 * i + 1] = x.y;
      v[4 * i + 2] = x.z;
      v[4 * i + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = p[i];
  }
}

// Blocked right-looking band LU (no pivoting, diagonal boosting, Sec. 2.3) of one
// leaf, with the L-sweep of the top spike fused as extra columns: for a middle
// leaf, Z[:, 0:k] <- L^{-1} [R_top; 0] as the factorization proceeds (the first
// of the three factor-stage sweeps of a middle partition, Table tab:sweeps).
// Per block of NB columns: panel LU in shared memory (NB columns x NB+k rows),
// U12 = L11^{-1} A12 (and the fused Z rows), then A22 -= L21 U12 on the k x k
// window (and the fused Z rows below the panel).
template <typename T>
__device__ void factor_leaf(const LeafDev &L, int k, int ldf, T *fb_all, T *dinv_all, T *Z,
                            const unsigned long long *amax_bits, double boost_eps, unsigned long long *status,
                            const SweepDesc &sw0, const SweepDesc &sw1, T *smem) {
  const int64_t nl = L.len;
  T *fb = fb_all + L.start * (int64_t)ldf;
  T *dinv = dinv_all + L.start;
  const bool fuse = L.top_nbr && L.bot_nbr;
  const int kz = fuse ? k : 0;
  const int PLD = NB + k + 1;
  const int TLD = FACTOR_TLD<T>;
  T *P = smem;                // NB columns x PLD rows, column-major
  T *T12 = smem + NB * PLD;   // NB rows x TLD, row-major
  __shared__ T s_rinv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T tau = (T)(boost_eps * __longlong_as_double((long long)*amax_bits));
  unsigned long long nboost = 0;

  for (int64_t j0 = 0; j0 < nl; j0 += NB) {
    const int jb = (int)min((int64_t)NB, nl - j0);
    const int prow = (int)min((int64_t)(jb + k), nl - j0);
    // (a) panel load
    for (int base = tid; base < NB * PLD; base += NTHREADS * 8) {
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = base + u * NTHREADS;
        const int c = idx / PLD, r = idx - c * PLD;
        v[u] = (idx < NB * PLD && c < jb && r < prow && r - c <= k && c - r <= k) ? fb[(j0 + c) * ldf + k + r - c]
                                                                                   : (T)0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (base + u * NTHREADS < NB * PLD) P[base + u * NTHREADS] = v[u];
    }
    __syncthreads();
    // (b) panel LU
    for (int c = 0; c < jb; ++c) {
      if (tid == 0) {
        T piv = P[c * PLD + c];
        if (isnan(piv)) {
          atomicOr(&status[2], 1ull);
        } else if (!(fabs(piv) >= tau) || piv == (T)0) {
          piv = (piv < (T)0) ? -tau : tau;
          ++nboost;
          if (piv == (T)0) {
            const int64_t gcol = L.rev ? (L.start + nl - 1 - (j0 + c)) : (L.start + j0 + c);
            atomicMin(&status[1], (unsigned long long)(gcol + 1));
          }
          P[c * PLD + c] = piv;
        }
        const T rinv = (T)1 / piv;
        s_rinv = rinv;
        dinv[j0 + c] = rinv;
      }
      __syncthreads();
      const T rinv = s_rinv;
      const int rlast = min(c + k, prow - 1);
      const int nr = rlast - c;
      for (int r = c + 1 + tid; r <= rlast; r += NTHREADS) P[c * PLD + r] *= rinv;
      __syncthreads();
      const int ncl = jb - c - 1;
      for (int idx = tid; idx < nr * ncl; idx += NTHREADS) {
        const int r = c + 1 + idx % nr, cc = c + 1 + idx / nr;
        P[cc * PLD + r] -= P[c * PLD + r] * P[cc * PLD + c];
      }
      __syncthreads();
    }
    // (c) panel write-back
    for (int idx = tid; idx < NB * PLD; idx += NTHREADS) {
      const int c = idx / PLD, r = idx - c * PLD;
      if (c < jb && r < prow && r - c <= k && c - r <= k) fb[(j0 + c) * ldf + k + r - c] = P[idx];
    }
    // (d)+(e) U12 / fused Z rows, column chunks of CW
    const int kc = (int)min((int64_t)k, nl - j0 - jb);  // U12 columns and A22 rows present
    const int ntot = kc + kz;
    for (int q0 = 0; q0 < ntot; q0 += CW) {
      const int nq = min(CW, ntot - q0);
      __syncthreads();
      for (int base = tid; base < NB * nq; base += NTHREADS * 8) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int idx = base + u * NTHREADS;
          const int a = idx % NB, qq = idx / NB, q = q0 + qq;
          T w = (T)0;
          if (idx < NB * nq && a < jb) {
            if (q < kc) {
              if (jb + q - a <= k) w = fb[(j0 + jb + q) * ldf + k + a - jb - q];
            } else {
              w = Z[(int64_t)(q - kc) * nl + j0 + a];
            }
          }
          v[u] = w;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int idx = base + u * NTHREADS;
          if (idx < NB * nq) T12[(idx % NB) * TLD + idx / NB] = v[u];
        }
      }
      __syncthreads();
      // TRSM with the unit lower L11 = P[0:jb, 0:jb]: one column per thread
      for (int qq = tid; qq < nq; qq += NTHREADS) {
        T x[NB];
#pragma unroll
        for (int a = 0; a < NB; ++a) x[a] = T12[a * TLD + qq];
#pragma unroll
        for (int a = 1; a < NB; ++a) {
          T s = x[a];
#pragma unroll
          for (int b = 0; b < a; ++b) s = fma(-P[b * PLD + a], x[b], s);
          x[a] = s;
        }
#pragma unroll
        for (int a = 0; a < NB; ++a) T12[a * TLD + qq] = x[a];
      }
      __syncthreads();
      for (int idx = tid; idx < NB * nq; idx += NTHREADS) {
        const int a = idx % NB, qq = idx / NB, q = q0 + qq;
        if (a < jb) {
          if (q < kc) {
            if (jb + q - a <= k) fb[(j0 + jb + q) * ldf + k + a - jb - q] = T12[a * TLD + qq];
          } else {
            Z[(int64_t)(q - kc) * nl + j0 + a] = T12[a * TLD + qq];
          }
        }
      }
      // GEMM: window rows i in [0, kc), columns of this chunk; lanes <-> rows, 16 columns per tile
      const int RT = (kc + 31) / 32, CT = (nq + 15) / 16;
      for (int tile = warp; tile < RT * CT; tile += NTHREADS / 32) {
        const int i0 = (tile % RT) * 32, qq0 = (tile / RT) * 16;
        if (sizeof(T) == 8 && jb == NB && kc == k && (k & 31) == 0 && i0 + 32 == k) {
          // The last row tile of a full window: the multiplier of row i0 + l in panel column a is
          // zero for a < l (band edge), a triangle that lanes <-> rows would walk at full cost on
          // the FP64 pipe.  Lane (p, h) updates row i0 + p over columns a = p..31 and then row
          // i0 + 31 - p over a = 31 - p..31 (33 steps), on 8 of the tile's 16 columns.  Each entry
          // gets the same nonzero products in the same order as below.
          const int p = lane & 15, qb = qq0 + 8 * (lane >> 4);
          auto row_io = [&](int ii, T *c8, bool store) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int qq = qb + q, qabs = q0 + qq;
              if (qq < nq) {
                T *e = (qabs < kc) ? &fb[(j0 + jb + qabs) * ldf + k + ii - qabs]
                                   : &Z[(int64_t)(qabs - kc) * nl + j0 + jb + ii];
                if (store) *e = c8[q];
                else c8[q] = *e;
              } else if (!store) {
                c8[q] = (T)0;
              }
            }
          };
          T c8[8];
          row_io(i0 + p, c8, false);
          for (int v = 0; v < 33; ++v) {
            const bool first = v < 32 - p;
            if (v == 32 - p) {
              row_io(i0 + p, c8, true);
              row_io(i0 + 31 - p, c8, false);
            }
            const int row = first ? i0 + p : i0 + 31 - p;
            const int a = first ? p + v : v - 1;
            const T l = P[a * PLD + jb + row];
            const T *tr = T12 + a * TLD + qb;
#pragma unroll
            for (int q = 0; q < 8; ++q) c8[q] = fma(-l, tr[q], c8[q]);
          }
          row_io(i0 + 31 - p, c8, true);
          continue;
        }
        const int i = i0 + lane;
        const bool vi = i < kc;
        const int qa = q0 + qq0;                       // first absolute column of the tile
        const bool anyz = (q0 + min(qq0 + 16, nq) - 1) >= kc;
        int astart = anyz ? (jb + i0 - k) : (jb + max(i0, qa) - k);
        astart = max(astart, 0);
        T acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int qq = qq0 + q, qabs = q0 + qq;
          T v = (T)0;
          if (vi && qq < nq) {
            if (qabs < kc) v = fb[(j0 + jb + qabs) * ldf + k + i - qabs];
            else v = Z[(int64_t)(qabs - kc) * nl + j0 + jb + i];
          }
          acc[q] = v;
        }
        for (int a = astart; a < jb; ++a) {
          const T l = vi ? P[a * PLD + jb + i] : (T)0;
          T u[16];
          load16(T12 + a * TLD + qq0, u);
#pragma unroll
          for (int q = 0; q < 16; ++q) acc[q] = fma(-l, u[q], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int qq = qq0 + q, qabs = q0 + qq;
          if (vi && qq < nq) {
            if (qabs < kc) fb[(j0 + jb + qabs) * ldf + k + i - qabs] = acc[q];
            else Z[(int64_t)(qabs - kc) * nl + j0 + jb + i] = acc[q];
          }
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0 && nboost) atomicAdd(&status[0], nboost);
  // the leaf's spike sweeps, in the same CTA (shared memory reused)
  __syncthreads();
  sweep_run<T>(sw0, ldf, k, smem);
  __syncthreads();
  sweep_run<T>(sw1, ldf, k, smem);
}

template <typename T>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_factor_nopiv(const LeafDev *leaves, int k, int ldf, T *fb_all, T *dinv_all, T *zbuf,
                   const int64_t *zoff, const unsigned long long *amax_bits, double boost_eps,
                   unsigned long long *status, const SweepDesc *sweeps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  factor_leaf<T>(leaves[blockIdx.x], k, ldf, fb_all, dinv_all, zbuf + zoff[blockIdx.x], amax_bits, boost_eps,
                 status, sweeps[2 * blockIdx.x], sweeps[2 * blockIdx.x + 1], (T *)smem_raw);
}

// Blocks of several systems in one launch (spike_factor_batch): persistent CTAs take the tasks
// from a zeroed counter in index order (the host lists them largest first); each task is one
// block with its own system's bandwidth, storage and status words.
__global__ void __launch_bounds__(NTHREADS, 1) k_factor_tasks(const FactorTask *tasks, int ntasks, unsigned *queue,
                                                              double boost_eps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_task;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_task = (int)atomicAdd(queue, 1u);
    __syncthreads();
    const int t = s_task;
    if (t >= ntasks) break;
    const FactorTask &T = tasks[t];
    factor_leaf<double>(T.leaf, T.k, T.ldf, (double *)T.fb_all, (double *)T.dinv_all, (double *)T.Z, T.amax_bits,
                        boost_eps, T.status, T.sw[0], T.sw[1], (double *)smem_raw);
  }
}

int launch_factor_tasks(const FactorTask *tasks, int ntasks, int maxk, unsigned *queue, void *stream) {
  if (ntasks <= 0) return 0;
  size_t smem = sizeof(double) * ((size_t)NB * (NB + maxk + 1) + (size_t)NB * FACTOR_TLD<double>);
  if (smem < SWEEP_SMEM) smem = SWEEP_SMEM;
  const int e = smem_at_least((const void *)k_factor_tasks, smem);
  if (e) return e;
  const int grid = std::min(ntasks, device_sms());
  k_factor_tasks<<<grid, NTHREADS, smem, (cudaStream_t)stream>>>(tasks, ntasks, queue, 1.4901161193847656e-08);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_factor_nopiv(const LeafDev *leaves, int nleaves, int k, int ldf, void *fb, void *dinv, void *zbuf,
                        const int64_t *zoff, const unsigned long long *amax_bits, double boost_eps,
                        unsigned long long *status, const SweepDesc *sweeps, void *stream, int f32) {
  const size_t es = f32 ? sizeof(float) : sizeof(double);
  size_t smem = es * ((size_t)NB * (NB + k + 1) + (size_t)NB * (f32 ? FACTOR_TLD<float> : FACTOR_TLD<double>));
  if (smem < SWEEP_SMEM) smem = SWEEP_SMEM;
  cudaError_t e;
  if (f32) {
    e = (cudaError_t)smem_at_least((const void *)k_factor_nopiv<float>, smem);
    if (e != cudaSuccess) return (int)e;
    k_factor_nopiv<float><<<nleaves, NTHREADS, smem, (cudaStream_t)stream>>>(
        leaves, k, ldf, (float *)fb, (float *)dinv, (float *)zbuf, zoff, amax_bits, boost_eps, status, sweeps);
  } else {
    e = (cudaError_t)smem_at_least((const void *)k_factor_nopiv<double>, smem);
    if (e != cudaSuccess) return (int)e;
    k_factor_nopiv<double><<<nleaves, NTHREADS, smem, (cudaStream_t)stream>>>(
        leaves, k, ldf, (double *)fb, (double *)dinv, (double *)zbuf, zoff, amax_bits, boost_eps, status, sweeps);
  }
  count_launch();
  return (int)cudaGetLastError();
}

// ------------------------------------------------------ pivoting block LU
// Blocked banded GEPP of one leaf (Sec. 5.1), right-looking over panels of PNB columns.  The
// pivot of a column is the first entry of largest magnitude among its k + 1 band candidates;
// U fills up to kl + ku = 2k superdiagonals; the multipliers are stored as computed at their
// own step (not permuted by later interchanges: the sweeps apply the interchanges interleaved
// with the L columns); ipiv holds leaf-local rows and dinv the pivots' reciprocals (0 for an
// all-zero column, whose step then changes nothing).  The UL of the last block is this LU of
// Q A Q (Sec. 5.2), stored in the reversed local frame.  Per panel j0 .. j0 + jb - 1:
//  (a) the panel's rows j0 .. j0 + jb + k - 1 (all candidate rows of its columns) are loaded
//      into shared memory;
//  (b) panel GEPP in shared memory: per column, warp 0 picks the pivot (first row of largest
//      magnitude) and interchanges the two rows across the whole panel (earlier columns too,
//      so that L11 and L21 are the permuted factors of a block LU); all threads then update
//      the panel's later columns and write this column's multipliers to the leaf storage;
//  (c) the panel's L columns are scaled and its U rows written back;
//  (d) the trailing columns j0 + jb .. j0 + jb + 2k - 1 (the reach of the U fill), in chunks
//      of cw columns: the window rows are gathered through the panel's row permutation,
//      U12 = L11^{-1} A12 (one column per thread), A22 -= L21 U12 (register tiles), stored.
// In exact arithmetic this performs the eliminations of the unblocked algorithm; entries of a
// row beyond its fill reach are zero, so gathering them through the permutation changes nothing.
constexpr int PNB = 32;
constexpr size_t PIV_SMEM_MAX = 220 * 1024;  // dynamic shared memory budget of the kernel (a CTA may use 227 KB)

__device__ void factor_piv_leaf(const LeafDev &L, int k, int ldf, double *fb_all, double *dinv_all, int *ipiv_all,
                                unsigned long long *status, int cw, double *smem) {
  const int PLD = PNB + k + 1;  // panel: PNB columns x PLD rows, column-major
  const int TLD = cw + 1;       // trailing chunk: PNB + k rows x TLD, row-major
  double *P = smem;
  double *Wt = P + (size_t)PNB * PLD;
  int *perm = (int *)(Wt + (size_t)(PNB + k) * TLD);
  __shared__ double s_rinv[PNB];
  const int nl = (int)L.len;
  double *fb = fb_all + L.start * (int64_t)ldf;
  double *dinv = dinv_all + L.start;
  int *ipiv = ipiv_all + L.start;
  const int dofs = 2 * k;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // leaf-local (r, c) -> storage index; stored entries have -2k <= r - c <= k
  auto at = [&](int r, int c) -> int64_t { return (int64_t)c * ldf + dofs + r - c; };
  auto stored = [&](int r, int c) { return r - c <= k && c - r <= dofs; };
  for (int j0 = 0; j0 < nl; j0 += PNB) {
    const int jb = min(PNB, nl - j0);
    const int prow = min(jb + k, nl - j0);
    // (a)
    for (int idx = tid; idx < PNB * PLD; idx += NTHREADS) {
      const int c = idx / PLD, r = idx - c * PLD;
      P[idx] = (c < jb && r < prow && stored(r, c)) ? fb[at(j0 + r, j0 + c)] : 0.0;
    }
    for (int r = tid; r < prow; r += NTHREADS) perm[r] = r;
    __syncthreads();
    // (b)
    for (int c = 0; c < jb; ++c) {
      const int dl = min(c + k, prow - 1);
      if (warp == 0) {
        double best = -1.0;
        int bd = c;
        for (int r = c + lane; r <= dl; r += 32) {
          const double v = fabs(P[c * PLD + r]);
          if (v > best) {
            best = v;
            bd = r;
          }
        }
        for (int o = 16; o; o >>= 1) {
          const double ov = __shfl_xor_sync(FULLMASK, best, o);
          const int od = __shfl_xor_sync(FULLMASK, bd, o);
          if (ov > best || (ov == best && od < bd)) {
            best = ov;
            bd = od;
          }
        }
        const bool zero = !(best > 0.0);
        if (bd != c) {
          for (int cc = lane; cc < jb; cc += 32) {
            const double t = P[cc * PLD + c];
            P[cc * PLD + c] = P[cc * PLD + bd];
            P[cc * PLD + bd] = t;
          }
        }
        __syncwarp();
        if (lane == 0) {
          if (bd != c) {
            const int t = perm[c];
            perm[c] = perm[bd];
            perm[bd] = t;
          }
          ipiv[j0 + c] = j0 + bd;
          if (zero) {
            const int64_t gcol = L.rev ? (L.start + nl - 1 - (j0 + c)) : (L.start + j0 + c);
            atomicMin(&status[1], (unsigned long long)(gcol + 1));
            if (isnan(best)) atomicOr(&status[2], 1ull);
          }
          const double ri = zero ? 0.0 : 1.0 / P[c * PLD + c];
          s_rinv[c] = ri;
          dinv[j0 + c] = ri;
        }
      }
      __syncthreads();
      // column c stays unscaled in P until (c); q = 0 writes the multiplier, q > 0 updates column c + q
      const double rinv = s_rinv[c];
      const int nr = dl - c, ncl = jb - c;
      for (int idx = tid; idx < nr * ncl; idx += NTHREADS) {
        const int q = idx / nr, r = c + 1 + (idx - q * nr);
        const double l = P[c * PLD + r] * rinv;
        if (q == 0) {
          fb[at(j0 + r, j0 + c)] = l;
        } else {
          double *pc = P + (c + q) * PLD;
          pc[r] = fma(-l, pc[c], pc[r]);
        }
      }
      __syncthreads();
    }
    // (c)
    for (int idx = tid; idx < jb * PLD; idx += NTHREADS) {
      const int c = idx / PLD, r = idx - c * PLD;
      if (r < prow) {
        if (r > c) P[idx] *= s_rinv[c];
        else if (c - r <= dofs) fb[at(j0 + r, j0 + c)] = P[idx];
      }
    }
    __syncthreads();
    // (d)
    const int nt = min(dofs, nl - j0 - jb);
    for (int q0 = 0; q0 < nt; q0 += cw) {
      const int nq = min(cw, nt - q0);
      for (int base = tid; base < prow * nq; base += NTHREADS * 8) {  // 8 loads in flight per thread
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int idx = base + u * NTHREADS;
          const int qq = idx / prow, r = idx - qq * prow;
          const int sr = (idx < prow * nq) ? perm[r] : 0, c = jb + q0 + qq;
          v[u] = (idx < prow * nq && stored(sr, c)) ? fb[at(j0 + sr, j0 + c)] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int idx = base + u * NTHREADS;
          if (idx < prow * nq) Wt[(idx % prow) * TLD + idx / prow] = v[u];
        }
      }
      __syncthreads();
      for (int qq = tid; qq < nq; qq += NTHREADS) {
        double x[PNB];
#pragma unroll
        for (int a = 0; a < PNB; ++a) x[a] = (a < jb) ? Wt[a * TLD + qq] : 0.0;
#pragma unroll
        for (int b = 0; b < PNB - 1; ++b) {
          const double xb = x[b];
#pragma unroll
          for (int a = b + 1; a < PNB; ++a) x[a] = fma(-P[b * PLD + a], xb, x[a]);
        }
#pragma unroll
        for (int a = 0; a < PNB; ++a)
          if (a < jb) Wt[a * TLD + qq] = x[a];
      }
      __syncthreads();
      const int nrr = prow - jb;
      const int RT = (nrr + 31) / 32, CT = (nq + 15) / 16;
      for (int tile = warp; tile < RT * CT; tile += NTHREADS / 32) {
        const int i0 = (tile % RT) * 32, qq0 = (tile / RT) * 16;
        const int i = i0 + lane;
        const bool vi = i < nrr;
        // U12 row a is zero beyond column a + 2k (relative to j0): rows a < q + jb - 2k vanish
        const int astart = max(0, q0 + qq0 + jb - dofs);
        double acc[16];
        double *wrow = Wt + (size_t)(jb + (vi ? i : 0)) * TLD + qq0;
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = (vi && qq0 + q < nq) ? wrow[q] : 0.0;
        for (int a = astart; a < jb; ++a) {
          const double l = vi ? P[a * PLD + jb + i] : 0.0;
          const double *trow = Wt + (size_t)a * TLD + qq0;
#pragma unroll
          for (int q = 0; q < 16; ++q) acc[q] = fma(-l, trow[q], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q)
          if (vi && qq0 + q < nq) wrow[q] = acc[q];
      }
      __syncthreads();
      for (int idx = tid; idx < prow * nq; idx += NTHREADS) {
        const int qq = idx / prow, r = idx - qq * prow;
        const int c = jb + q0 + qq;
        if (stored(r, c)) fb[at(j0 + r, j0 + c)] = Wt[r * TLD + qq];
      }
      __syncthreads();
    }
  }
}

// The same block GEPP with look-ahead, for bandwidths whose two panel buffers fit in shared
// memory.  The panel factorization is a chain of small dependent steps and the trailing update
// is throughput-bound FP64 work, so they overlap: with panel i factored,
//  (T1) all warps update the columns of panel i+1 by panel i (interchanges, U12 by a warp-wide
//       triangular solve, A22 -= L21 U12) and build panel i+1 in the other buffer (its top k rows
//       are the updated A22 rows, the rest come from the leaf storage);
//  (T2) warp 0 factors panel i+1 (lanes over rows for the updates, over columns for the
//       interchanges, no CTA barrier) while warps 1..7 update the remaining trailing columns of
//       panel i (up to column j0 + jb + 2k), synchronised by a named barrier among themselves.
// Panel i+1 reads only its own columns, which T1 completed; T2's two parts write disjoint
// columns.  Results are those of factor_piv_leaf up to the summation order of the updates.
__device__ __forceinline__ void bar_rest() { asm volatile("bar.sync 1, %0;" ::"n"(NTHREADS - 32) : "memory"); }

__device__ void factor_piv_leaf_la(const LeafDev &L, int k, int ldf, double *fb_all, double *dinv_all,
                                   int *ipiv_all, unsigned long long *status, int cw, double *smem) {
  const int PLD = PNB + k + 1;  // panels: PNB columns x PLD rows, column-major (two buffers)
  const int TLD = cw + 1;       // trailing chunk: PNB + k rows x TLD, row-major
  double *Pbuf0 = smem;
  double *Pbuf1 = smem + (size_t)PNB * PLD;
  double *Wt = smem + (size_t)2 * PNB * PLD;
  int *perm0 = (int *)(Wt + (size_t)(PNB + k) * TLD);
  int *perm1 = perm0 + (PNB + k);
  const int nl = (int)L.len;
  double *fb = fb_all + L.start * (int64_t)ldf;
  double *dinv = dinv_all + L.start;
  int *ipiv = ipiv_all + L.start;
  const int dofs = 2 * k;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  auto at = [&](int r, int c) -> int64_t { return (int64_t)c * ldf + dofs + r - c; };
  auto stored = [&](int r, int c) { return r - c <= k && c - r <= dofs; };

  // GEPP of the panel in P (rows [0, prow) of the window at j0, jb columns) by warp 0
  auto panel = [&](double *P, int *perm, int j0, int jb, int prow) {
    for (int c = 0; c < jb; ++c) {
      const int dl = min(c + k, prow - 1);
      double best = -1.0;
      int bd = c;
      for (int r = c + lane; r <= dl; r += 32) {
        const double v = fabs(P[c * PLD + r]);
        if (v > best) {
          best = v;
          bd = r;
        }
      }
      for (int o = 16; o; o >>= 1) {
        const double ov = __shfl_xor_sync(FULLMASK, best, o);
        const int od = __shfl_xor_sync(FULLMASK, bd, o);
        if (ov > best || (ov == best && od < bd)) {
          best = ov;
          bd = od;
        }
      }
      const bool zero = !(best > 0.0);
      if (bd != c) {
        for (int cc = lane; cc < jb; cc += 32) {
          const double t = P[cc * PLD + c];
          P[cc * PLD + c] = P[cc * PLD + bd];
          P[cc * PLD + bd] = t;
        }
      }
      if (lane == 0) {
        if (bd != c) {
          const int t = perm[c];
          perm[c] = perm[bd];
          perm[bd] = t;
        }
        ipiv[j0 + c] = j0 + bd;
        if (zero) {
          const int64_t gcol = L.rev ? (L.start + nl - 1 - (j0 + c)) : (L.start + j0 + c);
          atomicMin(&status[1], (unsigned long long)(gcol + 1));
          if (isnan(best)) atomicOr(&status[2], 1ull);
        }
      }
      __syncwarp();
      const double rinv = zero ? 0.0 : 1.0 / P[c * PLD + c];
      if (lane == 0) dinv[j0 + c] = rinv;
      for (int r = c + 1 + lane; r <= dl; r += 32) {
        const double l = P[c * PLD + r] * rinv;
        P[c * PLD + r] = l;
        fb[at(j0 + r, j0 + c)] = l;
        for (int cc = c + 1; cc < jb; ++cc) P[cc * PLD + r] = fma(-l, P[cc * PLD + c], P[cc * PLD + r]);
      }
      __syncwarp();
    }
    for (int idx = lane; idx < jb * PNB; idx += 32) {
      const int c = idx / PNB, r = idx - c * PNB;
      if (r <= c && c - r <= dofs) fb[at(j0 + r, j0 + c)] = P[c * PLD + r];
    }
  };
  // gather rows [0, prow) of columns [jb + q0, jb + q0 + nq) (relative to j0) through perm into Wt,
  // by the threads t0 + (0 .. nth-1); 8 loads in flight per thread
  auto gather = [&](const int *perm, int j0, int jb, int prow, int q0, int nq, int t0, int nth) {
    const int tot = prow * nq;
    for (int base = t0; base < tot; base += nth * 8) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = base + u * nth;
        const int qq = idx / prow, r = idx - qq * prow;
        const int sr = (idx < tot) ? perm[r] : 0, c = jb + q0 + qq;
        v[u] = (idx < tot && stored(sr, c)) ? fb[at(j0 + sr, j0 + c)] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = base + u * nth;
        if (idx < tot) {
          const int qq = idx / prow, r = idx - qq * prow;
          Wt[r * TLD + qq] = v[u];
        }
      }
    }
  };
  // U12 = L11^{-1} A12 on Wt column qq by one warp (lanes <-> rows), for up to 4 columns at once
  auto trsm_warp = [&](const double *P, int jb, const int *cols, int ncol) {
    double x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = (u < ncol && lane < jb) ? Wt[lane * TLD + cols[u]] : 0.0;
    for (int b = 0; b + 1 < jb; ++b) {
      const double lb = (lane > b) ? P[b * PLD + lane] : 0.0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double xb = __shfl_sync(FULLMASK, x[u], b);
        if (lane > b) x[u] = fma(-lb, xb, x[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (u < ncol && lane < jb) Wt[lane * TLD + cols[u]] = x[u];
  };
  // U12 = L11^{-1} A12 on Wt column qq by one thread
  auto trsm_thread = [&](const double *P, int jb, int qq) {
    double x[PNB];
#pragma unroll
    for (int a = 0; a < PNB; ++a) x[a] = (a < jb) ? Wt[a * TLD + qq] : 0.0;
#pragma unroll
    for (int b = 0; b < PNB - 1; ++b) {
      const double xb = x[b];
#pragma unroll
      for (int a = b + 1; a < PNB; ++a) x[a] = fma(-P[b * PLD + a], xb, x[a]);
    }
#pragma unroll
    for (int a = 0; a < PNB; ++a)
      if (a < jb) Wt[a * TLD + qq] = x[a];
  };
  // A22 -= L21 U12 on one tile of 32 rows x C columns of Wt (rows jb + i0.., columns qq0..);
  // with dst the results go to the next panel (column-major, row i), else back to Wt
  auto gemm_tile = [&](const double *P, int jb, int nrr, int nq, int i0, int qq0, int astart, double *dst, auto cn) {
    constexpr int C = decltype(cn)::value;
    const int i = i0 + lane;
    const bool vi = i < nrr;
    double acc[C];
    double *wrow = Wt + (size_t)(jb + (vi ? i : 0)) * TLD + qq0;
#pragma unroll
    for (int q = 0; q < C; ++q) acc[q] = (vi && qq0 + q < nq) ? wrow[q] : 0.0;
    for (int a = astart; a < jb; ++a) {
      const double l = vi ? P[a * PLD + jb + i] : 0.0;
      const double *trow = Wt + (size_t)a * TLD + qq0;
#pragma unroll
      for (int q = 0; q < C; ++q) acc[q] = fma(-l, trow[q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < C; ++q)
      if (vi && qq0 + q < nq) {
        if (dst) dst[(qq0 + q) * PLD + i] = acc[q];
        else wrow[q] = acc[q];
      }
  };

  // panel 0
  {
    const int jb = min(PNB, nl), prow = min(jb + k, nl);
    for (int idx = tid; idx < PNB * PLD; idx += NTHREADS) {
      const int c = idx / PLD, r = idx - c * PLD;
      Pbuf0[idx] = (c < jb && r < prow && stored(r, c)) ? fb[at(r, c)] : 0.0;
    }
    for (int r = tid; r < prow; r += NTHREADS) perm0[r] = r;
    __syncthreads();
    if (warp == 0) panel(Pbuf0, perm0, 0, jb, prow);
    __syncthreads();
  }
  double *P = Pbuf0, *Pn = Pbuf1;
  int *perm = perm0, *permn = perm1;
  for (int j0 = 0; j0 < nl; j0 += PNB) {
    const int jb = min(PNB, nl - j0), prow = min(jb + k, nl - j0);
    const int nrr = prow - jb;
    const int nt = min(dofs, nl - j0 - jb);  // trailing columns reached by this panel
    const int j1 = j0 + jb;
    const int jb1 = max(0, min(PNB, nl - j1)), prow1 = max(0, min(jb1 + k, nl - j1));
    const int la = min(jb1, nt);  // columns of the next panel that this one updates
    // (T1)
    if (la > 0) {
      gather(perm, j0, jb, prow, 0, la, tid, NTHREADS);
      __syncthreads();
      {
        int cols[4], ncol = 0;
        for (int qq = warp; qq < la && ncol < 4; qq += NTHREADS / 32) cols[ncol++] = qq;
        if (ncol > 0) trsm_warp(P, jb, cols, ncol);
      }
      __syncthreads();
      const int RT = (nrr + 31) / 32, CT = (la + 7) / 8;
      for (int tile = warp; tile < RT * CT; tile += NTHREADS / 32) {
        const int i0 = (tile % RT) * 32, qq0 = (tile / RT) * 8;
        gemm_tile(P, jb, nrr, la, i0, qq0, max(0, qq0 + jb - dofs), Pn, std::integral_constant<int, 8>());
      }
      // U12 rows to the storage; the rest of the next panel from the storage
      for (int idx = tid; idx < jb * la; idx += NTHREADS) {
        const int qq = idx / jb, r = idx - qq * jb;
        if (stored(r, jb + qq)) fb[at(j0 + r, j1 + qq)] = Wt[r * TLD + qq];
      }
      for (int base = tid; base < PNB * PLD; base += NTHREADS * 4) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int idx = base + u * NTHREADS;
          const int c = idx / PLD, r = idx - c * PLD;
          v[u] = (idx < PNB * PLD && c < jb1 && r < prow1 && stored(r, c) && !(c < la && r < nrr))
                     ? fb[at(j1 + r, j1 + c)]
                     : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int idx = base + u * NTHREADS;
          const int c = idx / PLD, r = idx - c * PLD;
          if (idx < PNB * PLD && !(c < la && r < nrr)) Pn[idx] = v[u];
        }
      }
      for (int r = tid; r < prow1; r += NTHREADS) permn[r] = r;
      __syncthreads();
    } else if (jb1 > 0) {  // the next panel lies beyond this one's reach (2k < PNB)
      for (int idx = tid; idx < PNB * PLD; idx += NTHREADS) {
        const int c = idx / PLD, r = idx - c * PLD;
        Pn[idx] = (c < jb1 && r < prow1 && stored(r, c)) ? fb[at(j1 + r, j1 + c)] : 0.0;
      }
      for (int r = tid; r < prow1; r += NTHREADS) permn[r] = r;
      __syncthreads();
    }
    // (T2)
    if (warp == 0) {
      if (jb1 > 0) panel(Pn, permn, j1, jb1, prow1);
    } else {
      const int t2 = tid - 32, nw = NTHREADS / 32 - 1;
      for (int q0 = la; q0 < nt; q0 += cw) {
        const int nq = min(cw, nt - q0);
        gather(perm, j0, jb, prow, q0, nq, t2, NTHREADS - 32);
        bar_rest();
        if (nq >= 64) {
          for (int qq = t2; qq < nq; qq += NTHREADS - 32) trsm_thread(P, jb, qq);
        } else {
          int cols[4], ncol = 0;
          for (int qq = warp - 1; qq < nq && ncol < 4; qq += nw) cols[ncol++] = qq;
          if (ncol > 0) trsm_warp(P, jb, cols, ncol);
          for (int qq0 = warp - 1 + 4 * nw; qq0 < nq; qq0 += 4 * nw) {
            ncol = 0;
            for (int qq = qq0; qq < nq && ncol < 4; qq += nw) cols[ncol++] = qq;
            trsm_warp(P, jb, cols, ncol);
          }
        }
        bar_rest();
        const int RT = (nrr + 31) / 32, CT = (nq + 15) / 16;
        for (int tile = warp - 1; tile < RT * CT; tile += nw) {
          const int i0 = (tile % RT) * 32, qq0 = (tile / RT) * 16;
          gemm_tile(P, jb, nrr, nq, i0, qq0, max(0, q0 + qq0 + jb - dofs), nullptr,
                    std::integral_constant<int, 16>());
        }
        bar_rest();
        for (int idx = t2; idx < prow * nq; idx += NTHREADS - 32) {
          const int qq = idx / prow, r = idx - qq * prow;
          const int c = jb + q0 + qq;
          if (stored(r, c)) fb[at(j0 + r, j0 + c)] = Wt[r * TLD + qq];
        }
        bar_rest();
      }
    }
    __syncthreads();
    double *tp = P;
    P = Pn;
    Pn = tp;
    int *tq = perm;
    perm = permn;
    permn = tq;
  }
}

template <int KIND>
__device__ void piv_sweep_run(const SweepDesc &D, int k, int ldf, int dofs, double *pwin);

// One block per CTA: its GEPP, then its spike sweeps (Sec. 2.3 with the pivoted factors of
// Sec. 5.1), so a block's whole factor stage is one CTA's work, as for the non-pivoting LU:
// sweeps[3 b] and sweeps[3 b + 1] are pivoted L sweeps (the top spike's full sweep and the
// bottom spike's truncated one), sweeps[3 b + 2] the U sweep over both spikes.  lookahead
// selects factor_piv_leaf_la (two panel buffers) over factor_piv_leaf.
__global__ void __launch_bounds__(NTHREADS, 1)
    k_factor_piv(const LeafDev *leaves, int k, int ldf, double *fb_all, double *dinv_all, int *ipiv_all,
                 unsigned long long *status, int cw, int lookahead, const SweepDesc *sweeps) {
  extern __shared__ __align__(16) unsigned char pb_raw[];
  double *smem = (double *)pb_raw;
  const LeafDev L = leaves[blockIdx.x];
  if (lookahead) factor_piv_leaf_la(L, k, ldf, fb_all, dinv_all, ipiv_all, status, cw, smem);
  else factor_piv_leaf(L, k, ldf, fb_all, dinv_all, ipiv_all, status, cw, smem);
  const int dofs = 2 * k;
  const SweepDesc *sw = sweeps + 3 * (int64_t)blockIdx.x;
  __syncthreads();
  piv_sweep_run<LN>(sw[0], k, ldf, dofs, smem);
  __syncthreads();
  piv_sweep_run<LN>(sw[1], k, ldf, dofs, smem);
  __syncthreads();
  sweep_run<double>(sw[2], ldf, dofs, smem);
}

// Shared memory of the block GEPP (one or two panel buffers) for trailing chunk width cw.
static size_t piv_blk_smem(int k, int cw, int npanel) {
  return sizeof(double) * ((size_t)npanel * PNB * (PNB + k + 1) + (size_t)(PNB + k) * (cw + 1)) +
         sizeof(int) * (size_t)npanel * (PNB + k);
}

int launch_factor_piv(const LeafDev *leaves, int nleaves, int k, int ldf, double *fb, double *dinv, int *ipiv,
                      unsigned long long *status, const SweepDesc *sweeps, void *stream) {
  const size_t swp = std::max(SWEEP_SMEM, sizeof(double) * (size_t)(NTHREADS / 32) * (k + 2));
  // look-ahead when two panel buffers and a trailing chunk of at least PNB columns (the next
  // panel's, staged in the same array) fit; the chunk is as wide as the columns left after the
  // next panel's (at most 128, a multiple of 16)
  for (int la = 1; la >= 0; --la) {
    const int want = la ? 2 * k - PNB : 2 * k;
    const int cwmin = la ? PNB : 16;
    const int cwmax = std::max(cwmin, std::min(128, (want + 15) / 16 * 16));
    for (int cw = cwmax; cw >= cwmin; cw -= 16) {
      const size_t smem = std::max(piv_blk_smem(k, cw, la ? 2 : 1), swp);
      if (smem > PIV_SMEM_MAX) continue;
      const int e = smem_at_least((const void *)k_factor_piv, smem);
      if (e) return e;
      k_factor_piv<<<nleaves, NTHREADS, smem, (cudaStream_t)stream>>>(leaves, k, ldf, fb, dinv, ipiv, status, cw,
                                                                      la, sweeps);
      count_launch();
      return (int)cudaGetLastError();
    }
  }
  return SPIKE_ENOTSUP;
}

// ------------------------------------------------------ blocked sweep engine
// X = T^{-1} G over rows [r0, r1) of one leaf, T one of LN/UN/UT/LT (see internal.h).
// Rows are processed in blocks of NB in sweep order; per block:
//   (1) acc = G(block) - T(block, window) X(window)   (GEMM over the kw window rows,
//       lanes <-> block rows, warps <-> column groups, inner dimension split when
//       there are few columns),
//   (2) in-block triangular solve (lanes <-> columns when there are many columns,
//       lanes <-> rows with shuffles otherwise),
//   (3) store.
// Coefficients: LN/UN use column c of the band, UT/LT column r (transposed access).
template <typename T>
__device__ __forceinline__ T coef(int kind, const T *fb, int ldf, int dofs, int64_t r, int64_t c) {
  if (kind == LN || kind == UN) return fb[c * ldf + dofs + r - c];
  return fb[r * ldf + dofs + c - r];
}

template <typename T>
__device__ __forceinline__ const T *coef_ptr(int kind, const T *fb, int ldf, int dofs, int64_t r, int64_t c) {
  if (kind == LN || kind == UN) return fb + (c * ldf + dofs + r - c);
  return fb + (r * ldf + dofs + c - r);
}

// Asynchronous copy of one element global -> shared (cp.async); with valid == false nothing
// is read and the element is zero-filled.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? (int)sizeof(T) : 0;
  if (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// acc[q] += sum_j Tw[j*NB] * X(row_j, col_base + q), rows row_j = row_0 + j (stride xstep),
// for q < C.  Columns past `lastc` are clamped (their accumulators are never stored).
template <typename T, int C>
__device__ __forceinline__ void window_fma(T *acc, const T *tw, const T *xrow, int64_t xstep, int64_t xcs,
                                           int col_base, int lastc, int count) {
  // Row-major X with this warp's C columns contiguous and 16-byte aligned: one 16-byte load per
  // 16 / sizeof(T) columns (the same FMAs in the same order as the element-wise loop below).
  constexpr int V = 16 / (int)sizeof(T);
  constexpr int NV = (C >= V) ? C / V : 1;
  if (C >= V && C % V == 0 && xcs == 1 && col_base + C - 1 <= lastc && xstep % V == 0 &&
      ((uintptr_t)(xrow + col_base) & 15) == 0) {
    using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    const VT *xv = reinterpret_cast<const VT *>(xrow + col_base);
    const int64_t vstep = xstep / V;
    for (int j = 0; j < count; ++j) {
      const T t = tw[j * NB];
      VT x[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) x[v] = xv[v];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T *e = reinterpret_cast<const T *>(&x[v]);
#pragma unroll
        for (int u = 0; u < V; ++u) acc[v * V + u] = fma(t, e[u], acc[v * V + u]);
      }
      xv += vstep;
    }
    return;
  }
  int64_t coff[C];
#pragma unroll
  for (int q = 0; q < C; ++q) coff[q] = (int64_t)min(col_base + q, lastc) * xcs;
  for (int j = 0; j < count; ++j) {
    const T t = tw[j * NB];
#pragma unroll
    for (int q = 0; q < C; ++q) acc[q] = fma(t, xrow[coff[q]], acc[q]);
    xrow += xstep;
  }
}

// The 32 window rows of a full window that form a triangle with the block (forward sweeps: window
// rows [0, 32), block row a couples to window row j only for j >= a; backward: rows [kw - 32, kw),
// only for j - (kw - 32) <= 31 - a).  Walked with lanes <-> block rows, half the products there are
// zeros, and on the FP64 pipe a predicated-off or zero product costs as much as a useful one.  Here
// lane l (p = l mod 16, half h = l / 16) walks block rows p and 31 - p, the 32 - p window rows of
// the first and then the p + 1 of the second (33 steps in all), over the h-th half of this warp's
// C columns; the sums then go by shuffles to the lanes that own those rows and are added to acc.
// Each row's products are summed in window order.
template <typename T, int C>
__device__ __forceinline__ void window_tri(T *acc, const T *tw0, const T *x0, int64_t xstep, int64_t xcs,
                                           int col_base, int lastc, bool fwd) {
  constexpr int H = C / 2;
  const int lane = threadIdx.x & 31, p = lane & 15, h = lane >> 4;
  int64_t coff[H];
#pragma unroll
  for (int q = 0; q < H; ++q) coff[q] = (int64_t)min(col_base + h * H + q, lastc) * xcs;
  T cur[H], sav[H];
#pragma unroll
  for (int q = 0; q < H; ++q) {
    cur[q] = (T)0;
    sav[q] = (T)0;
  }
  for (int v = 0; v < 33; ++v) {
    const bool first = v < 32 - p;
    if (v == 32 - p) {
#pragma unroll
      for (int q = 0; q < H; ++q) {
        sav[q] = cur[q];
        cur[q] = (T)0;
      }
    }
    const int row = first ? p : 31 - p;
    const int jj = fwd ? (first ? p + v : v - 1) : (first ? v : v - (32 - p));
    const T t = tw0[jj * NB + row];
    const T *xr = x0 + jj * xstep;
#pragma unroll
    for (int q = 0; q < H; ++q) cur[q] = fma(t, xr[coff[q]], cur[q]);
  }
  // row r < 16: sav of lanes r (first half of the columns) and r + 16 (second half);
  // row r >= 16: cur of lanes 31 - r and 47 - r
  const int s0 = (lane < 16) ? lane : 31 - lane, s1 = s0 + 16;
#pragma unroll
  for (int q = 0; q < H; ++q) {
    const T a0 = __shfl_sync(FULLMASK, sav[q], s0), a1 = __shfl_sync(FULLMASK, cur[q], s0);
    const T b0 = __shfl_sync(FULLMASK, sav[q], s1), b1 = __shfl_sync(FULLMASK, cur[q], s1);
    acc[q] += (lane < 16) ? a0 : a1;
    acc[H + q] += (lane < 16) ? b0 : b1;
  }
}

template <typename T>
__device__ void sweep_run(const SweepDesc &D, int ldf, int dofs, T *sm) {
  if (D.ncols <= 0 || D.r1 <= D.r0) return;
  ldf = D.ldf;  // the descriptor carries its leaf's storage (several systems may share a launch)
  dofs = D.dofs;
  // descriptor pointers carry the leaf's storage type T
  const T *dfb = (const T *)D.fb;
  const T *ddinv = (const T *)D.dinv;
  const T *dga = (const T *)D.ga;
  const T *dgb = (const T *)D.gb;
  T *dx = (T *)D.x;
  const T gbs = (T)D.gb_scale;
  const int kind = D.kind, kw = D.kw;
  const bool FWD = (kind == LN || kind == UT);
  const bool UNIT = (kind == LN || kind == LT);
  const int GLD = SCW + 1;
  // per buffer: WCH x NB Tw[j*NB + a] = T(row(a), wrow(j)); NB x NB Td[a'*NB + a] = T(row(a), row(a'));
  // NB reciprocals (1 for unit triangles)
  constexpr int BUF = WCH * NB + NB * NB + NB;
  T *Gs = sm + 2 * BUF;       // NB x GLD
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = NTHREADS / 32;
  // When a block's window fits one staged chunk (kw <= WCH), the coefficients of block
  // bk+1 are copied asynchronously into the other buffer while block bk computes (they
  // are factor entries, independent of the results).
  const bool pre = kw <= WCH;
  const int nblk = (D.r1 - D.r0 + NB - 1) / NB;
  auto geom = [&](int bk, int64_t &b0, int64_t &b1, int &nbk, int &jlo, int &jhi) {
    if (FWD) {
      b0 = D.r0 + (int64_t)bk * NB;
      nbk = (int)min((int64_t)NB, D.r1 - b0);
      b1 = 0;
      jlo = (int)max((int64_t)0, D.r0 - (b0 - kw));
      jhi = kw;
    } else {
      b1 = D.r1 - (int64_t)bk * NB;
      nbk = (int)min((int64_t)NB, b1 - D.r0);
      b0 = 0;
      jlo = 0;
      jhi = (int)min((int64_t)kw, D.r1 - b1);
    }
  };
  auto stage_async = [&](int bk, int buf) {
    int64_t b0, b1;
    int nbk, jlo, jhi;
    geom(bk, b0, b1, nbk, jlo, jhi);
    auto row = [&](int a) -> int64_t { return FWD ? (b0 + a) : (b1 - 1 - a); };
    auto wrow = [&](int j) -> int64_t { return FWD ? (b0 - kw + j) : (b1 + j); };
    T *Twb = sm + buf * BUF, *Tdb = Twb + WCH * NB, *dsb = Tdb + NB * NB;
    for (int idx = tid; idx < NB * NB; idx += NTHREADS) {
      const int ap = idx / NB, a = idx - ap * NB;
      const bool v = ap < a && a < nbk && a - ap <= kw;
      cp_async_elem(Tdb + idx, v ? coef_ptr<T>(kind, dfb, ldf, dofs, row(a), row(ap)) : dfb, v);
    }
    for (int a = tid; a < NB; a += NTHREADS) {
      if (UNIT) dsb[a] = (a < nbk) ? (T)1 : (T)0;
      else cp_async_elem(dsb + a, a < nbk ? ddinv + row(a) : ddinv, a < nbk);
    }
    const int tot = (jhi - jlo) * NB;
    for (int idx = tid; idx < tot; idx += NTHREADS) {
      const int jj = idx / NB, a = idx - jj * NB, j = jlo + jj;
      const bool v = a < nbk && (FWD ? (j >= a) : (j <= kw - 1 - a));
      cp_async_elem(Twb + idx, v ? coef_ptr<T>(kind, dfb, ldf, dofs, row(a), wrow(j)) : dfb, v);
    }
    cp_async_commit();
  };

  for (int c0 = 0; c0 < D.ncols; c0 += SCW) {
    const int cw = min(SCW, D.ncols - c0);
    const bool fixed = D.fixed_split != 0;
    // Column split.  Default: with few columns (cw < nwarps) the window rows are split
    // over nsplit = nwarps / cw warp groups and the partial sums are combined at the
    // end, so the rounding of a column depends on how many columns share the pass.
    // fixed_split (batch-invariant): every staged window chunk is cut into WSPLIT fixed
    // sub-ranges whose products are subtracted from G one at a time in ascending order;
    // with few columns warp w owns sub-range w for all columns, otherwise a warp owns a
    // column group and walks the sub-ranges itself.  Each column then sees the same
    // sequence of roundings whatever the other right-hand sides of the pass.
    int nsplit, cpw, col_base, split;
    bool by_split;
    if (fixed) {
      by_split = cw < nwarps;
      nsplit = WSPLIT;
      cpw = by_split ? cw : (cw + nwarps - 1) / nwarps;
      col_base = by_split ? c0 : c0 + warp * cpw;
      split = by_split ? warp : 0;
    } else {
      nsplit = (cw < nwarps) ? (nwarps / cw) : 1;
      const int groups = nwarps / nsplit;
      cpw = (cw + groups - 1) / groups;
      const int grp = warp % groups;
      split = warp / groups;
      col_base = c0 + grp * cpw;
      by_split = false;
    }
    const int lastc = c0 + cw - 1;
    const bool owns = col_base <= lastc;
    if (pre) {
      __syncthreads();  // the buffers may still be read by the previous pass / sweep
      stage_async(0, 0);
    }
    for (int bk = 0; bk < nblk; ++bk) {
      int64_t b0, b1;
      int nbk, jlo, jhi;
      geom(bk, b0, b1, nbk, jlo, jhi);
      auto row = [&](int a) -> int64_t { return FWD ? (b0 + a) : (b1 - 1 - a); };
      auto wrow = [&](int j) -> int64_t { return FWD ? (b0 - kw + j) : (b1 + j); };
      const int buf = pre ? (bk & 1) : 0;
      T *Tw = sm + buf * BUF, *Td = Tw + WCH * NB, *dsm = Td + NB * NB;
      if (pre) {
        cp_async_wait_all();
        __syncthreads();  // this block's coefficients are in; the other buffer is free
        if (bk + 1 < nblk) stage_async(bk + 1, buf ^ 1);
      } else {
        __syncthreads();
        T v[NB * NB / NTHREADS];
#pragma unroll
        for (int u = 0; u < NB * NB / NTHREADS; ++u) {
          const int idx = tid + u * NTHREADS;
          const int ap = idx / NB, a = idx - ap * NB;
          v[u] = (ap < a && a < nbk && a - ap <= kw) ? coef<T>(kind, dfb, ldf, dofs, row(a), row(ap)) : (T)0;
        }
#pragma unroll
        for (int u = 0; u < NB * NB / NTHREADS; ++u) Td[tid + u * NTHREADS] = v[u];
        for (int a = tid; a < NB; a += NTHREADS) dsm[a] = (a < nbk) ? (UNIT ? (T)1 : ddinv[row(a)]) : (T)0;
      }
      if (fixed) {  // G block first (rows past the block end are zero)
        for (int idx = tid; idx < NB * cw; idx += NTHREADS) {
          const int a = idx % NB, cc = idx / NB, col = c0 + cc;
          T g = (T)0;
          if (a < nbk) {
            const int64_t r = row(a);
            g = dga[r * D.ga_rs + (int64_t)col * D.ga_cs];
            if (dgb) g = fma(gbs, dgb[r * D.gb_rs + (int64_t)col * D.gb_cs], g);
          }
          Gs[a * GLD + cc] = g;
        }
        // the window products below are subtracted by other threads (lanes <-> rows); without
        // the staging barriers of the synchronous path this one orders the two
        if (pre) __syncthreads();
      }

      T acc[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) acc[q] = (T)0;
      for (int jc0 = jlo; jc0 < jhi; jc0 += WCH) {
        const int jce = min(jhi, jc0 + WCH);
        const int tot = pre ? 0 : (jce - jc0) * NB;  // prefetched: the window is already staged
        if (!pre) __syncthreads();
        for (int base = tid; base < tot; base += NTHREADS * 8) {
          T v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int idx = base + u * NTHREADS;
            const int jj = idx / NB, a = idx - jj * NB, j = jc0 + jj;
            v[u] = (idx < tot && a < nbk && (FWD ? (j >= a) : (j <= kw - 1 - a)))
                       ? coef<T>(kind, dfb, ldf, dofs, row(a), wrow(j)) : (T)0;
          }
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (base + u * NTHREADS < tot) Tw[base + u * NTHREADS] = v[u];
        }
        if (!pre) __syncthreads();
        const int per = (jce - jc0 + nsplit - 1) / nsplit;
        // A predicated-off DFMA still occupies the FP64 pipe, so the accumulation loop is
        // instantiated for the exact column count; edge columns are clamped, not predicated.
        // FP64, one warp group per column group and a full window in one staged chunk: the window's
        // triangle rows take window_tri (33 steps over half the columns instead of 32 over all)
        const bool tri = sizeof(T) == 8 && !fixed && nsplit == 1 && pre && jlo == 0 && jhi == kw && kw >= 32 &&
                         cpw >= 2;
        auto partial = [&](int sp) {
          if (tri) {
            const int m0 = FWD ? 32 : 0, m1 = FWD ? kw : kw - 32, t0 = FWD ? 0 : kw - 32;
            const T *tm = Tw + (m0 - jc0) * NB + lane, *xm = dx + wrow(m0) * D.x_rs;
            const T *tt = Tw + (t0 - jc0) * NB, *xt = dx + wrow(t0) * D.x_rs;
            const int64_t step = D.x_rs;
            if (cpw <= 2) {
              window_fma<T, 2>(acc, tm, xm, step, D.x_cs, col_base, lastc, m1 - m0);
              window_tri<T, 2>(acc, tt, xt, step, D.x_cs, col_base, lastc, FWD);
            } else if (cpw <= 4) {
              window_fma<T, 4>(acc, tm, xm, step, D.x_cs, col_base, lastc, m1 - m0);
              window_tri<T, 4>(acc, tt, xt, step, D.x_cs, col_base, lastc, FWD);
            } else if (cpw <= 8) {
              window_fma<T, 8>(acc, tm, xm, step, D.x_cs, col_base, lastc, m1 - m0);
              window_tri<T, 8>(acc, tt, xt, step, D.x_cs, col_base, lastc, FWD);
            } else {
              window_fma<T, 16>(acc, tm, xm, step, D.x_cs, col_base, lastc, m1 - m0);
              window_tri<T, 16>(acc, tt, xt, step, D.x_cs, col_base, lastc, FWD);
            }
            return;
          }
          const int js = min(jce, jc0 + sp * per), je = min(jce, js + per);
          const T *xw = dx + wrow(js) * D.x_rs;
          const int64_t step = D.x_rs;  // wrow(j+1) = wrow(j) + 1 in both sweep directions
          const T *tw = Tw + (js - jc0) * NB + lane;
          if (cpw <= 1) window_fma<T, 1>(acc, tw, xw, step, D.x_cs, col_base, lastc, je - js);
          else if (cpw <= 2) window_fma<T, 2>(acc, tw, xw, step, D.x_cs, col_base, lastc, je - js);
          else if (cpw <= 4) window_fma<T, 4>(acc, tw, xw, step, D.x_cs, col_base, lastc, je - js);
          else if (cpw <= 8) window_fma<T, 8>(acc, tw, xw, step, D.x_cs, col_base, lastc, je - js);
          else window_fma<T, 16>(acc, tw, xw, step, D.x_cs, col_base, lastc, je - js);
        };
        auto subtract = [&]() {
          if (lane < nbk) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const int col = col_base + q;
              if (q < cpw && col <= lastc) Gs[lane * GLD + (col - c0)] -= acc[q];
            }
          }
#pragma unroll
          for (int q = 0; q < 16; ++q) acc[q] = (T)0;
        };
        if (!fixed) {
          partial(split);  // accumulates across chunks; combined after the last one
        } else if (by_split) {
          partial(warp);
          for (int sp = 0; sp < WSPLIT; ++sp) {
            __syncthreads();
            if (warp == sp) subtract();
          }
        } else if (owns) {
          for (int sp = 0; sp < WSPLIT; ++sp) {
            partial(sp);
            subtract();
          }
        }
      }
      __syncthreads();
      if (!fixed) {
        for (int s = 0; s < nsplit; ++s) {
          if (split == s) {
            if (lane < nbk) {
              const int64_t r = row(lane);
#pragma unroll
              for (int q = 0; q < 16; ++q) {
                const int col = col_base + q;
                if (q < cpw && col < c0 + cw) {
                  T g;
                  if (s == 0) {
                    g = dga[r * D.ga_rs + (int64_t)col * D.ga_cs];
                    if (dgb) g = fma(gbs, dgb[r * D.gb_rs + (int64_t)col * D.gb_cs], g);
                  } else {
                    g = Gs[lane * GLD + (col - c0)];
                  }
                  Gs[lane * GLD + (col - c0)] = g - acc[q];
                }
              }
            } else if (s == 0) {
#pragma unroll
              for (int q = 0; q < 16; ++q) {
                const int col = col_base + q;
                if (q < cpw && col < c0 + cw) Gs[lane * GLD + (col - c0)] = (T)0;
              }
            }
          }
          __syncthreads();
        }
      }
      // in-block triangular solve: X(a) = d(a) s(a), s(a) = G(a) - sum_{ap<a} T'(a, ap) s(ap)
      // with T'(a, ap) = T(a, ap) d(ap) and the sum taken in ascending ap.  Both schedules
      // below apply the same FMAs in the same order to every column, so a column's bits do
      // not depend on how many columns share the pass.
      for (int idx = tid; idx < NB * NB; idx += NTHREADS) Td[idx] *= dsm[idx / NB];  // Td[ap*NB + a] *= d(ap)
      __syncthreads();
      if (cw >= 32) {
        // blocked: sub-blocks of 8 rows; a thread per column solves the sub-block, then all
        // threads apply its 8 columns of T' to the rows below ((row, column) pairs in parallel)
        for (int q0 = 0; q0 < NB; q0 += 8) {
          for (int cc = tid; cc < cw; cc += NTHREADS) {
            T sv[8];
#pragma unroll
            for (int a = 0; a < 8; ++a) {
              T v = Gs[(q0 + a) * GLD + cc];
#pragma unroll
              for (int ap = 0; ap < a; ++ap) v = fma(-Td[(q0 + ap) * NB + q0 + a], sv[ap], v);
              sv[a] = v;
            }
#pragma unroll
            for (int a = 0; a < 8; ++a) Gs[(q0 + a) * GLD + cc] = sv[a];
          }
          __syncthreads();
          const int below = NB - q0 - 8;
          for (int idx = tid; idx < below * cw; idx += NTHREADS) {
            const int r = q0 + 8 + idx / cw, cc = idx - (idx / cw) * cw;
            T v = Gs[r * GLD + cc];
#pragma unroll
            for (int ap = 0; ap < 8; ++ap) v = fma(-Td[(q0 + ap) * NB + r], Gs[(q0 + ap) * GLD + cc], v);
            Gs[r * GLD + cc] = v;
          }
          __syncthreads();
        }
        for (int idx = tid; idx < NB * cw; idx += NTHREADS) {
          const int a = idx / cw, cc = idx - a * cw;
          Gs[a * GLD + cc] *= dsm[a];
        }
      } else {
        // a warp per column, lanes <-> rows: step ap broadcasts the finished s(ap)
        for (int cc = warp; cc < cw; cc += nwarps) {
          T v = Gs[lane * GLD + cc];
#pragma unroll
          for (int ap = 0; ap < NB; ++ap) {
            const T sa = __shfl_sync(FULLMASK, v, ap);
            if (lane > ap) v = fma(-Td[ap * NB + lane], sa, v);
          }
          Gs[lane * GLD + cc] = v * dsm[lane];
        }
      }
      __syncthreads();
      if (D.x_cs == 1) {  // row-major X: columns contiguous
        for (int idx = tid; idx < nbk * cw; idx += NTHREADS) {
          const int cc = idx % cw, a = idx / cw;
          dx[row(a) * D.x_rs + (c0 + cc)] = Gs[a * GLD + cc];
        }
      } else {
        for (int idx = tid; idx < nbk * cw; idx += NTHREADS) {
          const int a = idx % nbk, cc = idx / nbk;
          dx[row(a) * D.x_rs + (int64_t)(c0 + cc) * D.x_cs] = Gs[a * GLD + cc];
        }
      }
    }
    __syncthreads();
  }
}

// Task t = descriptors [t*per_cta, (t+1)*per_cta), run back to back by one CTA.  Without a
// queue CTA b runs task b; with one (a zeroed counter) a grid of persistent CTAs takes
// tasks in index order (tasks are listed largest first) until all ntasks are taken.
template <typename T>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_sweeps(const SweepDesc *descs, int per_cta, int ldf, int dofs, int ntasks, unsigned int *queue) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ int s_task;
  int task = blockIdx.x;
  for (;;) {
    if (queue) {
      __syncthreads();
      if (threadIdx.x == 0) s_task = (int)atomicAdd(queue, 1u);
      __syncthreads();
      task = s_task;
    }
    if (task >= ntasks) break;
    for (int s = 0; s < per_cta; ++s) {
      sweep_run<T>(descs[(int64_t)task * per_cta + s], ldf, dofs, (T *)sm_raw);
      __syncthreads();
    }
    if (!queue) break;
  }
}

int launch_sweeps(const SweepDesc *descs, int ncta, int per_cta, int ldf, int dofs, void *stream, int f32,
                  unsigned int *queue, int grid) {
  if (ncta <= 0 || per_cta <= 0) return 0;
  const int g = queue ? std::max(1, std::min(grid, ncta)) : ncta;
  cudaError_t e;
  if (f32) {
    e = (cudaError_t)smem_at_least((const void *)k_sweeps<float>, SWEEP_SMEM);
    if (e != cudaSuccess) return (int)e;
    k_sweeps<float><<<g, NTHREADS, SWEEP_SMEM, (cudaStream_t)stream>>>(descs, per_cta, ldf, dofs, ncta, queue);
  } else {
    e = (cudaError_t)smem_at_least((const void *)k_sweeps<double>, SWEEP_SMEM);
    if (e != cudaSuccess) return (int)e;
    k_sweeps<double><<<g, NTHREADS, SWEEP_SMEM, (cudaStream_t)stream>>>(descs, per_cta, ldf, dofs, ncta, queue);
  }
  count_launch();
  return (int)cudaGetLastError();
}

// ------------------------------------------------ pivoted L sweeps (Sec. 5.1)
// In place on X, rows [r0, r1) with r1 = nl.  One warp per RHS column.
//   LN (forward):  for j: swap X_j <-> X_ipiv[j]; X_{j+1..j+k} -= l_{.,j} X_j
//   LT (backward): for j descending: X_j -= sum_i l_{i,j} X_i; swap X_j <-> X_ipiv[j]
// The rows a step touches (j..j+k; ipiv[j] <= j+k) live in a per-warp circular window in
// shared memory (row i at slot i mod (k+1)); rows enter and leave it once, through registers
// that hold the next 32 rows to load and the last 32 finished rows (one per lane), so the
// dependent chain of a step stays in shared memory and shuffles.
constexpr int LPRE = 4;  // multipliers a lane prefetches per step (k <= 128; wider bands read the rest directly)

template <int KIND>
__device__ void piv_sweep_run(const SweepDesc &D, int k, int ldf, int dofs, double *pwin) {
  if (D.ncols <= 0 || D.r1 <= D.r0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int WIN = k + 1;
  double *buf = pwin + (size_t)warp * (k + 2);
  // row j + d (0 <= d <= k) sits in slot (jw + d) mod WIN, jw = j mod WIN kept incrementally
  auto wrap = [&](int x) { return x >= WIN ? x - WIN : x; };
  const int r0 = (int)D.r0, r1 = (int)D.r1;
  const int64_t rs = D.x_rs;
  for (int col = warp; col < D.ncols; col += NTHREADS / 32) {
    double *x = D.x + (int64_t)col * D.x_cs;
    if (KIND == LN) {
      int jw = r0 % WIN;
      const int top = min(r0 + k, r1 - 1);
      for (int d = lane; d <= top - r0; d += 32) buf[wrap(jw + d)] = x[(int64_t)(r0 + d) * rs];
      int pbase = r0 + k + 1;  // rows pbase .. pbase+31 are held in `pre` (lane l: row pbase + l)
      double pre = (pbase + lane < r1) ? x[(int64_t)(pbase + lane) * rs] : 0.0;
      int obase = r0;  // finished rows obase .. held in `outv` (lane l: row obase + l)
      double outv = 0.0;
      double lc[LPRE];  // multipliers of the current step (lane l: rows j + 1 + l + 32 t)
      {
        const double *l0 = D.fb + (int64_t)r0 * ldf + dofs;
        const int d0 = min(k, r1 - 1 - r0);
#pragma unroll
        for (int t = 0; t < LPRE; ++t) lc[t] = (1 + lane + 32 * t <= d0) ? l0[1 + lane + 32 * t] : 0.0;
      }
      __syncwarp();
      for (int j = r0; j < r1; ++j) {
        const int pd = D.ipiv[j] - j;
        if (lane == 0 && pd != 0) {
          const int b = wrap(jw + pd);
          const double t = buf[jw];
          buf[jw] = buf[b];
          buf[b] = t;
        }
        __syncwarp();
        const double xj = buf[jw];
        const int dl = min(k, r1 - 1 - j);
#pragma unroll
        for (int t = 0; t < LPRE; ++t) {
          const int d = 1 + lane + 32 * t;
          if (d <= dl) {
            const int sl = wrap(jw + d);
            buf[sl] = fma(-lc[t], xj, buf[sl]);
          }
        }
        for (int d = 1 + lane + 32 * LPRE; d <= dl; d += 32) {  // k > 32 LPRE
          const int sl = wrap(jw + d);
          buf[sl] = fma(-D.fb[(int64_t)j * ldf + dofs + d], xj, buf[sl]);
        }
        // the next step's multipliers (column j + 1 of L), read while this step finishes
        if (j + 1 < r1) {
          const double *ln = D.fb + (int64_t)(j + 1) * ldf + dofs;
          const int dn = min(k, r1 - 2 - j);
#pragma unroll
          for (int t = 0; t < LPRE; ++t) lc[t] = (1 + lane + 32 * t <= dn) ? ln[1 + lane + 32 * t] : 0.0;
        }
        if (lane == j - obase) outv = xj;
        if (j - obase == 31 || j == r1 - 1) {
          if (obase + lane <= j) x[(int64_t)(obase + lane) * rs] = outv;
          obase = j + 1;
        }
        __syncwarp();
        const int rn = j + k + 1;  // enters the slot row j leaves: (jw + k + 1) mod WIN = jw
        if (rn < r1) {
          const double v = __shfl_sync(FULLMASK, pre, rn - pbase);
          if (lane == 0) buf[jw] = v;
          if (rn - pbase == 31) {
            pbase += 32;
            pre = (pbase + lane < r1) ? x[(int64_t)(pbase + lane) * rs] : 0.0;
          }
        }
        jw = wrap(jw + 1);
      }
    } else {
      int jw = (r1 - 1) % WIN;
      int pbase = r1 - 1;  // rows pbase, pbase-1, ... held in `pre` (lane l: row pbase - l)
      double pre = (pbase - lane >= r0) ? x[(int64_t)(pbase - lane) * rs] : 0.0;
      int obase = r1 - 1;  // finished rows obase, obase-1, ... held in `outv`
      double outv = 0.0;
      double lc[LPRE];  // multipliers of the current step (the last row has none)
#pragma unroll
      for (int t = 0; t < LPRE; ++t) lc[t] = 0.0;
      for (int j = r1 - 1; j >= r0; --j) {
        const double xj = __shfl_sync(FULLMASK, pre, pbase - j);
        if (pbase - j == 31) {
          pbase -= 32;
          pre = (pbase - lane >= r0) ? x[(int64_t)(pbase - lane) * rs] : 0.0;
        }
        const int dl = min(k, r1 - 1 - j);
        double sacc = 0.0;
#pragma unroll
        for (int t = 0; t < LPRE; ++t) {
          const int d = 1 + lane + 32 * t;
          if (d <= dl) sacc = fma(lc[t], buf[wrap(jw + d)], sacc);
        }
        for (int d = 1 + lane + 32 * LPRE; d <= dl; d += 32)
          sacc = fma(D.fb[(int64_t)j * ldf + dofs + d], buf[wrap(jw + d)], sacc);
        // the next step's multipliers (column j - 1 of L)
        if (j - 1 >= r0) {
          const double *ln = D.fb + (int64_t)(j - 1) * ldf + dofs;
          const int dn = min(k, r1 - j);
#pragma unroll
          for (int t = 0; t < LPRE; ++t) lc[t] = (1 + lane + 32 * t <= dn) ? ln[1 + lane + 32 * t] : 0.0;
        }
        for (int o = 16; o; o >>= 1) sacc += __shfl_xor_sync(FULLMASK, sacc, o);
        const double v = xj - sacc;
        const int pd = D.ipiv[j] - j;
        if (lane == 0) {
          if (pd != 0) {
            const int b = wrap(jw + pd);
            buf[jw] = buf[b];
            buf[b] = v;
          } else {
            buf[jw] = v;
          }
        }
        __syncwarp();
        // row j + k is final now (later steps swap only rows below j + k); its slot is reused
        // by row j - 1
        const int rl = j + k;
        if (rl <= r1 - 1) {
          const double fv = buf[wrap(jw + k)];
          if (lane == obase - rl) outv = fv;
          if (obase - rl == 31) {
            if (obase - lane >= rl) x[(int64_t)(obase - lane) * rs] = outv;
            obase = rl - 1;
          }
        }
        __syncwarp();
        jw = (jw == 0) ? WIN - 1 : jw - 1;
      }
      // the rows still held: pending `outv` (obase down to r0 + k) and the window r0 .. r0+k-1
      const int wtop = min(r0 + k - 1, r1 - 1);
      if (obase > wtop && obase - lane > wtop && obase - lane >= r0) x[(int64_t)(obase - lane) * rs] = outv;
      const int w0 = r0 % WIN;
      for (int d = lane; d <= wtop - r0; d += 32) x[(int64_t)(r0 + d) * rs] = buf[wrap(w0 + d)];
    }
    __syncwarp();
  }
}

template <int KIND>
__global__ void __launch_bounds__(NTHREADS) k_piv_sweep(const SweepDesc *descs, int k, int ldf, int dofs) {
  extern __shared__ double pwin[];
  piv_sweep_run<KIND>(descs[blockIdx.x], k, ldf, dofs, pwin);
}

int launch_piv_sweep(int kind, const SweepDesc *descs, int ndesc, int k, int ldf, int dofs, void *stream) {
  if (ndesc <= 0) return 0;
  const size_t smem = sizeof(double) * (size_t)(NTHREADS / 32) * (k + 2);
  if (kind == LN)
    k_piv_sweep<LN><<<ndesc, NTHREADS, smem, (cudaStream_t)stream>>>(descs, k, ldf, dofs);
  else
    k_piv_sweep<LT><<<ndesc, NTHREADS, smem, (cudaStream_t)stream>>>(descs, k, ldf, dofs);
  count_launch();
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------ tips (level 0)
// Spike tips of each leaf in the global frame from the swept Z:
//   forward leaf : W = Z_top, V = Z_bot;   reversed leaf: V = Q Z_top, W = Q Z_bot.
// spk layout: [V/W][leaf][top/bottom] k x k row-major (level 0).
template <typename T>
__global__ void k_tips0(const LeafDev *leaves, int nleaves, int k, const T *zbuf, const int64_t *zoff,
                        double *spk) {
  const int i = blockIdx.x;
  const LeafDev L = leaves[i];
  const int64_t nl = L.len;
  const T *Z = zbuf + zoff[i];
  const int64_t kk = (int64_t)k * k;
  const bool mid = L.top_nbr && L.bot_nbr;
  for (int64_t idx = threadIdx.x; idx < kk; idx += blockDim.x) {
    const int j = (int)(idx / k), b = (int)(idx % k);  // tip row j, column b
    // local rows of global top/bottom tip row j
    const int64_t lt = L.rev ? (nl - 1 - j) : j;             // global top row j
    const int64_t lb = L.rev ? (k - 1 - j) : (nl - k + j);   // global bottom row j
    const T *Ztop = Z, *Zbot = Z + (int64_t)k * nl;
    // spike coupled through the local top rows is W (fwd) / V (rev); through the bottom: V (fwd) / W (rev)
    const int s_top = L.rev ? 0 : 1, s_bot = L.rev ? 1 : 0;
    if (mid) {
      spk[((int64_t)(s_top * nleaves + i) * 2 + 0) * kk + idx] = Ztop[(int64_t)b * nl + lt];
      spk[((int64_t)(s_top * nleaves + i) * 2 + 1) * kk + idx] = Ztop[(int64_t)b * nl + lb];
      spk[((int64_t)(s_bot * nleaves + i) * 2 + 0) * kk + idx] = Zbot[(int64_t)b * nl + lt];
      spk[((int64_t)(s_bot * nleaves + i) * 2 + 1) * kk + idx] = Zbot[(int64_t)b * nl + lb];
    } else if (L.bot_nbr) {
      // first-like leaf: only the tip at the local bottom of the bottom spike exists
      if (L.rev) spk[((int64_t)(s_bot * nleaves + i) * 2 + 0) * kk + idx] = Zbot[(int64_t)b * nl + lt];
      else spk[((int64_t)(s_bot * nleaves + i) * 2 + 1) * kk + idx] = Zbot[(int64_t)b * nl + lb];
    }
  }
}

int launch_tips0(const LeafDev *leaves, int nleaves, int k, const void *zbuf, const int64_t *zoff, double *spk,
                 void *stream, int f32) {
  if (f32)
    k_tips0<float><<<nleaves, 256, 0, (cudaStream_t)stream>>>(leaves, nleaves, k, (const float *)zbuf, zoff, spk);
  else
    k_tips0<double><<<nleaves, 256, 0, (cudaStream_t)stream>>>(leaves, nleaves, k, (const double *)zbuf, zoff, spk);
  count_launch();
  return (int)cudaGetLastError();
}

}  // namespace spk
