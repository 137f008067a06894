// FP64-accurate banded residual R = F - op(A) X on the tensor cores, for the iterative
// refinement of mixed-precision solves (Sec. 5: refinement after an approximate
// factorization; the residual must be formed to working (FP64) accuracy).
//
// Method (integer slices, exact products).  Every entry of op(A) is written, up to one
// rounding, as a 56-bit fixed-point number relative to a power of two of its row, and
// every entry of X relative to a power of two of its column:
//   a_ij = 2^(e_i - 56) * A_i,j ,  x_jc = 2^(f_c - 56) * X_j,c ,  |A|, |X| <= 2^54,
// and each fixed-point integer is split into 8 signed base-128 digits d in [-64, 63]:
//   A = sum_p dA_p 2^(7(8-p)),  X = sum_q dX_q 2^(7(8-q)),  p, q = 1..8
// (stored biased, u = d + 64 in [0, 127]).  Then
//   sum_j a_ij x_jc = 2^(e_i + f_c - 112) sum_{p,q} 2^(7(16-p-q)) P_pq,
//   P_pq = sum_j dA_p(i,j) dX_q(j,c).
// Each P_pq is a bf16 x bf16 tensor-core product (digits and their products are exact in
// bf16 / FP32) accumulated in FP32; the products of one level L = p + q share a weight and
// one accumulator.  Every partial sum is an integer below 2^23 (at most 8 products of
// |d d| <= 2^12 over 8 chunks of 32 terms between drains), so the FP32 accumulation is
// exact; the accumulators are drained into two exact int64 sums (levels 2..6 and 7..10).
// Levels above 10 (21 of the 64 products) weigh < 2^-63 of the leading one and are not
// formed.  The only roundings are therefore the two fixed-point conversions (2^-56 of the
// row / column scale), the sum of the two int64 groups in FP64 and the final f - Ax: below
// the rounding error of a plain FP64 dot product of the same length.  On this part the
// FP64 FMA pipe retires 2 FMAs per clock per SM; the bf16 tensor path ~1000 multiply-adds.
//
// Storage:
//   digits of op(A): per 16-row block mb, plane p, 32-column chunk c, lane: 16 biased
//     digits (one uint4) laid out as the lane's m16n8k32 int8 A fragment: rows g, g+8
//     (g = lane/4) x columns 4t..4t+3 and 16+4t..16+4t+3 (t = lane%4) of the chunk.  Each
//     32-column chunk feeds two m16n8k16 bf16 products whose K order is permuted (logical
//     k 2t, 2t+1, 2t+8, 2t+9 <-> physical 4t..4t+3), the same permutation on both operands,
//     so the lane converts its own bytes into both fragments.  Warps stream their
//     fragments with coalesced 16-byte loads.  The block's columns start at
//     j0(mb) = floor4(16 mb - lo) (lo = kl for N, ku for T) and span KP = 32 * nchunks
//     >= 16 + lo + hi + 3 columns.
//   row exponents e_i (int32) and ||op(A)||_inf (max row sum of |a|), per orientation.
//   digits of X: plane q, column c, row j + XPAD (uint8, XPAD rows of digit 64 (zero) on
//     both sides so every window read is in range), column stride ldx bytes.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace spk {

#define FULLMASK 0xffffffffu

constexpr int SPL_PLANES = 8;      // base-128 digits per 56-bit fixed-point value
constexpr int SPL_MAXLEVEL = 10;   // products p + q <= 10 are formed
constexpr int SPL_NLEV = SPL_MAXLEVEL - 1;  // levels 2..10
constexpr int SPL_MC = 32;         // right-hand-side columns per pass (4 n8 tiles per warp)
constexpr int SPL_WARPS = 8;       // warps per CTA: 4 16-row blocks x 2 column halves

// 2^s as a double (s in the normal range), else ldexp
__device__ __forceinline__ double pow2(int s) {
  if (s >= -1022 && s <= 1023) return __longlong_as_double((long long)(s + 1023) << 52);
  return ldexp(1.0, s);
}

// exponent e with max|v| < 2^(e-2) (so |v| 2^(56-e) < 2^54); 0 for v == 0
__device__ __forceinline__ int scale_exp(double amax) {
  if (!(amax > 0.0)) return 0;
  int e;
  frexp(amax, &e);  // amax = m 2^e, m in [0.5, 1)  ->  amax < 2^e
  return e + 2;
}

// 56-bit fixed point of v relative to 2^e, rounded to nearest, then biased so that the 8
// base-128 digits of the result minus 64 are the balanced digits of the fixed-point value.
// Returns the biased value U in [0, 2^56).
__device__ __forceinline__ unsigned long long fixed_biased(double v, int e) {
  // v * 2^(56 - e): exact scaling by a power of two, then round to the nearest integer
  const long long f = __double2ll_rn(v * pow2(56 - e));
  // bias = 64 * sum_{p=1..8} 2^(7(8-p)): every digit of f + bias then lies in [0, 127]
  const unsigned long long bias = 0x0081020408102040ull;
  return (unsigned long long)(f + (long long)bias);
}

// biased digit p = 0..7 (most significant first): d + 64 in [0, 127]
__device__ __forceinline__ uint32_t udigit(unsigned long long u, int p) { return (uint32_t)((u >> (7 * (7 - p))) & 127ull); }

// ------------------------------------------------------------ A: row exponents, norm
// One thread per row of op(A): e_i and the row sum of |a| (max over rows -> norm bits).
__global__ void __launch_bounds__(256) k_split_rows(const double *__restrict__ band, int64_t ldab, int64_t n, int kl,
                                                    int ku, int trans, int *rexp, unsigned long long *norm_bits) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double amax = 0.0, asum = 0.0;
  if (i < n) {
    const int lo = trans ? ku : kl, hi = trans ? kl : ku;
    const int64_t jlo = i - lo > 0 ? i - lo : 0, jhi = i + hi < n - 1 ? i + hi : n - 1;
    for (int64_t j = jlo; j <= jhi; ++j) {
      const double v = trans ? band[i * ldab + ku + j - i] : band[j * ldab + ku + i - j];
      amax = fmax(amax, fabs(v));
      asum += fabs(v);
    }
    rexp[i] = scale_exp(amax);
  }
  for (int o = 16; o; o >>= 1) asum = fmax(asum, __shfl_xor_sync(FULLMASK, asum, o));
  if ((threadIdx.x & 31) == 0) atomicMax(norm_bits, (unsigned long long)__double_as_longlong(asum));
}

// ------------------------------------------------------------ A: digit fragments
// One warp per (16-row block, 32-column chunk).  Lane (g = lane/4, t = lane%4) owns rows g
// and g + 8 and columns 4t..4t+3 and 16+4t..16+4t+3 of the chunk (m16n8k32 A fragment:
// reg0 (g, 4t..), reg1 (g+8, 4t..), reg2 (g, 16+4t..), reg3 (g+8, 16+4t..), byte u = column
// offset u).  Writes the 8 digit planes of that fragment.
__global__ void __launch_bounds__(256) k_split_band(const double *__restrict__ band, int64_t ldab, int64_t n, int kl,
                                                    int ku, int trans, int nchunks, const int *__restrict__ rexp,
                                                    uint4 *frag) {
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nmb = (n + 15) / 16;
  if (wid >= nmb * nchunks) return;
  const int64_t mb = wid / nchunks;
  const int ch = (int)(wid - mb * nchunks);
  const int lo = trans ? ku : kl, hi = trans ? kl : ku;
  const int64_t i0 = mb * 16;
  const int64_t j0 = ((i0 - lo) >= 0 ? (i0 - lo) : -((lo - i0 + 3) / 4) * 4) & ~(int64_t)3;  // floor to a multiple of 4
  const int g = lane >> 2, t = lane & 3;
  uint32_t w[SPL_PLANES][4];
#pragma unroll
  for (int p = 0; p < SPL_PLANES; ++p)
#pragma unroll
    for (int r = 0; r < 4; ++r) w[p][r] = 0u;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t i = i0 + g + ((r & 1) ? 8 : 0);
    const int kb = ch * 32 + ((r & 2) ? 16 : 0) + 4 * t;
    const int e = (i < n) ? rexp[i] : 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t j = j0 + kb + u;
      double v = 0.0;
      if (i < n && j >= 0 && j < n && j >= i - lo && j <= i + hi)
        v = trans ? band[i * ldab + ku + j - i] : band[j * ldab + ku + i - j];
      const unsigned long long U = fixed_biased(v, e);
#pragma unroll
      for (int p = 0; p < SPL_PLANES; ++p) w[p][r] |= udigit(U, p) << (8 * u);
    }
  }
#pragma unroll
  for (int p = 0; p < SPL_PLANES; ++p)
    frag[((mb * SPL_PLANES + p) * nchunks + ch) * 32 + lane] = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
}

// ------------------------------------------------------------ X: column maxima, digits
// norms[2 + 2c] = ||x_c||_inf (bit pattern, atomicMax; also the backward-error denominator)
__global__ void __launch_bounds__(256) k_split_colmax(const double *__restrict__ X, int64_t n,
                                                      unsigned long long *norms) {
  const int c = blockIdx.y;
  const double *x = X + (int64_t)c * n;
  double m = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[i]));
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(FULLMASK, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&norms[2 + 2 * c], (unsigned long long)__double_as_longlong(m));
}

// One thread per 4 consecutive rows of one column: one 32-bit word per digit plane.
// xd: plane q at xd + q * plane_stride, column c at + c * ldx, row j at + XPAD + j.
__global__ void __launch_bounds__(256) k_split_x(const double *__restrict__ X, int64_t n, int nrhs,
                                                 const unsigned long long *__restrict__ norms, uint8_t *xd, int64_t ldx,
                                                 int64_t plane_stride, int xpad) {
  const int c = blockIdx.y;
  const int64_t j4 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * 4;
  if (j4 >= n || c >= nrhs) return;
  const int f = scale_exp(__longlong_as_double((long long)norms[2 + 2 * c]));
  const double *x = X + (int64_t)c * n;
  uint32_t w[SPL_PLANES];
#pragma unroll
  for (int p = 0; p < SPL_PLANES; ++p) w[p] = 0u;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const double v = (j4 + u < n) ? x[j4 + u] : 0.0;
    const unsigned long long U = fixed_biased(v, f);
#pragma unroll
    for (int p = 0; p < SPL_PLANES; ++p) w[p] |= udigit(U, p) << (8 * u);
  }
  uint8_t *base = xd + (int64_t)c * ldx + xpad + j4;
#pragma unroll
  for (int p = 0; p < SPL_PLANES; ++p) *(uint32_t *)(base + (int64_t)p * plane_stride) = w[p];
}

// ------------------------------------------------------------ the product kernel
// Four biased digits (bytes of w) -> two bf16x2 of the digits: bytes (u0, u1) -> bf16 pair
// (128 + u0, 128 + u1) by placing 0x43 above each byte (bf16 0x43uu = 128 + uu for uu < 128),
// then subtract 192 (exact: the results are integers in [-64, 63]).
__device__ __forceinline__ void digits_to_bf16(uint32_t w, uint32_t &lo, uint32_t &hi) {
  uint32_t a, b;
  const uint32_t k43 = 0x43434343u;
  asm("prmt.b32 %0, %1, %2, 0x4140;" : "=r"(a) : "r"(w), "r"(k43));
  asm("prmt.b32 %0, %1, %2, 0x4342;" : "=r"(b) : "r"(w), "r"(k43));
  const uint32_t c192 = 0x43404340u;  // bf16x2 (192, 192)
  asm("sub.rn.bf16x2 %0, %1, %2;" : "=r"(lo) : "r"(a), "r"(c192));
  asm("sub.rn.bf16x2 %0, %1, %2;" : "=r"(hi) : "r"(b), "r"(c192));
}

__device__ __forceinline__ void mma_bf16(float *c, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

constexpr int SPL_NT = 2;       // n8 tiles per warp (16 right-hand-side columns)
constexpr int SPL_DRAIN = 8;    // chunks between drains of the FP32 accumulators (sums < 2^23)

// One CTA = SPL_WARPS / 2 consecutive 16-row blocks x the two 16-column halves of a pass of
// SPL_MC right-hand sides (warp w: block w % 4, columns 16 (w / 4) ..).  Per pass the CTA
// stages the digit planes of the X rows its blocks touch (XW rows x SPL_MC columns x 8
// planes) in shared memory; each warp streams its block's A fragments from global memory
// (the two column halves read the same fragments, the second from L1/L2) and accumulates
// the 9 levels in FP32, drained into two int64 sums.  Epilogue: the two sums -> FP64,
// scaled by 2^(e_i + f_c - ...), r = f - Ax, per-column max |r| (norms[1 + 2c]).
__global__ void __launch_bounds__(SPL_WARPS * 32, 1)
    k_resid_split(const uint4 *__restrict__ frag, const int *__restrict__ rexp, int nchunks, int64_t n, int lo,
                  const uint8_t *__restrict__ xd, int64_t ldx, int64_t plane_stride, int xpad, int nrhs,
                  const double *__restrict__ F, double *R, unsigned long long *norms, int XWP) {
  extern __shared__ __align__(16) uint8_t xs[];  // [plane][column][XWP]
  constexpr int MBS = SPL_WARPS / 2;             // 16-row blocks per CTA
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int wmb = warp % MBS, wcol = warp / MBS;
  const int64_t nmb = (n + 15) / 16;
  const int64_t mb0 = (int64_t)blockIdx.x * MBS;
  const int64_t mb = mb0 + wmb;
  auto floor_to = [](int64_t v, int64_t a) { return v >= 0 ? (v / a) * a : -((-v + a - 1) / a) * a; };
  // window of the CTA: J0 = floor16(16 mb0 - lo); each block's window starts at floor4(16 mb - lo)
  const int64_t J0 = floor_to(mb0 * 16 - lo, 16);
  const int64_t jw = floor_to(mb * 16 - lo, 4);
  const int woff = (int)(jw - J0);
  const int KP = nchunks * 32;
  const int XW = (MBS - 1) * 16 + KP + 16;  // staged rows (multiple of 16)
  const bool active = mb < nmb;
  const uint4 *fr = frag + (mb * SPL_PLANES) * (int64_t)nchunks * 32 + lane;
  // the warp's A fragments of the next chunk are copied to shared memory while the current
  // chunk computes (each lane copies and later reads back its own 16 bytes per plane)
  uint4 *abuf = (uint4 *)(xs + (size_t)SPL_PLANES * SPL_MC * XWP) + (size_t)warp * SPL_PLANES * 32 + lane;
  auto prefetch = [&](int ch) {
#pragma unroll
    for (int p = 0; p < SPL_PLANES; ++p) {
      const unsigned d = (unsigned)__cvta_generic_to_shared(abuf + p * 32);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(fr + ((int64_t)p * nchunks + ch) * 32)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  for (int c0 = 0; c0 < nrhs; c0 += SPL_MC) {
    __syncthreads();  // the previous pass's reads of xs are done
    {
      const int segs = XW / 16;
      const int total = SPL_PLANES * SPL_MC * segs;
      for (int idx = threadIdx.x; idx < total; idx += SPL_WARPS * 32) {
        const int sg = idx % segs, rest = idx / segs;
        const int cc = rest % SPL_MC, p = rest / SPL_MC;
        uint4 v = make_uint4(0x40404040u, 0x40404040u, 0x40404040u, 0x40404040u);  // digit 0
        if (c0 + cc < nrhs)
          v = *(const uint4 *)(xd + (int64_t)p * plane_stride + (int64_t)(c0 + cc) * ldx + xpad + J0 + 16 * sg);
        *(uint4 *)(xs + ((int64_t)p * SPL_MC + cc) * XWP + 16 * sg) = v;
      }
    }
    __syncthreads();
    if (!active || c0 + 16 * wcol >= nrhs) continue;
    float acc[SPL_NLEV][SPL_NT][4];
    long long vh[SPL_NT][4], vl[SPL_NT][4];
#pragma unroll
    for (int nt = 0; nt < SPL_NT; ++nt)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        vh[nt][r] = 0;
        vl[nt][r] = 0;
#pragma unroll
        for (int l = 0; l < SPL_NLEV; ++l) acc[l][nt][r] = 0.f;
      }
    auto drain = [&]() {
#pragma unroll
      for (int nt = 0; nt < SPL_NT; ++nt)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          long long h = 0, lw = 0;
#pragma unroll
          for (int l = 0; l < 5; ++l) h = h * 128 + (long long)__float2int_rn(acc[l][nt][r]);
#pragma unroll
          for (int l = 5; l < SPL_NLEV; ++l) lw = lw * 128 + (long long)__float2int_rn(acc[l][nt][r]);
          vh[nt][r] += h;
          vl[nt][r] += lw;
#pragma unroll
          for (int l = 0; l < SPL_NLEV; ++l) acc[l][nt][r] = 0.f;
        }
    };
    const uint8_t *xcol = xs + (int64_t)(16 * wcol + g) * XWP + woff + 4 * t;
    prefetch(0);
    for (int ch = 0; ch < nchunks; ++ch) {
      // A digits of the chunk, all planes: [plane][k-half][4 regs]
      uint32_t a[SPL_PLANES][2][4];
      asm volatile("cp.async.wait_all;\n" ::: "memory");
#pragma unroll
      for (int p = 0; p < SPL_PLANES; ++p) {
        const uint4 w = abuf[p * 32];
        // k-half 0: rows g (w.x) and g+8 (w.y), columns 4t..4t+3; k-half 1: w.z, w.w
        digits_to_bf16(w.x, a[p][0][0], a[p][0][2]);
        digits_to_bf16(w.y, a[p][0][1], a[p][0][3]);
        digits_to_bf16(w.z, a[p][1][0], a[p][1][2]);
        digits_to_bf16(w.w, a[p][1][1], a[p][1][3]);
      }
      // the converted fragments are in registers: the buffer takes the next chunk
      if (ch + 1 < nchunks) prefetch(ch + 1);
#pragma unroll
      for (int q = 0; q < SPL_PLANES; ++q) {
        uint32_t b[SPL_NT][2][2];
#pragma unroll
        for (int nt = 0; nt < SPL_NT; ++nt) {
          const uint8_t *col = xcol + ((int64_t)q * SPL_MC + nt * 8) * XWP + ch * 32;
          digits_to_bf16(*(const uint32_t *)col, b[nt][0][0], b[nt][0][1]);
          digits_to_bf16(*(const uint32_t *)(col + 16), b[nt][1][0], b[nt][1][1]);
        }
#pragma unroll
        for (int p = 0; p < SPL_PLANES; ++p) {
          if (p + q + 2 > SPL_MAXLEVEL) continue;  // level (p+1) + (q+1)
#pragma unroll
          for (int nt = 0; nt < SPL_NT; ++nt)
#pragma unroll
            for (int hk = 0; hk < 2; ++hk)
              mma_bf16(acc[p + q][nt], a[p][hk][0], a[p][hk][1], a[p][hk][2], a[p][hk][3], b[nt][hk][0],
                       b[nt][hk][1]);
        }
      }
      if ((ch + 1) % SPL_DRAIN == 0) drain();
    }
    drain();
    // epilogue: rows g and g+8 of the block, columns 2t, 2t+1 of each n8 tile
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int64_t i = mb * 16 + g + 8 * half;
      const int e = (i < n) ? rexp[i] : 0;
#pragma unroll
      for (int nt = 0; nt < SPL_NT; ++nt) {
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int col = c0 + 16 * wcol + nt * 8 + 2 * t + cc;
          const int r = half * 2 + cc;  // accumulator register: (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1)
          double rv = 0.0;
          if (i < n && col < nrhs) {
            const int f = scale_exp(__longlong_as_double((long long)norms[2 + 2 * col]));
            // sum = 2^(e+f-112) (vh 2^70 + vl 2^42)
            const double ax = fma((double)vl[nt][r], pow2(e + f - 70), (double)vh[nt][r] * pow2(e + f - 42));
            rv = F[(int64_t)col * n + i] - ax;
            R[(int64_t)col * n + i] = rv;
          }
          // column maximum of |r| over the 16 rows of the block: lanes with the same t
          double m = fabs(rv);
          for (int o = 4; o < 32; o <<= 1) m = fmax(m, __shfl_xor_sync(FULLMASK, m, o));
          if (g == 0 && col < nrhs) atomicMax(&norms[1 + 2 * col], (unsigned long long)__double_as_longlong(m));
        }
      }
    }
  }
}

// ------------------------------------------------------------ launchers
int split_chunks(int kl, int ku) { return (16 + kl + ku + 3 + 31) / 32; }

size_t split_band_bytes(int64_t n, int kl, int ku) {
  const int64_t nmb = (n + 15) / 16;
  return (size_t)nmb * SPL_PLANES * split_chunks(kl, ku) * 32 * sizeof(uint4);
}

// zero rows on each side of the X digit columns: the windows of the first and last CTAs reach
// at most kl + 15 rows above row 0 and ku + 113 rows below row n - 1
int split_xpad(int kl, int ku) { return ((kl > ku ? kl : ku) + 128 + 15) & ~15; }

static size_t split_smem(int kl, int ku, int *xwp) {
  const int KP = split_chunks(kl, ku) * 32;
  const int XW = (SPL_WARPS / 2 - 1) * 16 + KP + 16;
  int XWP = XW;
  while (XWP % 128 != 16) XWP += 16;  // column stride = 16 mod 128 bytes: conflict-free B fragments
  if (xwp) *xwp = XWP;
  // X digit planes, then one chunk of A fragments per warp (8 planes x 32 lanes x 16 bytes)
  return (size_t)SPL_PLANES * SPL_MC * XWP + (size_t)SPL_WARPS * SPL_PLANES * 32 * 16;
}

// The staged X digits and A fragments must fit a CTA's shared memory (kl + ku up to about 540).
bool split_supported(int kl, int ku) { return split_smem(kl, ku, nullptr) <= 227 * 1024; }

int64_t split_ldx(int64_t n, int kl, int ku) { return ((n + 2 * (int64_t)split_xpad(kl, ku)) + 15) & ~(int64_t)15; }

size_t split_x_bytes(int64_t n, int kl, int ku, int nrhs) {
  const int cols = (nrhs + SPL_MC - 1) / SPL_MC * SPL_MC;
  return (size_t)SPL_PLANES * cols * split_ldx(n, kl, ku);
}

int launch_split_band(const double *band, int64_t ldab, int64_t n, int kl, int ku, int trans, int *rexp,
                      unsigned long long *norm_bits, void *frag, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int nch = split_chunks(kl, ku);
  if (cudaMemsetAsync(norm_bits, 0, sizeof(unsigned long long), s) != cudaSuccess) return (int)cudaGetLastError();
  k_split_rows<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(band, ldab, n, kl, ku, trans, rexp, norm_bits);
  const int64_t warps = (n + 15) / 16 * nch;
  k_split_band<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(band, ldab, n, kl, ku, trans, nch, rexp,
                                                                    (uint4 *)frag);
  count_launch(2);
  return (int)cudaGetLastError();
}

int launch_resid_split(const void *frag, const int *rexp, const unsigned long long *anorm_bits, int64_t n, int kl,
                       int ku, int trans, const double *X, const double *F, double *R, int nrhs, void *xdig,
                       unsigned long long *norms, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int lo = trans ? ku : kl;
  const int nch = split_chunks(kl, ku);
  const int xpad = split_xpad(kl, ku);
  const int64_t ldx = split_ldx(n, kl, ku);
  const int cols = (nrhs + SPL_MC - 1) / SPL_MC * SPL_MC;
  const int64_t plane = (int64_t)cols * ldx;
  uint8_t *xd = (uint8_t *)xdig;
  // norms: [0] = ||op(A)||, [1+2c] = ||r_c|| (cleared), [2+2c] = ||x_c|| (computed here)
  if (cudaMemsetAsync(norms, 0, sizeof(unsigned long long) * (1 + 2 * (size_t)nrhs), s) != cudaSuccess ||
      cudaMemcpyAsync(norms, anorm_bits, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return (int)cudaGetLastError();
  int bx = (int)((n + 255) / 256);
  if (bx > 152 * 4) bx = 152 * 4;
  k_split_colmax<<<dim3(bx, nrhs), 256, 0, s>>>(X, n, norms);
  k_split_x<<<dim3((unsigned)((n + 4 * 256 - 1) / (4 * 256)), nrhs), 256, 0, s>>>(X, n, nrhs, norms, xd, ldx, plane,
                                                                                  xpad);
  int XWP = 0;
  const size_t smem = split_smem(kl, ku, &XWP);
  cudaError_t e = (cudaError_t)smem_at_least((const void *)k_resid_split, smem);
  if (e != cudaSuccess) return (int)e;
  const int64_t nmb = (n + 15) / 16;
  const unsigned grid = (unsigned)((nmb + SPL_WARPS / 2 - 1) / (SPL_WARPS / 2));
  k_resid_split<<<grid, SPL_WARPS * 32, smem, s>>>((const uint4 *)frag, rexp, nch, n, lo, xd, ldx, plane, xpad, nrhs,
                                                   F, R, norms, XWP);
  count_launch(3);
  return (int)cudaGetLastError();
}

}  // namespace spk
