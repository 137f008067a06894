/*
 * Oracle for the banded solve AX = F / A^T X = F  -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the plain, slow, obviously-correct CPU definition of what the
 * GPU SPIKE path computes.  In exact arithmetic recursive SPIKE returns
 * X = op(A)^{-1} F for every partition count p (it is a direct method:
 * A = D S, Sec. 2.1, Eqs. "Dstage"/"Sstage"), so the oracle is that definition:
 * banded Gaussian elimination with partial pivoting (the LAPACK-style banded
 * solver the paper wants SPIKE to replace, Sec. 1 and Sec. 5, where the pivot
 * is the entry of greatest magnitude in the column, searched only inside the
 * band, so a row moves at most kl places, Sec. 5.1).  It also carries the
 * non-pivoting banded LU and UL factorizations of Sec. 2.3 (LU for every
 * partition but the last, UL for the last), and a dense GEPP used only to
 * cross-check the banded code on tiny systems.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
 * this code.  It shares nothing with the CUDA path (no header, no helper, no
 * constant), and nothing here calls into the product.  Everything is FP64, no
 * blocking, no reordering: one column (or row) at a time in the textbook order.
 *
 * Storage conventions (column-major, 0-based):
 *   input band  : A(i,j) at band[j*ldb + ku + i - j], ldb >= kl+ku+1
 *                 (LAPACK band layout; entries outside the matrix are ignored)
 *   GEPP factor : A(i,j) at fac[j*ldf + kl + ku + i - j], ldf >= 2*kl+ku+1;
 *                 the top kl rows receive the fill of U caused by row swaps.
 *   dense       : A(i,j) at a[j*lda + i]
 *   RHS         : b[c*ldx + i], overwritten by the solution.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

static inline int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }
static inline int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

/* ------------------------------------------------------------------ GEPP -- */

#define FAC(i, j) fac[(j) * ldf + kl + ku + (i) - (j)]

/* Copy the input band into GEPP storage (fill rows zeroed), then factor
 * P A = L U by Gaussian elimination with partial pivoting.  ipiv[j] is the row
 * swapped with row j at step j.  Ties in |a_ij| keep the first (topmost) row.
 * Returns 0, or j+1 for the first column j whose pivot candidates are all zero
 * (that column is then left unscaled and elimination continues). */
int64_t oracle_gbtrf(int64_t n, int kl, int ku, const double *band, int64_t ldb, double *fac, int64_t ldf,
                     int64_t *ipiv) {
  int64_t info = 0;
  for (int64_t j = 0; j < n; ++j) {
    memset(&fac[j * ldf], 0, sizeof(double) * (size_t)ldf);
    for (int64_t i = imax64(0, j - ku); i <= imin64(n - 1, j + kl); ++i) FAC(i, j) = band[j * ldb + ku + i - j];
  }
  for (int64_t j = 0; j < n; ++j) {
    int64_t last = imin64(n - 1, j + kl);
    int64_t p = j;
    double amax = fabs(FAC(j, j));
    for (int64_t i = j + 1; i <= last; ++i) {
      if (fabs(FAC(i, j)) > amax) {
        amax = fabs(FAC(i, j));
        p = i;
      }
    }
    ipiv[j] = p;
    if (amax == 0.0) {
      if (info == 0) info = j + 1;
      continue;
    }
    int64_t cmax = imin64(n - 1, j + kl + ku);
    if (p != j) {
      for (int64_t c = j; c <= cmax; ++c) {
        double t = FAC(j, c);
        FAC(j, c) = FAC(p, c);
        FAC(p, c) = t;
      }
    }
    double piv = FAC(j, j);
    for (int64_t i = j + 1; i <= last; ++i) FAC(i, j) = FAC(i, j) / piv;
    for (int64_t c = j + 1; c <= cmax; ++c) {
      double u = FAC(j, c);
      if (u == 0.0) continue;
      for (int64_t i = j + 1; i <= last; ++i) FAC(i, c) -= FAC(i, j) * u;
    }
  }
  return info;
}

/* Solve op(A) X = B with the factors of oracle_gbtrf.  trans 'N' or 'T'. */
void oracle_gbtrs(char trans, int64_t n, int kl, int ku, int64_t nrhs, const double *fac, int64_t ldf,
                  const int64_t *ipiv, double *b, int64_t ldx) {
  for (int64_t r = 0; r < nrhs; ++r) {
    double *x = &b[r * ldx];
    if (trans == 'N' || trans == 'n') {
      /* x <- L^{-1} P x : interchange then eliminate, column by column. */
      for (int64_t j = 0; j < n; ++j) {
        int64_t p = ipiv[j];
        if (p != j) {
          double t = x[j];
          x[j] = x[p];
          x[p] = t;
        }
        for (int64_t i = j + 1; i <= imin64(n - 1, j + kl); ++i) x[i] -= FAC(i, j) * x[j];
      }
      /* x <- U^{-1} x : U has kl+ku superdiagonals. */
      for (int64_t j = n - 1; j >= 0; --j) {
        x[j] = x[j] / FAC(j, j);
        for (int64_t i = imax64(0, j - kl - ku); i < j; ++i) x[i] -= FAC(i, j) * x[j];
      }
    } else {
      /* A = P_0 L_0^{-1} ... P_{n-1} L_{n-1}^{-1} U, so A^T x = b is
       * U^T y = b followed by x = P_0 L_0^T ( ... (P_{n-1} L_{n-1}^T y)). */
      for (int64_t j = 0; j < n; ++j) {
        double s = x[j];
        for (int64_t i = imax64(0, j - kl - ku); i < j; ++i) s -= FAC(i, j) * x[i];
        x[j] = s / FAC(j, j);
      }
      for (int64_t j = n - 1; j >= 0; --j) {
        double s = x[j];
        for (int64_t i = j + 1; i <= imin64(n - 1, j + kl); ++i) s -= FAC(i, j) * x[i];
        x[j] = s;
        int64_t p = ipiv[j];
        if (p != j) {
          double t = x[j];
          x[j] = x[p];
          x[p] = t;
        }
      }
    }
  }
}
#undef FAC

/* ------------------------------------------- non-pivoting LU and UL (Sec. 2.3) */

#define AB(i, j) ab[(j) * ldb + ku + (i) - (j)]

/* In-place banded LU without pivoting: A = L U, L unit lower (multipliers stored
 * below the diagonal), U upper.  Returns 0 or j+1 at the first zero pivot. */
int64_t oracle_lu_nopiv(int64_t n, int kl, int ku, double *ab, int64_t ldb) {
  for (int64_t j = 0; j < n; ++j) {
    double piv = AB(j, j);
    if (piv == 0.0) return j + 1;
    for (int64_t i = j + 1; i <= imin64(n - 1, j + kl); ++i) {
      double m = AB(i, j) / piv;
      AB(i, j) = m;
      for (int64_t c = j + 1; c <= imin64(n - 1, j + ku); ++c) AB(i, c) -= m * AB(j, c);
    }
  }
  return 0;
}

void oracle_lu_nopiv_solve(char trans, int64_t n, int kl, int ku, int64_t nrhs, const double *ab, int64_t ldb,
                           double *b, int64_t ldx) {
  for (int64_t r = 0; r < nrhs; ++r) {
    double *x = &b[r * ldx];
    if (trans == 'N' || trans == 'n') {
      for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j + 1; i <= imin64(n - 1, j + kl); ++i) x[i] -= AB(i, j) * x[j];
      for (int64_t j = n - 1; j >= 0; --j) {
        x[j] = x[j] / AB(j, j);
        for (int64_t i = imax64(0, j - ku); i < j; ++i) x[i] -= AB(i, j) * x[j];
      }
    } else {
      for (int64_t j = 0; j < n; ++j) { /* U^T z = b */
        double s = x[j];
        for (int64_t i = imax64(0, j - ku); i < j; ++i) s -= AB(i, j) * x[i];
        x[j] = s / AB(j, j);
      }
      for (int64_t j = n - 1; j >= 0; --j) { /* L^T x = z */
        double s = x[j];
        for (int64_t i = j + 1; i <= imin64(n - 1, j + kl); ++i) s -= AB(i, j) * x[i];
        x[j] = s;
      }
    }
  }
}

/* In-place banded UL without pivoting: A = U L, U unit upper (multipliers stored
 * above the diagonal), L lower with the diagonal.  Elimination runs from the
 * last column upward (the factorization used for the last partition, Sec. 2.3). */
int64_t oracle_ul_nopiv(int64_t n, int kl, int ku, double *ab, int64_t ldb) {
  for (int64_t j = n - 1; j >= 0; --j) {
    double piv = AB(j, j);
    if (piv == 0.0) return j + 1;
    for (int64_t i = imax64(0, j - ku); i < j; ++i) {
      double m = AB(i, j) / piv;
      AB(i, j) = m;
      for (int64_t c = imax64(0, j - kl); c < j; ++c) AB(i, c) -= m * AB(j, c);
    }
  }
  return 0;
}

void oracle_ul_nopiv_solve(char trans, int64_t n, int kl, int ku, int64_t nrhs, const double *ab, int64_t ldb,
                           double *b, int64_t ldx) {
  for (int64_t r = 0; r < nrhs; ++r) {
    double *x = &b[r * ldx];
    if (trans == 'N' || trans == 'n') {
      for (int64_t j = n - 1; j >= 0; --j) /* U y = b, U unit upper */
        for (int64_t i = imax64(0, j - ku); i < j; ++i) x[i] -= AB(i, j) * x[j];
      for (int64_t j = 0; j < n; ++j) { /* L x = y */
        double s = x[j];
        for (int64_t c = imax64(0, j - kl); c < j; ++c) s -= AB(j, c) * x[c];
        x[j] = s / AB(j, j);
      }
    } else {
      for (int64_t j = n - 1; j >= 0; --j) { /* L^T z = b */
        double s = x[j];
        for (int64_t i = j + 1; i <= imin64(n - 1, j + kl); ++i) s -= AB(i, j) * x[i];
        x[j] = s / AB(j, j);
      }
      for (int64_t j = 0; j < n; ++j) { /* U^T x = z */
        double s = x[j];
        for (int64_t i = imax64(0, j - ku); i < j; ++i) s -= AB(i, j) * x[i];
        x[j] = s;
      }
    }
  }
}

/* y = op(A) x for the input band (plain sums in row/column order). */
void oracle_gbmv(char trans, int64_t n, int kl, int ku, int64_t nrhs, const double *ab, int64_t ldb,
                 const double *x, int64_t ldx, double *y, int64_t ldy) {
  for (int64_t r = 0; r < nrhs; ++r) {
    const double *xr = &x[r * ldx];
    double *yr = &y[r * ldy];
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      if (trans == 'N' || trans == 'n') {
        for (int64_t j = imax64(0, i - kl); j <= imin64(n - 1, i + ku); ++j) s += AB(i, j) * xr[j];
      } else {
        for (int64_t j = imax64(0, i - ku); j <= imin64(n - 1, i + kl); ++j) s += AB(j, i) * xr[j];
      }
      yr[i] = s;
    }
  }
}
#undef AB

/* ------------------------------------------------ dense GEPP (cross-check) -- */

int64_t oracle_dense_getrf(int64_t n, double *a, int64_t lda, int64_t *ipiv) {
  int64_t info = 0;
  for (int64_t j = 0; j < n; ++j) {
    int64_t p = j;
    double amax = fabs(a[j * lda + j]);
    for (int64_t i = j + 1; i < n; ++i)
      if (fabs(a[j * lda + i]) > amax) {
        amax = fabs(a[j * lda + i]);
        p = i;
      }
    ipiv[j] = p;
    if (amax == 0.0) {
      if (info == 0) info = j + 1;
      continue;
    }
    if (p != j)
      for (int64_t c = 0; c < n; ++c) {
        double t = a[c * lda + j];
        a[c * lda + j] = a[c * lda + p];
        a[c * lda + p] = t;
      }
    for (int64_t i = j + 1; i < n; ++i) a[j * lda + i] = a[j * lda + i] / a[j * lda + j];
    for (int64_t c = j + 1; c < n; ++c) {
      double u = a[c * lda + j];
      if (u == 0.0) continue;
      for (int64_t i = j + 1; i < n; ++i) a[c * lda + i] -= a[j * lda + i] * u;
    }
  }
  return info;
}

void oracle_dense_getrs(char trans, int64_t n, int64_t nrhs, const double *a, int64_t lda, const int64_t *ipiv,
                        double *b, int64_t ldx) {
  for (int64_t r = 0; r < nrhs; ++r) {
    double *x = &b[r * ldx];
    if (trans == 'N' || trans == 'n') {
      for (int64_t j = 0; j < n; ++j) { /* whole-row swaps were applied to L too */
        int64_t p = ipiv[j];
        if (p != j) {
          double t = x[j];
          x[j] = x[p];
          x[p] = t;
        }
      }
      for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j + 1; i < n; ++i) x[i] -= a[j * lda + i] * x[j];
      for (int64_t j = n - 1; j >= 0; --j) {
        x[j] = x[j] / a[j * lda + j];
        for (int64_t i = 0; i < j; ++i) x[i] -= a[j * lda + i] * x[j];
      }
    } else {
      for (int64_t j = 0; j < n; ++j) {
        double s = x[j];
        for (int64_t i = 0; i < j; ++i) s -= a[j * lda + i] * x[i];
        x[j] = s / a[j * lda + j];
      }
      for (int64_t j = n - 1; j >= 0; --j) {
        double s = x[j];
        for (int64_t i = j + 1; i < n; ++i) s -= a[j * lda + i] * x[i];
        x[j] = s;
      }
      for (int64_t j = n - 1; j >= 0; --j) {
        int64_t p = ipiv[j];
        if (p != j) {
          double t = x[j];
          x[j] = x[p];
          x[p] = t;
        }
      }
    }
  }
}
