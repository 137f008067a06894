"""Oracle for the recursive SPIKE banded solve -- TEST INFRASTRUCTURE ONLY.

What it is: the plain CPU FP64 definition of what the GPU path computes.
Recursive SPIKE is a direct method: A = D S (Sec. 2.1), so in exact arithmetic
it returns X = op(A)^{-1} F for any partition count p.  The oracle therefore
solves the banded system by Gaussian elimination with partial pivoting inside
the band (Sec. 5.1; pivot = first entry of greatest magnitude), with the
transpose option (Sec. 4: A^T X = F reusing the factors).  It also exposes the
non-pivoting LU and UL factorizations of Sec. 2.3, a dense GEPP cross-check, a
banded mat-vec for residuals, and (in sibling modules) an exact rational solver,
error metrics and a Hager/Higham condition estimator.

Who may use it: only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline.  The product (paper_1811_03559_gb300) never imports it and it never
imports the product.  The C code in oracle.c is compiled by build() (or on first
use) into oracle/liboracle.so.

Array conventions (NumPy, float64):
  band : shape (n, kl+ku+1), C-contiguous; band[j, ku+i-j] = A(i, j)
         (LAPACK band layout, column-major).
  F, X : shape (nrhs, n), C-contiguous; F[c, i] = F(i, c) (column-major n x nrhs).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lib = None


def build_oracle(force=False):
    """Compile oracle.c into liboracle.so with the host C compiler."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        i64, dp, ip, ch = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_char
        lib.oracle_gbtrf.argtypes = [i64, ip, ip, dp, i64, dp, i64, dp]
        lib.oracle_gbtrf.restype = i64
        lib.oracle_gbtrs.argtypes = [ch, i64, ip, ip, i64, dp, i64, dp, dp, i64]
        lib.oracle_gbtrs.restype = None
        for nm in ("oracle_lu_nopiv", "oracle_ul_nopiv"):
            getattr(lib, nm).argtypes = [i64, ip, ip, dp, i64]
            getattr(lib, nm).restype = i64
        for nm in ("oracle_lu_nopiv_solve", "oracle_ul_nopiv_solve"):
            getattr(lib, nm).argtypes = [ch, i64, ip, ip, i64, dp, i64, dp, i64]
            getattr(lib, nm).restype = None
        lib.oracle_gbmv.argtypes = [ch, i64, ip, ip, i64, dp, i64, dp, i64, dp, i64]
        lib.oracle_gbmv.restype = None
        lib.oracle_dense_getrf.argtypes = [i64, dp, i64, dp]
        lib.oracle_dense_getrf.restype = i64
        lib.oracle_dense_getrs.argtypes = [ch, i64, i64, dp, i64, dp, dp, i64]
        lib.oracle_dense_getrs.restype = None
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _rhs(F, n):
    X = np.array(F, dtype=np.float64, order="C", copy=True)
    one = X.ndim == 1
    X = X.reshape(-1, n)
    return X, one


class BandLU:
    """P A = L U of a band matrix (GEPP inside the band), reusable for 'N' and 'T'."""

    def __init__(self, band, kl, ku):
        band = np.ascontiguousarray(band, dtype=np.float64)
        self.n, ldb = band.shape
        assert ldb >= kl + ku + 1
        self.kl, self.ku = kl, ku
        self.ldf = 2 * kl + ku + 1
        self.fac = np.zeros((self.n, self.ldf))
        self.ipiv = np.zeros(self.n, dtype=np.int64)
        self.info = _load().oracle_gbtrf(self.n, kl, ku, _ptr(band), ldb, _ptr(self.fac), self.ldf, _ptr(self.ipiv))

    def solve(self, F, trans="N"):
        X, one = _rhs(F, self.n)
        _load().oracle_gbtrs(trans.encode(), self.n, self.kl, self.ku, X.shape[0], _ptr(self.fac), self.ldf,
                             _ptr(self.ipiv), _ptr(X), self.n)
        return X[0] if one else X


def gbsv(band, kl, ku, F, trans="N"):
    """X = op(A)^{-1} F by banded GEPP.  Returns (X, info); info > 0 means singular."""
    lu = BandLU(band, kl, ku)
    return lu.solve(F, trans), lu.info


def nopiv_solve(band, kl, ku, F, trans="N", kind="LU"):
    """Solve with the non-pivoting banded LU (kind='LU') or UL (kind='UL') of Sec. 2.3."""
    ab = np.array(band, dtype=np.float64, order="C", copy=True)
    n, ldb = ab.shape
    lib = _load()
    info = (lib.oracle_lu_nopiv if kind == "LU" else lib.oracle_ul_nopiv)(n, kl, ku, _ptr(ab), ldb)
    X, one = _rhs(F, n)
    (lib.oracle_lu_nopiv_solve if kind == "LU" else lib.oracle_ul_nopiv_solve)(
        trans.encode(), n, kl, ku, X.shape[0], _ptr(ab), ldb, _ptr(X), n)
    return (X[0] if one else X), info


def nopiv_factor(band, kl, ku, kind="LU"):
    """Return the in-place non-pivoting factor band (LU: unit L below, U on/above; UL: unit U above, L on/below)."""
    ab = np.array(band, dtype=np.float64, order="C", copy=True)
    n, ldb = ab.shape
    lib = _load()
    info = (lib.oracle_lu_nopiv if kind == "LU" else lib.oracle_ul_nopiv)(n, kl, ku, _ptr(ab), ldb)
    return ab, info


def gbmv(band, kl, ku, X, trans="N"):
    """Y = op(A) X for the band (FP64, plain sums)."""
    band = np.ascontiguousarray(band, dtype=np.float64)
    n, ldb = band.shape
    Xc, one = _rhs(X, n)
    Y = np.zeros_like(Xc)
    _load().oracle_gbmv(trans.encode(), n, kl, ku, Xc.shape[0], _ptr(band), ldb, _ptr(Xc), n, _ptr(Y), n)
    return Y[0] if one else Y


def dense_solve(A, F, trans="N"):
    """Dense GEPP solve (cross-check only).  A is an (n, n) array with A[i, j] = A(i, j)."""
    n = A.shape[0]
    a = np.array(A.T, dtype=np.float64, order="C", copy=True)  # column-major storage
    ipiv = np.zeros(n, dtype=np.int64)
    lib = _load()
    info = lib.oracle_dense_getrf(n, _ptr(a), n, _ptr(ipiv))
    X, one = _rhs(F, n)
    lib.oracle_dense_getrs(trans.encode(), n, X.shape[0], _ptr(a), n, _ptr(ipiv), _ptr(X), n)
    return (X[0] if one else X), info


def band_to_dense(band, kl, ku):
    """Dense n x n copy of a band (tiny n only)."""
    n = band.shape[0]
    A = np.zeros((n, n))
    for j in range(n):
        for i in range(max(0, j - ku), min(n, j + kl + 1)):
            A[i, j] = band[j, ku + i - j]
    return A
