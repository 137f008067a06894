"""Thin ctypes binding of libspike.so (C ABI in include/spike.h).

Argument marshalling only: every step of the factorization and solves runs in
the library's CUDA kernels.  If libspike.so is missing, or no GPU is present,
calls raise -- there is no CPU fallback.

Arrays: `band` has shape (n, kl+ku+1) (LAPACK band layout, column-major), and
right-hand sides have shape (nrhs, n) or (n,), row-contiguous (column-major
n x nrhs).  They may be CUDA torch tensors (used in place, on the current torch
stream) or NumPy arrays (host memory; the library stages them through the GPU).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspike.so")
_lib = None

SPIKE_ENOMEM, SPIKE_ECUDA, SPIKE_EHANDLE, SPIKE_ENOTSUP, SPIKE_ENOGPU = -1001, -1002, -1003, -1004, -1005


class SpikeInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("kl", ctypes.c_int32), ("ku", ctypes.c_int32), ("k", ctypes.c_int32),
                ("p_requested", ctypes.c_int32), ("p_effective", ctypes.c_int32), ("m", ctypes.c_int32),
                ("P", ctypes.c_int32), ("r", ctypes.c_int32), ("leaves", ctypes.c_int32),
                ("levels", ctypes.c_int32), ("pivot", ctypes.c_int32), ("n1", ctypes.c_int64),
                ("n2", ctypes.c_int64), ("n3", ctypes.c_int64), ("R12", ctypes.c_double), ("R13", ctypes.c_double),
                ("K", ctypes.c_double), ("boosts", ctypes.c_int64), ("zero_pivot_col", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("mixed", ctypes.c_int32), ("refine_steps", ctypes.c_int32),
                ("refine_berr", ctypes.c_double), ("graph_captures", ctypes.c_int64),
                ("graph_replays", ctypes.c_int64), ("numerics", ctypes.c_int32), ("reserved0", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved0"}


class TuneResult(ctypes.Structure):
    _fields_ = [("K_measured", ctypes.c_double), ("best_p", ctypes.c_int32), ("best_mode", ctypes.c_int32),
                ("best_R13", ctypes.c_double), ("best_ms", ctypes.c_double), ("default_ms", ctypes.c_double),
                ("tried", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class SpikeOptions(ctypes.Structure):
    _fields_ = [("K", ctypes.c_double), ("nrhs_hint", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("R13", ctypes.c_double), ("refine_tol", ctypes.c_double),
                ("reserved", ctypes.c_int64 * 2)]


EXPORTS = ["spike_plan", "spike_factor", "spike_factor_ex", "spike_solve", "spike_solve_ex", "spike_set_stream",
           "spike_get_info", "spike_get_tips", "spike_backward_error", "spike_get_timings", "spike_kernel_launches",
           "spike_free", "spike_strerror", "spike_last_cuda_error", "spike_backward_error_noalloc",
           "spike_measure_fp64_peak", "spike_factor_bytes", "spike_solve_workspace", "spike_solve_ws",
           "spike_measure_K", "spike_tune", "spike_solve_batch", "spike_solve_batch_workspace",
           "spike_release_cached", "spike_residual", "spike_factor_batch", "spike_measure_pipes"]
SPIKE_ELIMIT = -1006
NOALLOC_MAX_NRHS = 1024

FLAG_TIMING = 1
FLAG_STAGE_BALANCE = 2
FLAG_MIXED = 4
FLAG_BATCH_INVARIANT = 8
FLAG_BORROW_BAND = 16
FLAG_GRAPHS = 32
FLAG_FP64_RESIDUAL = 64
NUMERICS_NAN_PIVOT = 1
NUMERICS_SINGULAR_INTERFACE = 2
MIXED_TOL = 1e-14
PIVOT_R13 = 1.5  # default partition ratio of pivoting factorizations (spike.h SPIKE_PIVOT_R13)
STAGES = ["factor", "setup", "block_lu", "spikes", "reduced", "solve_n", "solve_n_d", "solve_n_reduced",
          "solve_n_retrieval", "solve_t", "solve_t_s", "solve_t_reduced", "solve_t_d"]


class SpikeError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = "%s failed: %d (%s)" % (where, code, lib().spike_strerror(code).decode())
        if code == SPIKE_ECUDA:
            msg += ": " + lib().spike_last_cuda_error().decode()
        super().__init__(msg)


def lib():
    """Load libspike.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libspike.so not found at %s: run `python -m paper_1811_03559_gb300.build`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        i64, i32, vp, dp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p
        L.spike_plan.argtypes = [i64, i32, i32, i32, ctypes.POINTER(SpikeOptions), ctypes.POINTER(SpikeInfo), vp, vp]
        L.spike_factor.argtypes = [dp, i64, i32, i32, i32, i32, ctypes.POINTER(vp)]
        L.spike_factor_ex.argtypes = [dp, i64, i64, i32, i32, i32, i32, ctypes.POINTER(SpikeOptions),
                                      ctypes.POINTER(vp)]
        L.spike_solve.argtypes = [vp, dp, i32, ctypes.c_char]
        L.spike_solve_ex.argtypes = [vp, dp, i64, i32, ctypes.c_char]
        L.spike_set_stream.argtypes = [vp, vp]
        L.spike_get_info.argtypes = [vp, ctypes.POINTER(SpikeInfo)]
        L.spike_get_tips.argtypes = [vp, i32, dp]
        L.spike_backward_error.argtypes = [dp, i64, i64, i32, i32, dp, dp, i32, ctypes.c_char, vp, dp]
        L.spike_backward_error_noalloc.argtypes = [dp, i64, i64, i32, i32, dp, dp, i32, ctypes.c_char, vp, dp]
        L.spike_get_timings.argtypes = [vp, dp, i32]
        L.spike_measure_fp64_peak.argtypes = [vp, dp]
        L.spike_measure_pipes.argtypes = [vp, dp, i32]
        L.spike_factor_bytes.argtypes = [i64, i32, i32, i32, i32, ctypes.POINTER(SpikeOptions), i32,
                                         ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.spike_solve_workspace.argtypes = [vp, i32, ctypes.c_char, i32, ctypes.POINTER(i64)]
        L.spike_solve_ws.argtypes = [vp, dp, i64, i32, ctypes.c_char, vp, i64]
        L.spike_measure_K.argtypes = [dp, i64, i64, i32, i32, vp, ctypes.POINTER(ctypes.c_double)]
        L.spike_solve_batch.argtypes = [vp, vp, vp, i32, ctypes.c_char, vp, vp, i64]
        L.spike_release_cached.argtypes = [ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.spike_residual.argtypes = [vp, dp, dp, dp, i32, ctypes.c_char, dp]
        L.spike_factor_batch.argtypes = [vp, vp, vp, vp, vp, vp, i32, ctypes.POINTER(SpikeOptions), vp]
        L.spike_solve_batch_workspace.argtypes = [vp, vp, i32, ctypes.c_char, ctypes.POINTER(i64)]
        L.spike_tune.argtypes = [dp, i64, i64, i32, i32, i32, i32, vp, i32, vp, i32, vp, vp,
                                 ctypes.POINTER(TuneResult)]
        L.spike_kernel_launches.argtypes = []
        L.spike_kernel_launches.restype = ctypes.c_int64
        L.spike_free.argtypes = [vp]
        L.spike_free.restype = None
        L.spike_strerror.argtypes = [i32]
        L.spike_strerror.restype = ctypes.c_char_p
        L.spike_last_cuda_error.argtypes = []
        L.spike_last_cuda_error.restype = ctypes.c_char_p
        for nm in EXPORTS:
            f = getattr(L, nm)
            if nm not in ("spike_free", "spike_strerror", "spike_last_cuda_error", "spike_kernel_launches"):
                f.restype = ctypes.c_int
        _lib = L
    return _lib


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if _is_torch(x):
        if not (x.is_contiguous() and str(x.dtype) == "torch.float64"):
            raise ValueError("expected a contiguous float64 tensor, got %s %s" % (x.dtype, tuple(x.stride())))
        return ctypes.c_void_p(x.data_ptr())
    if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags["C_CONTIGUOUS"]):
        raise ValueError("expected a C-contiguous float64 array or a CUDA float64 tensor")
    return x.ctypes.data_as(ctypes.c_void_p)


def _check_rhs(F, n):
    if F.ndim not in (1, 2) or F.shape[-1] != n:
        raise ValueError("right-hand sides must have shape (nrhs, %d) or (%d,), got %s" % (n, n, tuple(F.shape)))
    return 1 if F.ndim == 1 else F.shape[0]


def _torch_stream(x):
    if _is_torch(x) and x.is_cuda:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
    return ctypes.c_void_p(0)


def plan(n, kl, ku, p, K=0.0, nrhs_hint=0, stage_balance=False, R13=0.0):
    """Partition plan (Sec. 3.1, 3.3) without a GPU: (info dict, block offsets, block flags)."""
    info = SpikeInfo()
    opt = SpikeOptions(K=K, nrhs_hint=nrhs_hint, flags=FLAG_STAGE_BALANCE if stage_balance else 0, R13=R13)
    offs = np.zeros(p + 2, dtype=np.int64)
    flags = np.zeros(p + 2, dtype=np.int32)
    rc = lib().spike_plan(n, kl, ku, p, ctypes.byref(opt), ctypes.byref(info), offs.ctypes.data_as(ctypes.c_void_p),
                          flags.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise SpikeError(rc, "spike_plan")
    nb = info.leaves
    return info.as_dict(), offs[: nb + 1].copy(), flags[:nb].copy()


class Factorization:
    """A SPIKE factorization handle (spike_factor_ex); free with .free() or by garbage collection."""

    def __init__(self, band, kl, ku, p, pivot=0, K=0.0, nrhs_hint=0, stream=None, timing=False, n=None,
                 stage_balance=False, mixed=False, batch_invariant=False, R13=0.0, borrow_band=False,
                 refine_tol=0.0, graphs=False, fp64_residual=False):
        rows, ldab = band.shape
        self.n, self.kl, self.ku = (rows if n is None else n), kl, ku
        n = self.n
        s = _torch_stream(band) if stream is None else ctypes.c_void_p(stream)
        flags = (FLAG_TIMING if timing else 0) | (FLAG_STAGE_BALANCE if stage_balance else 0) | \
            (FLAG_MIXED if mixed else 0) | (FLAG_BATCH_INVARIANT if batch_invariant else 0) | \
            (FLAG_BORROW_BAND if borrow_band else 0) | (FLAG_GRAPHS if graphs else 0) | \
            (FLAG_FP64_RESIDUAL if fp64_residual else 0)
        self._opt = SpikeOptions(K=K, nrhs_hint=nrhs_hint, flags=flags, stream=s, R13=R13, refine_tol=refine_tol)
        # a borrowed device band is read by every mixed-precision solve until spike_free
        self._borrowed = band if borrow_band else None
        h = ctypes.c_void_p()
        rc = lib().spike_factor_ex(_ptr(band), ldab, n, kl, ku, p, pivot, ctypes.byref(self._opt), ctypes.byref(h))
        self._h = h
        self.status = rc
        if rc < 0:
            raise SpikeError(rc, "spike_factor_ex")

    @classmethod
    def _adopt(cls, h, n, kl, ku, opt):
        """Wrap a handle made by spike_factor_batch."""
        self = cls.__new__(cls)
        self.n, self.kl, self.ku = n, kl, ku
        self._opt, self._borrowed, self._h, self.status = opt, None, ctypes.c_void_p(h), 0
        return self

    def solve(self, F, trans="N"):
        """Overwrite F (shape (nrhs, n) or (n,)) with op(A)^{-1} F.  Returns F."""
        nrhs = _check_rhs(F, self.n)
        rc = lib().spike_solve_ex(self._h, _ptr(F), self.n, nrhs, trans.encode())
        if rc != 0:
            raise SpikeError(rc, "spike_solve_ex")
        return F

    def residual(self, X, F, R, trans="N"):
        """R = F - op(A) X with the tensor-core residual of a mixed-precision handle
        (spike_residual; device tensors of shape (nrhs, n)).  Returns the per-column
        backward errors."""
        nrhs = _check_rhs(X, self.n)
        out = np.zeros(nrhs)
        rc = lib().spike_residual(self._h, _ptr(X), _ptr(F), _ptr(R), nrhs, trans.encode(),
                                  out.ctypes.data_as(ctypes.c_void_p))
        if rc != 0:
            raise SpikeError(rc, "spike_residual")
        return out

    def workspace_bytes(self, nrhs, trans="N", host_f=False):
        """Device scratch that solve_ws needs for nrhs columns (spike_solve_workspace)."""
        out = ctypes.c_int64(0)
        rc = lib().spike_solve_workspace(self._h, nrhs, trans.encode(), 1 if host_f else 0, ctypes.byref(out))
        if rc != 0:
            raise SpikeError(rc, "spike_solve_workspace")
        return out.value

    def solve_ws(self, F, workspace, trans="N"):
        """solve() on caller-provided device scratch (a CUDA uint8 tensor of workspace_bytes)."""
        nrhs = _check_rhs(F, self.n)
        rc = lib().spike_solve_ws(self._h, _ptr(F), self.n, nrhs, trans.encode(),
                                  ctypes.c_void_p(workspace.data_ptr()), workspace.numel() * workspace.element_size())
        if rc != 0:
            raise SpikeError(rc, "spike_solve_ws")
        return F

    def set_stream(self, stream):
        rc = lib().spike_set_stream(self._h, ctypes.c_void_p(stream))
        if rc != 0:
            raise SpikeError(rc, "spike_set_stream")

    def info(self):
        out = SpikeInfo()
        rc = lib().spike_get_info(self._h, ctypes.byref(out))
        if rc != 0:
            raise SpikeError(rc, "spike_get_info")
        return out.as_dict()

    def timings(self):
        """Stage times (ms) of the last factor / N solve / T solve (handle created with timing=True)."""
        out = np.zeros(len(STAGES))
        rc = lib().spike_get_timings(self._h, out.ctypes.data_as(ctypes.c_void_p), len(STAGES))
        if rc != 0:
            raise SpikeError(rc, "spike_get_timings")
        return dict(zip(STAGES, out.tolist()))

    def tips(self, level=0):
        """Spike tips of a merge level: array (leaves, 4, k, k) with [V_t, V_b, W_t, W_b]."""
        inf = self.info()
        out = np.zeros((inf["leaves"], 4, inf["k"], inf["k"]))
        rc = lib().spike_get_tips(self._h, level, out.ctypes.data_as(ctypes.c_void_p))
        if rc != 0:
            raise SpikeError(rc, "spike_get_tips")
        return out

    def free(self):
        if self._h:
            lib().spike_free(self._h)
            self._h = ctypes.c_void_p()
        self._borrowed = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def measure_fp64_peak(stream=None):
    """Measured FP64 FMA throughput of the current GPU in TFLOP/s (library probe kernel)."""
    out = ctypes.c_double(0.0)
    rc = lib().spike_measure_fp64_peak(ctypes.c_void_p(stream or 0), ctypes.byref(out))
    if rc != 0:
        raise SpikeError(rc, "spike_measure_fp64_peak")
    return out.value


PIPE_KEYS = ("dfma_tflops", "dmma_tflops", "fp32_fma_tflops", "bf16_mma_sync_tflops",
             "dfma_even_warps_ms", "dmma_odd_warps_ms", "both_alternate_warps_ms")


def measure_pipes(stream=None):
    """Throughput probes of the FP64 FMA, FP64 MMA, FP32 FMA and bf16 MMA pipes and the
    DFMA/DMMA shared-pipe experiment (spike_measure_pipes), as a dict."""
    out = np.zeros(len(PIPE_KEYS))
    rc = lib().spike_measure_pipes(ctypes.c_void_p(stream or 0), out.ctypes.data_as(ctypes.c_void_p), len(PIPE_KEYS))
    if rc != 0:
        raise SpikeError(rc, "spike_measure_pipes")
    return dict(zip(PIPE_KEYS, out.tolist()))


def kernel_launches():
    """Kernels launched by libspike.so in this process so far."""
    return int(lib().spike_kernel_launches())


def factor_bytes(n, kl, ku, p, pivot=0, mixed=False, host_band=False, K=0.0, nrhs_hint=0, stage_balance=False,
                 borrow_band=False, fp64_residual=False):
    """(resident, transient) device bytes of a factorization, computed without a GPU."""
    flags = (FLAG_STAGE_BALANCE if stage_balance else 0) | (FLAG_MIXED if mixed else 0) | \
        (FLAG_BORROW_BAND if borrow_band else 0) | (FLAG_FP64_RESIDUAL if fp64_residual else 0)
    opt = SpikeOptions(K=K, nrhs_hint=nrhs_hint, flags=flags)
    res, tr = ctypes.c_int64(0), ctypes.c_int64(0)
    rc = lib().spike_factor_bytes(n, kl, ku, p, pivot, ctypes.byref(opt), 1 if host_band else 0, ctypes.byref(res),
                                  ctypes.byref(tr))
    if rc != 0:
        raise SpikeError(rc, "spike_factor_bytes")
    return res.value, tr.value


def release_cached():
    """Return the library pools' cached device memory to the driver: (reserved before, after)."""
    a, b = ctypes.c_int64(0), ctypes.c_int64(0)
    rc = lib().spike_release_cached(ctypes.byref(a), ctypes.byref(b))
    if rc != 0:
        raise SpikeError(rc, "spike_release_cached")
    return a.value, b.value


def measure_K(band, kl, ku):
    """The load-balancing constant K (Sec. 3.3) measured on the leading block of a device band."""
    n, ldab = band.shape
    out = ctypes.c_double(0.0)
    rc = lib().spike_measure_K(_ptr(band), ldab, n, kl, ku, _torch_stream(band), ctypes.byref(out))
    if rc != 0:
        raise SpikeError(rc, "spike_measure_K")
    return out.value


def tune(band, kl, ku, nrhs, p_candidates, r13_candidates=(), nsolves=2):
    """spike_tune: (result dict, table ms array of shape (len(p_candidates), 2 + len(r13_candidates)))."""
    n, ldab = band.shape
    ps = np.asarray(p_candidates, dtype=np.int32)
    rs = np.asarray(r13_candidates, dtype=np.float64)
    table = np.zeros((len(ps), 2 + len(rs)))
    res = TuneResult()
    rc = lib().spike_tune(_ptr(band), ldab, n, kl, ku, nrhs, nsolves, ps.ctypes.data_as(ctypes.c_void_p), len(ps),
                          rs.ctypes.data_as(ctypes.c_void_p) if len(rs) else None, len(rs), _torch_stream(band),
                          table.ctypes.data_as(ctypes.c_void_p), ctypes.byref(res))
    if rc != 0:
        raise SpikeError(rc, "spike_tune")
    return res.as_dict(), table


def solve_batch(facs, Fs, trans="N", workspace=None):
    """spike_solve_batch: overwrite every device tensor Fs[i] (shape (nrhs_i, n_i)) with
    op(A_i)^{-1} Fs[i], all systems stage by stage in shared launches.  Returns the
    workspace tensor (reusable for the same shapes)."""
    import torch
    cnt = len(facs)
    hs = (ctypes.c_void_p * cnt)(*[f._h.value for f in facs])
    ptrs = (ctypes.c_void_p * cnt)(*[F.data_ptr() for F in Fs])
    nr = (ctypes.c_int * cnt)(*[1 if F.ndim == 1 else F.shape[0] for F in Fs])
    for f, F in zip(facs, Fs):
        if not (F.is_cuda and F.is_contiguous()):
            raise ValueError("solve_batch takes contiguous CUDA tensors")
        _check_rhs(F, f.n)
    need = ctypes.c_int64(0)
    rc = lib().spike_solve_batch_workspace(hs, nr, cnt, trans.encode(), ctypes.byref(need))
    if rc != 0:
        raise SpikeError(rc, "spike_solve_batch_workspace")
    if workspace is None or workspace.numel() < need.value:
        workspace = torch.empty(max(need.value, 1), dtype=torch.uint8, device=Fs[0].device)
    rc = lib().spike_solve_batch(hs, ptrs, nr, cnt, trans.encode(), _torch_stream(Fs[0]),
                                 ctypes.c_void_p(workspace.data_ptr()), workspace.numel())
    if rc != 0:
        raise SpikeError(rc, "spike_solve_batch")
    return workspace


def factor_batch(bands, kls, kus, ps, nrhs_hint=0, stage_balance=False, batch_invariant=False):
    """spike_factor_batch: factor several device bands (torch tensors (n_i, kl_i+ku_i+1)) together,
    their blocks in one launch and their reduced systems level by level.  Returns one
    Factorization per band."""
    cnt = len(bands)
    for b in bands:
        if not (_is_torch(b) and b.is_cuda):
            raise ValueError("factor_batch takes CUDA tensors")
    ptrs = (ctypes.c_void_p * cnt)(*[b.data_ptr() for b in bands])
    ld = (ctypes.c_int64 * cnt)(*[b.shape[1] for b in bands])
    ns = (ctypes.c_int64 * cnt)(*[b.shape[0] for b in bands])
    kl_ = (ctypes.c_int * cnt)(*kls)
    ku_ = (ctypes.c_int * cnt)(*kus)
    p_ = (ctypes.c_int * cnt)(*ps)
    flags = (FLAG_STAGE_BALANCE if stage_balance else 0) | (FLAG_BATCH_INVARIANT if batch_invariant else 0)
    opt = SpikeOptions(nrhs_hint=nrhs_hint, flags=flags, stream=_torch_stream(bands[0]))
    out = (ctypes.c_void_p * cnt)()
    rc = lib().spike_factor_batch(ptrs, ld, ns, kl_, ku_, p_, cnt, ctypes.byref(opt), out)
    if rc != 0:
        raise SpikeError(rc, "spike_factor_batch")
    return [Factorization._adopt(out[i], bands[i].shape[0], kls[i], kus[i], opt) for i in range(cnt)]


def factor(band, kl, ku, p, pivot=0, **kw):
    return Factorization(band, kl, ku, p, pivot, **kw)


def backward_error(band, kl, ku, X, F, trans="N"):
    """Per-column backward error on the GPU (device torch tensors)."""
    n, ldab = band.shape
    nrhs = 1 if X.ndim == 1 else X.shape[0]
    out = np.zeros(nrhs)
    rc = lib().spike_backward_error(_ptr(band), ldab, n, kl, ku, _ptr(X), _ptr(F), nrhs, trans.encode(),
                                    _torch_stream(X), out.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise SpikeError(rc, "spike_backward_error")
    return out


def backward_error_noalloc(band, kl, ku, X, F, trans="N"):
    """As backward_error, through the entry point that allocates nothing (fixed device scratch,
    nrhs <= NOALLOC_MAX_NRHS; calls whose GPU work overlaps must not share it)."""
    n, ldab = band.shape
    nrhs = 1 if X.ndim == 1 else X.shape[0]
    out = np.zeros(nrhs)
    rc = lib().spike_backward_error_noalloc(_ptr(band), ldab, n, kl, ku, _ptr(X), _ptr(F), nrhs, trans.encode(),
                                            _torch_stream(X), out.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise SpikeError(rc, "spike_backward_error_noalloc")
    return out
