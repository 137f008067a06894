"""Thin ctypes binding of the serving engine in libspike.so (C ABI in include/spike_serve.h).

Argument marshalling only: admission, eviction, batching and the solves run in the
library (native worker threads driving CUDA streams).  Arrays follow spike.py: a band
of shape (n, kl+ku+1), right-hand sides of shape (nrhs, n) or (n,), FP64, contiguous;
NumPy arrays (host; pinned buffers copy fastest) or CUDA torch tensors.  The caller
keeps every band, F and X alive until the server is destroyed / the request is done.
"""
import ctypes

import numpy as np

from . import spike

DRYRUN = 1
GRAPHS = 2
TUNED = 4
FP64_RESIDUAL = 8  # SPIKE_SERVE_FP64_RESIDUAL
EVICT_LRU, EVICT_COST = 0, 1


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("streams", ctypes.c_int32), ("max_batch_rhs", ctypes.c_int32),
                ("p", ctypes.c_int32), ("nrhs_hint", ctypes.c_int32), ("K", ctypes.c_double),
                ("flags", ctypes.c_int32), ("dryrun_factor_us", ctypes.c_int32),
                ("dryrun_solve_us", ctypes.c_int32), ("batch_systems", ctypes.c_int32),
                ("evict_policy", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("rhs", ctypes.c_int64), ("factorizations", ctypes.c_int64),
                ("evictions", ctypes.c_int64), ("admission_waits", ctypes.c_int64),
                ("used_bytes", ctypes.c_int64), ("peak_bytes", ctypes.c_int64), ("resident", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("multi_solves", ctypes.c_int64), ("max_systems", ctypes.c_int32),
                ("tuned_classes", ctypes.c_int32), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("mean_ms", ctypes.c_double), ("span_s", ctypes.c_double),
                ("solves_per_s", ctypes.c_double), ("rhs_per_s", ctypes.c_double),
                ("graph_replays", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_bound = False


def _lib():
    global _bound
    L = spike.lib()
    if not _bound:
        i64, i32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        L.spike_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
        L.spike_server_create.restype = i32
        L.spike_server_add_matrix.argtypes = [vp, i64, vp, i64, i64, i32, i32, i32]
        L.spike_server_add_matrix.restype = i32
        L.spike_server_submit.argtypes = [vp, i64, vp, vp, i32, ctypes.c_char, i32]
        L.spike_server_submit.restype = i64
        L.spike_server_wait.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_double)]
        L.spike_server_wait.restype = i32
        L.spike_server_request_latency.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_double)]
        L.spike_server_request_latency.restype = i32
        L.spike_server_drain.argtypes = [vp]
        L.spike_server_drain.restype = i32
        L.spike_server_stats_get.argtypes = [vp, ctypes.POINTER(ServerStats)]
        L.spike_server_stats_get.restype = i32
        L.spike_server_latencies.argtypes = [vp, vp, i64, ctypes.POINTER(i64)]
        L.spike_server_latencies.restype = i32
        L.spike_server_last_error.argtypes = [vp]
        L.spike_server_last_error.restype = ctypes.c_char_p
        L.spike_server_destroy.argtypes = [vp]
        L.spike_server_destroy.restype = None
        _bound = True
    return L


class Server:
    """A spike_server: resident factorizations under `budget_bytes`, `streams` workers,
    up to `max_batch_rhs` right-hand sides merged per solve; `evict` is "lru" (least
    recently used first) or "cost" (greedy-dual size-frequency, spike_serve.h)."""

    def __init__(self, budget_bytes, streams=4, max_batch_rhs=64, p=0, nrhs_hint=0, K=0.0, dryrun=False,
                 dryrun_factor_us=0, dryrun_solve_us=0, batch_systems=0, evict="lru", graphs=False, tuned=False,
                 fp64_residual=False):
        self._keep = {}
        cfg = ServerConfig(budget_bytes=int(budget_bytes), streams=streams, max_batch_rhs=max_batch_rhs, p=p,
                           nrhs_hint=nrhs_hint, K=K,
                           flags=(DRYRUN if dryrun else 0) | (GRAPHS if graphs else 0) | (TUNED if tuned else 0) |
                                 (FP64_RESIDUAL if fp64_residual else 0),
                           dryrun_factor_us=dryrun_factor_us, dryrun_solve_us=dryrun_solve_us,
                           batch_systems=batch_systems, evict_policy={"lru": EVICT_LRU, "cost": EVICT_COST}[evict])
        h = ctypes.c_void_p()
        rc = _lib().spike_server_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc != 0:
            raise spike.SpikeError(rc, "spike_server_create")
        self._h = h
        self._n = {}

    def add_matrix(self, mid, band, kl, ku, pivot=0):
        n, ldab = band.shape
        rc = _lib().spike_server_add_matrix(self._h, mid, spike._ptr(band), ldab, n, kl, ku, pivot)
        if rc != 0:
            raise spike.SpikeError(rc, "spike_server_add_matrix")
        self._keep[("band", mid)] = band
        self._n[mid] = n

    def submit(self, mid, F, X=None, trans="N", mixed=False):
        """Queue op(A_mid) X = F; returns (request id, X).  X defaults to a new array like F."""
        if X is None:
            X = np.empty_like(F) if isinstance(F, np.ndarray) else F.clone()
        nrhs = spike._check_rhs(F, self._n[mid])
        if tuple(X.shape) != tuple(F.shape):
            raise ValueError("X has shape %s, F has %s" % (tuple(X.shape), tuple(F.shape)))
        rid = _lib().spike_server_submit(self._h, mid, spike._ptr(F), spike._ptr(X), nrhs, trans.encode(),
                                         1 if mixed else 0)
        if rid < 0:
            raise spike.SpikeError(int(rid), "spike_server_submit")
        self._keep[rid] = (F, X)
        return rid, X

    def wait(self, rid):
        """Block until request rid is done; returns its latency in ms (raises on failure)."""
        lat = ctypes.c_double(0.0)
        rc = _lib().spike_server_wait(self._h, rid, ctypes.byref(lat))
        self._keep.pop(rid, None)
        if rc != 0:
            raise spike.SpikeError(rc, "request %d (%s)" % (rid, _lib().spike_server_last_error(self._h).decode()))
        return lat.value

    def latency(self, rid):
        """Latency (ms) of request rid if it has completed, else None (does not block)."""
        lat = ctypes.c_double(0.0)
        rc = _lib().spike_server_request_latency(self._h, rid, ctypes.byref(lat))
        if rc < 0:
            raise spike.SpikeError(rc, "spike_server_request_latency")
        if rc == 0:
            self._keep.pop(rid, None)  # done: the engine no longer touches its buffers
            return lat.value
        return None

    def drain(self):
        submitted = [key for key in list(self._keep) if not isinstance(key, tuple)]
        rc = _lib().spike_server_drain(self._h)
        if rc != 0:
            raise spike.SpikeError(rc, "spike_server_drain")
        # the requests submitted before the drain have finished: release their F and X references
        for key in submitted:
            self._keep.pop(key, None)

    def stats(self):
        out = ServerStats()
        rc = _lib().spike_server_stats_get(self._h, ctypes.byref(out))
        if rc != 0:
            raise spike.SpikeError(rc, "spike_server_stats_get")
        return out.as_dict()

    def latencies(self):
        cnt = ctypes.c_int64(0)
        _lib().spike_server_latencies(self._h, None, 0, ctypes.byref(cnt))
        out = np.zeros(cnt.value)
        _lib().spike_server_latencies(self._h, out.ctypes.data_as(ctypes.c_void_p), cnt.value, ctypes.byref(cnt))
        return out

    def close(self):
        if self._h:
            _lib().spike_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
