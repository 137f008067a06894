"""Partition-range sharding of one banded system over several ranks, one GPU each.

ctypes binding of the spike_shard_* entry points of libspike.so (include/spike.h) and the
exchange loop that drives them.  Rank g owns a contiguous power-of-two range of the
partitions (Sec. 3); the merge levels of the recursive reduced system (Sec. 2.2) inside
that range run on its GPU, and each level above it is one exchange: every rank exports a
fixed-size buffer of boundary tips (or, in the transposed solve, a partial product), the
buffers are all-gathered, and every rank imports the gathered buffers.  The collective is
the caller's: `TorchCollective` uses torch.distributed (NCCL for CUDA tensors), and
`run_local` runs the ranks of one process in lock step (an all-gather by concatenation).

Marshalling only: every step of the factorization and the solves runs in the library's
kernels.
"""
import ctypes

import numpy as np

from . import spike


def _lib():
    L = spike.lib()
    if not getattr(L, "_shard_types", False):
        i64, i32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        L.spike_shard_plan.argtypes = [i64, i32, i32, i32, i32, ctypes.POINTER(spike.SpikeOptions), vp, vp,
                                       ctypes.POINTER(ctypes.c_int32)]
        L.spike_shard_factor.argtypes = [vp, i64, i64, i64, i32, i32, i32, i32, i32, ctypes.POINTER(spike.SpikeOptions),
                                         ctypes.POINTER(vp)]
        L.spike_shard_solve.argtypes = [vp, vp, i64, i32, ctypes.c_char]
        L.spike_shard_pending.argtypes = [vp, ctypes.POINTER(i64)]
        L.spike_shard_export.argtypes = [vp, vp]
        L.spike_shard_import.argtypes = [vp, vp]
        for nm in ("spike_shard_plan", "spike_shard_factor", "spike_shard_solve", "spike_shard_pending",
                   "spike_shard_export", "spike_shard_import"):
            getattr(L, nm).restype = ctypes.c_int
        L._shard_types = True
    return L


def plan(n, kl, ku, p, nranks, nrhs_hint=0, stage_balance=False):
    """(row_first, leaf_first, local_levels) of the ranks, without a GPU (spike_shard_plan)."""
    opt = spike.SpikeOptions(nrhs_hint=nrhs_hint, flags=spike.FLAG_STAGE_BALANCE if stage_balance else 0)
    rows = np.zeros(nranks + 1, dtype=np.int64)
    leaves = np.zeros(nranks + 1, dtype=np.int32)
    ll = ctypes.c_int32(0)
    rc = _lib().spike_shard_plan(n, kl, ku, p, nranks, ctypes.byref(opt), rows.ctypes.data_as(ctypes.c_void_p),
                                 leaves.ctypes.data_as(ctypes.c_void_p), ctypes.byref(ll))
    if rc != 0:
        raise spike.SpikeError(rc, "spike_shard_plan")
    return rows, leaves, ll.value


def band_columns(n, kl, ku, row_first, rank):
    """Global band columns [c0, c1) rank `rank` passes to spike_shard_factor: its rows and
    the k columns on each side that hold its couplings."""
    k = max(kl, ku, 1)
    return max(0, int(row_first[rank]) - k), min(n, int(row_first[rank + 1]) + k)


def exchange_loop(engine, all_gather):
    """Run the pending exchanges of one rank: while the engine has one, export its buffer,
    all-gather it over the ranks, import the result.  `engine` has pending() -> count,
    export(count) -> tensor and import_(recv); `all_gather(send)` returns the ranks'
    buffers concatenated in rank order.  Returns the number of exchanges."""
    rounds = 0
    while True:
        count = engine.pending()
        if count == 0:
            return rounds
        recv = all_gather(engine.export(count))
        engine.import_(recv)
        rounds += 1


class TorchCollective:
    """all_gather over torch.distributed (any backend; NCCL for CUDA tensors)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.size = dist.get_world_size(group)

    def __call__(self, send):
        import torch
        recv = torch.empty(self.size * send.numel(), dtype=send.dtype, device=send.device)
        self.dist.all_gather_into_tensor(recv, send.contiguous(), group=self.group)
        if send.is_cuda:
            torch.cuda.current_stream().synchronize()
        return recv


class ShardEngine:
    """One rank's handle (spike_shard_factor) with the engine interface of exchange_loop."""

    def __init__(self, band_cols, col0, n, kl, ku, p, rank, nranks, nrhs_hint=0, stage_balance=False):
        import torch
        self.torch = torch
        self.n, self.kl, self.ku, self.rank, self.nranks = n, kl, ku, rank, nranks
        self.device = band_cols.device
        s = ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        self._opt = spike.SpikeOptions(nrhs_hint=nrhs_hint, flags=spike.FLAG_STAGE_BALANCE if stage_balance else 0,
                                       stream=s)
        h = ctypes.c_void_p()
        rc = _lib().spike_shard_factor(spike._ptr(band_cols), band_cols.shape[1], col0, n, kl, ku, p, rank, nranks,
                                       ctypes.byref(self._opt), ctypes.byref(h))
        if rc < 0:
            raise spike.SpikeError(rc, "spike_shard_factor")
        self._h = h
        rows, _, _ = plan(n, kl, ku, p, nranks, nrhs_hint, stage_balance)
        self.row0, self.row1 = int(rows[rank]), int(rows[rank + 1])

    def pending(self):
        out = ctypes.c_int64(0)
        rc = _lib().spike_shard_pending(self._h, ctypes.byref(out))
        if rc != 0:
            raise spike.SpikeError(rc, "spike_shard_pending")
        return out.value

    def export(self, count):
        send = self.torch.empty(count, dtype=self.torch.float64, device=self.device)
        rc = _lib().spike_shard_export(self._h, ctypes.c_void_p(send.data_ptr()))
        if rc != 0:
            raise spike.SpikeError(rc, "spike_shard_export")
        return send

    def import_(self, recv):
        rc = _lib().spike_shard_import(self._h, ctypes.c_void_p(recv.data_ptr()))
        if rc != 0:
            raise spike.SpikeError(rc, "spike_shard_import")

    def start_solve(self, F, trans="N"):
        """Start a solve on this rank's rows F (CUDA tensor (nrhs, rows) or (rows,)); F holds
        X once the exchanges are done."""
        rows = self.row1 - self.row0
        nrhs = spike._check_rhs(F, rows)
        rc = _lib().spike_shard_solve(self._h, spike._ptr(F), rows, nrhs, trans.encode())
        if rc != 0:
            raise spike.SpikeError(rc, "spike_shard_solve")

    def info(self):
        out = spike.SpikeInfo()
        rc = spike.lib().spike_get_info(self._h, ctypes.byref(out))
        if rc != 0:
            raise spike.SpikeError(rc, "spike_get_info")
        return out.as_dict()

    def free(self):
        if self._h:
            spike.lib().spike_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def run_local(engines):
    """Run the pending exchanges of all ranks of one process in lock step: every round, each
    rank exports, the buffers are concatenated in rank order (the all-gather) and every rank
    imports them.  For ranks that share a GPU no kernel waits on another: each import only
    starts after every export has completed.  Returns the number of rounds."""
    import torch
    rounds = 0
    while True:
        counts = [e.pending() for e in engines]
        if len(set(counts)) != 1:
            raise RuntimeError("ranks disagree on the pending exchange: %s" % counts)
        if counts[0] == 0:
            return rounds
        recv = torch.cat([e.export(counts[0]) for e in engines])
        for e in engines:
            e.import_(recv)
        rounds += 1


class ShardedFactorization:
    """One rank of a sharded factorization: factor, then solve with the rank's rows, each
    followed by the exchanges over `all_gather` (e.g. TorchCollective())."""

    def __init__(self, band_cols, col0, n, kl, ku, p, rank, nranks, all_gather, **kw):
        self.engine = ShardEngine(band_cols, col0, n, kl, ku, p, rank, nranks, **kw)
        self.all_gather = all_gather
        self.factor_exchanges = exchange_loop(self.engine, all_gather)

    def solve(self, F, trans="N"):
        self.engine.start_solve(F, trans)
        exchange_loop(self.engine, self.all_gather)
        return F

    def free(self):
        self.engine.free()
