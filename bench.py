#!/usr/bin/env python3
"""Benchmark of the recursive SPIKE hot path on GB300.

One step = spike_factor + spike_solve('N') + spike_solve('T') + spike_free on the
workload n = 1,048,576, kl = ku = 128, p = 148 workers (128 partitions, 20 of
them run as SPIKE 2x2 pairs: 148 blocks), nrhs = 64, dominance factor 1.01,
synthetic inputs from paper_1811_03559_gb300.inputs (seed 1).

Printed JSON line (rank 0):
  value   whole-job GB/s of algorithmic bytes: 16n(2k+1) for the factorization
          (band in, factors out) + per solve 8n(2k+1) (factors read) + 16 n nrhs
          (F in, X out), with inputs resident in HBM, timed with CUDA events;
  e2e     the same metric through the C ABI with pinned HOST buffers (host<->device
          copies inside the timed calls);
  roofline  the dominant kernel (block LU + fused spike sweep): method FP64 flops
          per launch / its mean duration from events recorded on the library's
          stream, against the FP64 FMA peak;
  cpu_baseline  the CPU oracle (banded GEPP + N and T solves) on a bounded sample.
Multi-GPU: replicas only (each rank solves its own copy; the method has no
data-parallel exchange within one system on one GPU), value = sum over ranks.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "n=1M k=128 factor+solve GB/s & % roofline vs FP64; serving p50/p99, solves/s"
# FP64 FMA peak derived from unit counts and clock: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # FP32 FMA: 4 x 32 lanes per SM and clock
FP64_PEAK_NOTE = "derived: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz (the recipe's 1.25 TFLOP/s nominal); " \
                 "peak_measured is the library's DFMA probe (spike_measure_fp64_peak) run in this process"


def aggregate_over_ranks(ms_local, bytes_per_step_local, steps, dist=None, device=None):
    """Max of the timed region over ranks and the whole-job throughput (GB/s) of N replicas."""
    ms = float(ms_local)
    world = 1
    if dist is not None:
        import torch
        world = dist.get_world_size()
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        tb = torch.tensor([float(bytes_per_step_local)], dtype=torch.float64, device=device)
        dist.all_reduce(tb, op=dist.ReduceOp.SUM)
        total_bytes = float(tb.item())
    else:
        total_bytes = float(bytes_per_step_local)
    return ms, total_bytes * steps / (ms * 1e-3) / 1e9, world


def alg_bytes(n, k, m, nsolves=2):
    return 16.0 * n * (2 * k + 1) + nsolves * (8.0 * n * (2 * k + 1) + 16.0 * n * m)


def plan_groups(offs, flags):
    """Merge levels as lists of (a, b, c) leaf ranges (mirrors the planner, Sec. 2.2 / 3.1)."""
    nb = len(offs) - 1
    groups = [(i, i + 1) for i in range(nb)]
    levels = []
    if any(f & 2 for f in flags):
        lv, merged, i = [], [], 0
        while i < nb:
            if flags[i] & 2:
                lv.append((i, i + 1, i + 2))
                merged.append((i, i + 2))
                i += 2
            else:
                merged.append((i, i + 1))
                i += 1
        levels.append(lv)
        groups = merged
    while len(groups) > 1:
        lv, nxt = [], []
        for j in range(0, len(groups), 2):
            lv.append((groups[j][0], groups[j][1], groups[j + 1][1]))
            nxt.append((groups[j][0], groups[j + 1][1]))
        levels.append(lv)
        groups = nxt
    return levels


def pivot_block_flops(offs, k):
    """FP64 flops of the pivoting block stage (Sec. 5.1 with the sweeps of Sec. 2.3): per row the
    GEPP's k multipliers and k x 2k update (U filled to 2k); middle blocks add the full L sweep of
    the top spike (k columns) and the U sweep of both spikes (2k columns, 2k superdiagonals); each
    end block's truncated sweeps of its one spike (2k rows of L, k rows of U, k columns) add 8k^3."""
    sizes = np.diff(offs).astype(np.float64)
    nb, k = len(sizes), float(k)
    f = 0.0
    for i, nl in enumerate(sizes):
        f += nl * (4 * k * k + k)
        if 0 < i < nb - 1:
            f += nl * 2 * k * k + nl * 8 * k * k
        elif nb > 1:
            f += 8 * k ** 3
    return f


def method_flops(offs, flags, k, m):
    """FP64 flops the method performs (Sec. 2.3 sweep counts, Sec. 2.2 reduced system)."""
    nb = len(offs) - 1
    sizes = np.diff(offs).astype(np.float64)
    f = {"block_lu": 0.0, "factor_spikes": 0.0, "factor_reduced": 0.0, "solve_n": 0.0, "solve_t": 0.0}
    k = float(k)
    for i, nl in enumerate(sizes):
        mid = 0 < i < nb - 1
        lu = nl * (2 * k * k + k)                  # band LU: k multipliers + k x k update per column
        f["block_lu"] += lu + (2 * nl * k * k if mid else 0.0)   # + fused L-sweep of the top spike
        if nb > 1:  # the other spike sweeps run in the same launch as the block LU
            f["block_lu"] += (nl * (4 * k * k + 2 * k)) if mid else 2 * k ** 3  # U sweep of both spikes
            f["block_lu"] += k ** 3  # truncated L sweep of the bottom spike
        sweeps = 4 if mid else (2 if nb > 1 else 2)
        f["solve_n"] += sweeps * 2 * nl * k * m
        f["solve_t"] += sweeps * 2 * nl * k * m
        f["solve_n"] += (2 if mid else 1) * 2 * k * k * m * (nb > 1)
        f["solve_t"] += (2 if mid else 1) * 2 * k * k * m * (nb > 1)
    for lv in plan_groups(offs, flags):
        for (a, b, c) in lv:
            nL, nR = b - a, c - b
            hasV, hasW = c != nb, a != 0
            fr = 2 * k ** 3 + 2 * k ** 3 / 3            # S = I - W V, LU(S)
            fr += (2 * k ** 3 + 2 * k ** 3) * hasV + (4 * k ** 3 + 2 * k ** 3) * hasW
            fr += (2 * k ** 3) * (2 * nL + 2 * nR - 1) * (hasV + hasW)
            f["factor_reduced"] += fr
            f["solve_n"] += 2 * k * k * m * (3 + (2 * nL - 1) + (2 * nR - 1))
            f["solve_t"] += 2 * k * k * m * (2 * nL + 2 * nR + 3 + 2)
    f["factor"] = f["block_lu"] + f["factor_spikes"] + f["factor_reduced"]
    f["step"] = f["factor"] + f["solve_n"] + f["solve_t"]
    return f


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(r[0] for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": rows[0][1], "samples": len(rows),
                "power_w_max": max(r[2] for r in rows), "reasons": reasons}


def cpu_oracle_sample(k, m, dd, n_sample, seed):
    """Time the CPU oracle (banded GEPP + N and T solves) on the first rows of the workload's generator."""
    import oracle
    from paper_1811_03559_gb300 import inputs
    pr = inputs.make_problem(n_sample, k, k, m, seed=seed, dd=dd)
    oracle.build_oracle()
    t0 = time.perf_counter()
    lu = oracle.BandLU(pr["band"], k, k)
    lu.solve(pr["F"], "N")
    lu.solve(pr["F"], "T")
    dt = time.perf_counter() - t0
    return {"value": alg_bytes(n_sample, k, m) / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "n=%d kl=ku=%d nrhs=%d DD=%g: banded GEPP factor + N solve + T solve, single thread, "
                      "%.2f s" % (n_sample, k, m, dd, dt), "seconds": dt}


def source_hash():
    h = hashlib.sha256()
    for f in ("leaf.cu", "internal.h"):
        h.update(open(os.path.join(ROOT, "paper_1811_03559_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def load_traffic():
    path = os.path.join(ROOT, "profiles", "block_lu_k128_traffic.json")
    if not os.path.exists(path):
        return None, None
    d = json.load(open(path))
    if d.get("source_hash") != source_hash():
        return None, d
    return d.get("dram_bytes_per_launch_full"), d


def graphs_leg(dev, solves=200):
    """Repeated solves of small systems, direct launches against CUDA-graph replay
    (SPIKE_FLAG_GRAPHS): wall microseconds per solve on a side stream (F re-copied into X each
    time, in both variants)."""
    import torch
    from paper_1811_03559_gb300 import inputs, spike
    s = torch.cuda.Stream()
    out = {}
    for n, k, p, m in [(20_000, 16, 16, 4), (200_000, 64, 64, 16)]:
        band = inputs.make_band_torch(n, k, k, seed=9, dd=1.1, device=dev)
        res = {}
        with torch.cuda.stream(s):
            for graphs in (False, True):
                fac = spike.Factorization(band, k, k, p, graphs=graphs)
                F = torch.rand((m, n), dtype=torch.float64, device=dev)
                X = F.clone()
                for _ in range(3):  # direct, captured, replayed
                    X.copy_(F)
                    fac.solve(X, "N")
                s.synchronize()
                t0 = time.perf_counter()
                for _ in range(solves):
                    X.copy_(F)
                    fac.solve(X, "N")
                s.synchronize()
                res["graphs_us" if graphs else "direct_us"] = 1e6 * (time.perf_counter() - t0) / solves
                if graphs:
                    res["graph_replays"] = fac.info()["graph_replays"]
                fac.free()
        res["speedup"] = res["direct_us"] / res["graphs_us"]
        out["n=%d k=%d p=%d nrhs=%d" % (n, k, p, m)] = res
    return out


def mixed_workload_leg(dev, reps=2):
    """The mixed-precision workload (n = 2^20, DD 1.05, k in {64, 256}, nrhs in {1, 32, 256}):
    factor + one N solve, FP64 against SPIKE_FLAG_MIXED (FP32 blocks + FP64 refinement), with the
    backward error of each.  Inputs are drawn on the device (inputs.make_band_torch)."""
    import torch
    from paper_1811_03559_gb300 import inputs, spike
    n, dd, p = 1 << 20, 1.05, 148
    out = {"workload": "n=%d DD=%g p=%d: spike_factor + spike_solve N, FP64 vs mixed" % (n, dd, p), "cases": []}
    for k in (64, 256):
        band = inputs.make_band_torch(n, k, k, seed=3, dd=dd, device=dev)
        for m in (1, 32, 256):
            g = torch.Generator(device=dev)
            g.manual_seed(7 + m)
            xs = torch.rand((m, n), generator=g, dtype=torch.float64, device=dev) * 2.0 - 1.0
            F = inputs.band_matvec_torch(band, k, k, xs, "N")
            row = {"k": k, "nrhs": m}
            for mixed in (False, True):
                times = []
                X = None
                for _ in range(reps + 1):
                    X = F.clone()
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    fac = spike.Factorization(band, k, k, p, nrhs_hint=m, stage_balance=True, mixed=mixed)
                    fac.solve(X, "N")
                    torch.cuda.synchronize()
                    times.append(time.perf_counter() - t0)
                    steps = fac.info()["refine_steps"]
                    fac.free()
                key = "mixed" if mixed else "fp64"
                row[key + "_ms"] = 1e3 * float(np.median(times[1:]))
                row[key + "_backward_error"] = float(spike.backward_error(band, k, k, X, F, "N").max())
                if mixed:
                    row["refine_steps"] = steps
            row["speedup"] = row["fp64_ms"] / row["mixed_ms"]
            out["cases"].append(row)
            del xs, F
        del band
    return out


def tensor_residual_leg(band, k, X, FN, FT, p, reps=5):
    """The mixed-precision refinement residual on the tensor cores (spike_residual: int8 digit
    slices, bf16 products with exact FP32 accumulation) against the FP64 kernel
    (spike_backward_error) on the step's matrix and right-hand sides; tensor flops = 43 digit
    products x 2 x (rows x K x columns) with K = 32 ceil((19 + kl + ku) / 32) columns per
    16-row block."""
    import torch
    from paper_1811_03559_gb300 import spike
    n, m = band.shape[0], X.shape[0]
    fac = spike.Factorization(band, k, k, p, nrhs_hint=m, stage_balance=True, mixed=True)
    R = torch.empty_like(FN)

    def t(fn):
        ts = []
        for _ in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts[1:]))

    out = {}
    KP = 32 * ((19 + 2 * k + 31) // 32)
    flops = 43 * 2.0 * n * KP * m
    for tr, F in (("N", FN), ("T", FT)):
        ms = t(lambda: fac.residual(X, F, R, tr))
        out[tr] = {"tensor_ms": ms, "fp64_ms": t(lambda: spike.backward_error(band, k, k, X, F, tr)),
                   "tensor_tflops": flops / (ms * 1e-3) / 1e12}
    fac.free()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    bf16 = peaks.get("bf16_tflops")
    out["flops_per_call"] = flops
    out["peak_bf16_tflops_measured"] = bf16
    out["frac_of_measured_bf16"] = out["N"]["tensor_tflops"] / bf16 if bf16 else None
    out["note"] = ("legacy mma.sync bf16 path; an in-process probe of mma.sync m16n8k16 measured about 600 TFLOP/s "
                   "on this part, the measured peak is cuBLAS (tcgen05)")
    return out


def config_grid_leg(dev, reps=2):
    """Every point of the large dominant workload: n = 2^20, k in {32, 128, 320}, p in {64, 148,
    192}, nrhs in {1, 64} (DD 1.01; the times do not depend on the values): factor + N solve +
    T solve per point, with algorithmic GB/s, method TFLOP/s against the FP64 peak and the
    backward error.  Bands are drawn on the device (inputs.make_band_torch)."""
    import torch
    from paper_1811_03559_gb300 import inputs, spike
    n, dd = 1 << 20, 1.01
    rows = []
    for k in (32, 128, 320):
        band = inputs.make_band_torch(n, k, k, seed=1, dd=dd, device=dev)
        for m in (1, 64):
            g = torch.Generator(device=dev)
            g.manual_seed(11 + m)
            xs = torch.rand((m, n), generator=g, dtype=torch.float64, device=dev) * 2.0 - 1.0
            FN = inputs.band_matvec_torch(band, k, k, xs, "N")
            FT = inputs.band_matvec_torch(band, k, k, xs, "T")
            for p in (64, 148, 192):
                _, offs, flags = spike.plan(n, k, k, p, nrhs_hint=m, stage_balance=True)
                fl = method_flops(offs, flags, k, m)
                times, st = [], {}
                for rep in range(reps + 1):
                    X1, X2 = FN.clone(), FT.clone()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record()
                    fac = spike.Factorization(band, k, k, p, nrhs_hint=m, stage_balance=True, timing=rep == reps)
                    fac.solve(X1, "N")
                    fac.solve(X2, "T")
                    e1.record()
                    torch.cuda.synchronize()
                    if rep:
                        times.append(e0.elapsed_time(e1))
                    if rep == reps:
                        st = fac.timings()
                    fac.free()
                ms = float(np.median(times))
                rows.append({"k": k, "nrhs": m, "p": p, "ms_per_step": ms, "GB_s": alg_bytes(n, k, m) / (ms * 1e-3) / 1e9,
                             "method_tflops": fl["step"] / (ms * 1e-3) / 1e12,
                             "frac_fp64": fl["step"] / (ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                             "block_lu_frac_fp64": fl["block_lu"] / (st["block_lu"] * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                             "factor_ms": st["factor"], "solve_n_ms": st["solve_n"], "solve_t_ms": st["solve_t"],
                             "backward_error": max(float(spike.backward_error(band, k, k, X1, FN, "N").max()),
                                                   float(spike.backward_error(band, k, k, X2, FT, "T").max()))})
            del FN, FT, xs
        del band
        torch.cuda.empty_cache()
    return {"workload": "n=%d, DD %g, k in {32,128,320}, p in {64,148,192}, nrhs in {1,64}: spike_factor + "
                        "spike_solve N + spike_solve T (stage-balanced sizing), median of %d" % (n, dd, reps),
            "unit": "GB/s", "points": rows}


def pivoting_leg(dev, reps=3):
    """The pivoting workload (Sec. 5): n = 262,144, k in {16, 64}, nrhs = 8, p = 148, N(0,1) entries
    with the diagonal at 0.3 x the row's off-diagonal absolute sum (sign kept), factor + N + T.
    The block GEPP's method flops (k multipliers and a k x 2k update per column, U filled to
    2k) against the FP64 peak, beside the non-pivoting block LU's rate on the same matrix."""
    import torch
    from paper_1811_03559_gb300 import inputs, spike
    n, p, m = 262_144, 148, 8
    out = {"workload": "n=%d p=%d nrhs=%d, N(0,1) entries, diagonal 0.3 x row off-diagonal |.| sum (seed 2)"
                       % (n, p, m), "cases": []}
    for k in (16, 64):
        seed = 2
        while True:
            pr = inputs.make_problem(n, k, k, m, seed=seed, dist="normal", dd=0.3, keep_sign=True)
            band = torch.from_numpy(pr["band"]).to(dev)
            fac = spike.Factorization(band, k, k, p, pivot=1, nrhs_hint=m)
            ok = fac.status == 0
            fac.free()
            if ok:
                break
            seed += 1
        FN = torch.from_numpy(pr["F"]).to(dev)
        FT = torch.from_numpy(inputs.band_matvec(pr["band"], k, k, pr["xstar"], "T")).to(dev)
        # method flops of the block stage (one launch: block factorizations + spike sweeps), from
        # each factorization's own plan (pivoting: default ratio R13 = spike.PIVOT_R13)
        _, offs, _ = spike.plan(n, k, k, p, nrhs_hint=m, R13=spike.PIVOT_R13)
        _, offs0, flags0 = spike.plan(n, k, k, p, nrhs_hint=m)
        stage_flops = {1: pivot_block_flops(offs, k), 0: method_flops(offs0, flags0, k, m)["block_lu"]}
        row = {"k": k, "seed": seed}
        for piv in (1, 0):
            times, st = [], {}
            for rep in range(reps + 1):
                X1, X2 = FN.clone(), FT.clone()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                fac = spike.Factorization(band, k, k, p, pivot=piv, nrhs_hint=m, timing=True)
                fac.solve(X1, "N")
                fac.solve(X2, "T")
                e1.record()
                torch.cuda.synchronize()
                if rep:
                    times.append(e0.elapsed_time(e1))
                st = fac.timings()
                fac.free()
            ms = float(np.median(times))
            key = "pivoting" if piv else "non_pivoting"
            flops = stage_flops[piv]
            row[key] = {"ms_per_step": ms, "GB_s": alg_bytes(n, k, m) / (ms * 1e-3) / 1e9,
                        "factor_ms": st["factor"], "block_stage_ms": st["block_lu"], "spikes_ms": st["spikes"],
                        "solve_n_ms": st["solve_n"], "solve_t_ms": st["solve_t"],
                        "block_stage_gflops": flops / (st["block_lu"] * 1e-3) / 1e9,
                        "block_stage_frac_fp64": flops / (st["block_lu"] * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                        "backward_error": max(float(spike.backward_error(band, k, k, X1, FN, "N").max()),
                                              float(spike.backward_error(band, k, k, X2, FT, "T").max()))}
        out["cases"].append(row)
        del band, FN, FT
    return out


def _cpu_serve_one(args):
    """One request of the serving workload on the CPU oracle: banded GEPP + solve (one core)."""
    import oracle
    from paper_1811_03559_gb300 import inputs
    n, k, m, trans, seed = args
    band, rng = inputs.make_band(n, k, k, seed=seed, dd=1.1)
    F = rng.uniform(-1.0, 1.0, size=(m, n))
    t0 = time.perf_counter()
    oracle.gbsv(band, k, k, F, trans)
    return time.perf_counter() - t0


def cpu_serving_baseline(nreq=160, seed=None):
    """Requests of the serving workload solved by the CPU oracle, one per host core in
    parallel (spawned processes): CPU solves/s.  Each request factors its matrix (the oracle
    keeps no factorization) and solves its right-hand sides; the matrix generation is not
    timed."""
    import multiprocessing as mp
    from paper_1811_03559_gb300 import inputs
    cfg = dict(inputs.SERVING)
    if seed is not None:
        cfg["seed"] = seed
    ns, ks, _ = inputs.serving_catalogue(cfg)
    arrivals, mids, nrhs, trans, mixed = inputs.serving_trace(cfg)
    jobs = [(int(ns[mids[i]]), int(ks[mids[i]]), int(nrhs[i]), str(trans[i]), 1000 + int(mids[i]))
            for i in range(nreq)]
    cores = os.cpu_count() or 1
    import oracle
    oracle.build_oracle()
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        t0 = time.perf_counter()
        times = pool.map(_cpu_serve_one, jobs, chunksize=1)
        wall = time.perf_counter() - t0
    busy = float(sum(times))
    return {"solves_per_s": nreq * cores / busy, "cores": cores, "kind": "oracle", "requests": nreq,
            "sample": "first %d requests of the serving trace, banded GEPP factor + solve per request, one request "
                      "per core (%d spawned processes); rate = requests / (summed solve seconds / cores), "
                      "wall %.1f s" % (nreq, cores, wall)}


def tuning_leg(band, k, nrhs):
    """The load-balancing constant K measured on one block (Sec. 3.3), a partition-ratio sweep
    at p = 148 (the paper's ratio experiment), and the fastest worker count (spike_tune)."""
    from paper_1811_03559_gb300 import spike
    ps = [128, 148, 152, 192]
    rs = [1.0, 1.5, 2.0, 2.5, 3.0, 4.0]
    t0 = time.perf_counter()
    res, table = spike.tune(band, k, k, nrhs, ps, r13_candidates=rs, nsolves=2)
    cols = ["paper_ratio_measured_K", "stage_balance"] + ["R13=%g" % r for r in rs]
    info_formula, _, _ = spike.plan(band.shape[0], k, k, 148, K=res["K_measured"], nrhs_hint=nrhs)
    return {"K_measured": res["K_measured"],
            "formula_R13_at_measured_K": info_formula["R13"],
            "best": {"p": res["best_p"], "mode": ["paper_ratio", "stage_balance", "explicit_R13"][res["best_mode"]],
                     "R13": res["best_R13"], "ms": res["best_ms"]},
            "default_ms": res["default_ms"], "columns": cols,
            "table_ms": {str(p): [round(float(x), 2) for x in row] for p, row in zip(ps, table)},
            "step": "factor + 2 N solves, nrhs = %d (zero right-hand sides; times do not depend on values)" % nrhs,
            "seconds": time.perf_counter() - t0}


def serving_leg(dev, requests, streams, max_batch, passes=2, seed=None, batch_systems=1, evict="lru",
                fp64_residual=False):
    """Many-matrix serving workload (inputs.SERVING) through the native serving engine.

    The catalogue bands live in device memory (the caller's; the budget covers the
    factorizations, their scratch and the workspaces).  Right-hand sides come from
    pinned host memory and results go back to pinned host memory: every request's
    latency is submit -> X in host memory.  Arrivals are open-loop (Poisson, replayed
    on the host clock) and every latency counts from the request's intended arrival, so
    time a request spent waiting to be submitted (result buffers full) is included.  The
    trace runs `passes` times at its own rate on the same server (the first pass starts
    with nothing factored), then once more slowed to 60 % of the measured capacity.
    """
    import collections
    import torch
    from paper_1811_03559_gb300 import inputs, serve, spike
    cfg = dict(inputs.SERVING)
    cfg["requests"] = requests
    if seed is not None:
        cfg["seed"] = seed
    ns, ks, _ = inputs.serving_catalogue(cfg)
    arrivals, mids, nrhs, trans, mixed = inputs.serving_trace(cfg)
    used = sorted(set(int(x) for x in mids))
    t_gen = time.perf_counter()
    bands = {i: inputs.make_band_torch(int(ns[i]), int(ks[i]), int(ks[i]), 7919 * cfg["seed"] + i, cfg["dd"], dev)
             for i in used}
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    nmax = int(ns.max())
    fbuf = torch.empty(cfg["nrhs_max"] * nmax, dtype=torch.float64).uniform_(-1.0, 1.0).pin_memory().numpy()
    cap = 1 << 29  # 4 GB of pinned result space, reused as a ring
    arena = torch.empty(cap, dtype=torch.float64).pin_memory().numpy()
    budget = int(cfg["budget_gb"] * 1e9)
    S = serve.Server(budget, streams=streams, max_batch_rhs=max_batch, nrhs_hint=16, batch_systems=batch_systems,
                     evict=evict, fp64_residual=fp64_residual)
    for i in used:
        S.add_matrix(i, bands[i], int(ks[i]), int(ks[i]))
    out = {"workload": "%d requests, Poisson %g/s, %d matrices (n log-uniform [%d, %d], k uniform {4..128 step 4}, "
                       "DD %g), Zipf(%g) popularity, nrhs U[1,%d], %d%% T, %d%% mixed, %g GB budget"
                       % (requests, cfg["rate"], cfg["matrices"], cfg["n_lo"], cfg["n_hi"], cfg["dd"], cfg["zipf"],
                          cfg["nrhs_max"], round(100 * cfg["trans_t"]), round(100 * cfg["mixed"]), cfg["budget_gb"]),
           "matrices_used": len(used), "catalogue_gb": sum(8.0 * ns[i] * (2 * ks[i] + 1) for i in used) / 1e9,
           "streams": streams, "max_batch_rhs": max_batch, "batch_systems": batch_systems, "evict": evict,
           "mixed_residual": "FP64 FMAs" if fp64_residual else "tensor cores (digit planes of op(A) kept per handle)",
           "catalogue_gen_s": t_gen,
           "data": "synthetic (torch generator on the device for the bands, seeded per matrix)", "passes": []}
    launches0 = spike.kernel_launches()

    def replay(scale):
        """Replay the trace with arrival times x scale; latency counts from the intended arrival."""
        prev = S.stats()
        outstanding = collections.deque()
        head, lag, rids = 0, np.zeros(requests), np.zeros(requests, dtype=np.int64)
        t0 = time.perf_counter()
        for i in range(requests):
            target = t0 + arrivals[i] * scale
            now = time.perf_counter()
            while now < target:
                if target - now > 5e-4:
                    time.sleep(target - now - 3e-4)
                now = time.perf_counter()
            n, m = int(ns[mids[i]]), int(nrhs[i])
            sz = n * m
            if head + sz > cap:
                head = 0
            lo, hi = head, head + sz
            # regions are handed out in ring order, so the oldest outstanding ones are the
            # first that the new region can overlap
            while outstanding and not (outstanding[0][2] <= lo or outstanding[0][1] >= hi):
                S.wait(outstanding.popleft()[0])
            lag[i] = time.perf_counter() - target
            X = arena[lo:hi].reshape(m, n)
            rid, _ = S.submit(int(mids[i]), fbuf[:sz].reshape(m, n), X, trans=str(trans[i]), mixed=bool(mixed[i]))
            rids[i] = rid
            outstanding.append((rid, lo, hi))
            head = hi
        S.drain()
        wall = time.perf_counter() - t0
        st = S.stats()
        lat = np.sort(np.array([S.latency(int(r)) for r in rids]) + 1e3 * lag)
        rank = lambda q: float(lat[max(1, int(np.ceil(q * len(lat)))) - 1])
        done = st["completed"] - prev["completed"]
        nb = st["batches"] - prev["batches"]
        return {"rate_per_s": requests / (arrivals[-1] * scale), "p50_ms": rank(0.5), "p99_ms": rank(0.99),
                "max_ms": float(lat[-1]), "mean_ms": float(lat.mean()), "solves_per_s": done / wall,
                "rhs_per_s": (st["rhs"] - prev["rhs"]) / wall, "wall_s": wall,
                "failed": st["failed"] - prev["failed"], "batches": nb, "mean_requests_per_batch": done / max(1, nb),
                "factorizations": st["factorizations"] - prev["factorizations"],
                "evictions": st["evictions"] - prev["evictions"], "peak_gb": st["peak_bytes"] / 1e9,
                "solves_over_several_matrices": st["multi_solves"] - prev["multi_solves"],
                "max_matrices_per_solve": st["max_systems"], "max_submit_lag_ms": 1e3 * float(lag.max())}

    # the workload's own rate (cold, then warm), then the same trace slowed to 60 % of the
    # measured capacity, where the queue stays bounded
    for ps in range(passes):
        out["passes"].append(dict(replay(1.0), phase="offered rate, pass %d" % ps))
    cap_rate = out["passes"][-1]["solves_per_s"]
    scale = max(1.0, (requests / arrivals[-1]) / (0.6 * cap_rate))
    out["sustainable"] = dict(replay(scale), phase="60 % of measured capacity")
    out["gpu_launches"] = int(spike.kernel_launches() - launches0)
    # baseline: the same requests one at a time with no resident factorizations and no
    # merging (FP64 factor + solve + free per request, whole GPU per request), on a sample
    nb = min(300, requests)
    t0 = time.perf_counter()
    for i in range(nb):
        n, kk, m = int(ns[mids[i]]), int(ks[mids[i]]), int(nrhs[i])
        fac = spike.Factorization(bands[int(mids[i])], kk, kk, min(148, max(1, n // (8 * kk))), nrhs_hint=m,
                                  stage_balance=True, stream=0)
        X = np.array(fbuf[: n * m].reshape(m, n))
        fac.solve(X, str(trans[i]))
        fac.free()
    naive = nb / (time.perf_counter() - t0)
    out["unbatched_fp64_baseline"] = {"solves_per_s": naive, "sample_requests": nb,
                                      "method": "per request: FP64 spike_factor + spike_solve (host F/X) + spike_free, "
                                                "one stream, t = min(148, n/(8k)), first %d requests of the trace" % nb}
    # accuracy of served results: one request per (trans, precision) on the largest used matrix
    big = max(used, key=lambda i: ns[i] * ks[i])
    n, k = int(ns[big]), int(ks[big])
    berr = {}
    for tr in "NT":
        for mx in (False, True):
            F = np.ascontiguousarray(fbuf[: 4 * n].reshape(4, n))
            rid, X = S.submit(big, F, trans=tr, mixed=mx)
            S.wait(rid)
            be = spike.backward_error(bands[big], k, k, torch.from_numpy(X).to(dev), torch.from_numpy(F).to(dev), tr)
            berr["%s_%s" % (tr, "mixed" if mx else "fp64")] = float(be.max())
    out["backward_error_max"] = max(berr.values())
    out["backward_error"] = berr
    out["check_matrix"] = {"n": n, "k": k}
    S.close()
    w = out["passes"][-1]
    out.update({"p50_ms": w["p50_ms"], "p99_ms": w["p99_ms"], "solves_per_s": w["solves_per_s"],
                "rhs_per_s": w["rhs_per_s"], "capacity_solves_per_s": cap_rate,
                "capacity_vs_unbatched_fp64": cap_rate / naive,
                "p50_ms_at_60pct_capacity": out["sustainable"]["p50_ms"],
                "p99_ms_at_60pct_capacity": out["sustainable"]["p99_ms"]})
    return out


def profile_case(case):
    """One small factor + N + T solve for a profiler capture (inputs > L2, a few GB at most)."""
    import torch
    from paper_1811_03559_gb300 import inputs, spike
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n, p = 262_144, 148
    if case == "pivot":
        k, m = 64, 8
        pr = inputs.make_problem(n, k, k, m, seed=2, dist="normal", dd=0.3, keep_sign=True)
        kw = {"pivot": 1}
    else:
        k, m = 128, 64
        pr = inputs.make_problem(n, k, k, m, seed=1, dd=1.01)
        kw = {"mixed": True, "stage_balance": True}
    band = torch.from_numpy(pr["band"]).to(dev)
    FN = torch.from_numpy(pr["F"]).to(dev)
    FT = torch.from_numpy(inputs.band_matvec(pr["band"], k, k, pr["xstar"], "T")).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fac = spike.Factorization(band, k, k, p, nrhs_hint=m, **kw)
    X1, X2 = FN.clone(), FT.clone()
    fac.solve(X1, "N")
    fac.solve(X2, "T")
    torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t0)
    be = max(float(spike.backward_error(band, k, k, X1, FN, "N").max()),
             float(spike.backward_error(band, k, k, X2, FT, "T").max()))
    fac.free()
    print(json.dumps({"profile_case": case, "n": n, "k": k, "nrhs": m, "p": p, "wall_ms": ms, "backward_error": be}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="spike", choices=["spike", "reference"])
    ap.add_argument("--n", type=int, default=1_048_576)
    ap.add_argument("--k", type=int, default=128)
    ap.add_argument("--p", type=int, default=148)
    ap.add_argument("--nrhs", type=int, default=64)
    ap.add_argument("--dd", type=float, default=1.01)
    ap.add_argument("--e2e-steps", type=int, default=None, help="host-buffer steps (default: --steps)")
    ap.add_argument("--no-grid", action="store_true", help="skip the timed grid of the large dominant workload")
    ap.add_argument("--no-pivot", action="store_true", help="skip the pivoting workload leg")
    ap.add_argument("--cpu-sample", type=int, default=262144,
                    help="rows of the workload the CPU oracle baseline solves (about 10 s on one Arm core)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer (e2e) leg, e.g. under a profiler")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision variant")
    ap.add_argument("--no-serve", action="store_true", help="skip the many-matrix serving leg")
    ap.add_argument("--no-tune", action="store_true", help="skip the partition tuning leg")
    ap.add_argument("--serve-requests", type=int, default=10_000)
    ap.add_argument("--serve-streams", type=int, default=8)
    ap.add_argument("--serve-batch", type=int, default=64)
    ap.add_argument("--serve-passes", type=int, default=2)
    ap.add_argument("--serve-tensor-residual", action="store_true",
                    help="mixed-precision serving handles keep op(A)'s digit planes and form their residuals on "
                         "the tensor cores (default: FP64 FMAs, smaller handles)")
    ap.add_argument("--serve-evict", choices=("lru", "cost"), default="lru",
                    help="eviction policy of the serving engine (SPIKE_SERVE_EVICT_LRU / _COST)")
    ap.add_argument("--serve-batch-systems", type=int, default=1,
                    help="matrices whose FP64 requests may share one solve (spike_solve_batch)")
    ap.add_argument("--profile-case", choices=["pivot", "mixed"], default=None,
                    help="run one small case for a profiler capture (n = 262,144; pivot: k = 64, nrhs = 8, "
                         "factor + N + T; mixed: k = 128, nrhs = 64, FP32 factor + refined N + T) and exit")
    args = ap.parse_args()
    if args.profile_case:
        profile_case(args.profile_case)
        return
    if args.e2e_steps is None:
        args.e2e_steps = args.steps
    n, k, p, m, dd, seed = args.n, args.k, args.p, args.nrhs, args.dd, 1
    workload = "n=%d kl=ku=%d p=%d nrhs=%d DD=%g: spike_factor + spike_solve N + spike_solve T" % (n, k, p, m, dd)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        # The reference arm is the CPU oracle, timed on this host; only rank 0 runs it.
        if rank != 0:
            return
        ref_rows = max(4096, args.cpu_sample // 16)  # a short sample per step
        steps = []
        for _ in range(max(args.warmup, 0)):
            cpu_oracle_sample(k, m, dd, ref_rows, seed)
        for _ in range(args.steps):
            steps.append(cpu_oracle_sample(k, m, dd, ref_rows, seed))
        v = float(np.mean([s["value"] for s in steps]))
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": 0,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean([s["seconds"] for s in steps])),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload, "sample_rows": ref_rows},
                "cpu_baseline": {"value": v, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": steps[0]["sample"]},
                "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_1811_03559_gb300 import inputs, spike
    spike.lib()
    pr = inputs.make_problem(n, k, k, m, seed=seed, dd=dd)
    F2h = inputs.band_matvec(pr["band"], k, k, pr["xstar"], "T")
    band = torch.from_numpy(pr["band"]).to(dev)
    F1src = torch.from_numpy(pr["F"]).to(dev)
    F2src = torch.from_numpy(F2h).to(dev)
    F1, F2 = torch.empty_like(F1src), torch.empty_like(F2src)
    info, offs, flags = spike.plan(n, k, k, p, nrhs_hint=m, stage_balance=True)
    fl = method_flops(offs, flags, k, m)

    stage_acc = {}

    def step(record):
        F1.copy_(F1src)
        F2.copy_(F2src)
        fac = spike.Factorization(band, k, k, p, nrhs_hint=m, timing=record, stage_balance=True)
        fac.solve(F1, "N")
        fac.solve(F2, "T")
        if record:
            for key, val in fac.timings().items():
                stage_acc.setdefault(key, []).append(val)
        fac.free()

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    launches0 = spike.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        step(True)
    e1.record()
    torch.cuda.synchronize()
    launches = spike.kernel_launches() - launches0
    ms = e0.elapsed_time(e1)
    clocks = sampler.stop() if sampler else None
    bytes_step = alg_bytes(n, k, m)
    ms, value, _ = aggregate_over_ranks(ms, bytes_step, args.steps, dist, dev)
    if dist:
        dist.barrier()
    peak_meas = spike.measure_fp64_peak(torch.cuda.current_stream().cuda_stream) if rank == 0 else None
    pipes = spike.measure_pipes(torch.cuda.current_stream().cuda_stream) if rank == 0 else None

    # accuracy of the last timed step (GPU residual from the original band)
    be_n = float(spike.backward_error(band, k, k, F1, F1src, "N").max())
    be_t = float(spike.backward_error(band, k, k, F2, F2src, "T").max())

    # mixed-precision variant (SPIKE_FLAG_MIXED: FP32 blocks + FP64 refinement) against plain FP64,
    # on this step (nrhs = m) and with nrhs = 1, where the factorization dominates.
    # the variant, tuning and serving legs run at N = 1 only (under torchrun they would run on
    # rank 0 alone while the other ranks hold their GPUs)
    extras = world == 1
    mixed = None
    if not args.no_mixed and extras:
        def variant(nr, use_mixed):
            A1, A2 = F1src[:nr], F2src[:nr]
            B1, B2 = torch.empty_like(A1), torch.empty_like(A2)
            stg, refs = {}, []

            def one(record):
                B1.copy_(A1)
                B2.copy_(A2)
                fac = spike.Factorization(band, k, k, p, nrhs_hint=nr, timing=record, stage_balance=True,
                                          mixed=use_mixed)
                fac.solve(B1, "N")
                r1 = fac.info()["refine_steps"]
                fac.solve(B2, "T")
                r2 = fac.info()["refine_steps"]
                if record:
                    for key, val in fac.timings().items():
                        stg.setdefault(key, []).append(val)
                    refs.append((r1, r2))
                fac.free()

            for _ in range(max(1, args.warmup)):
                one(False)
            torch.cuda.synchronize()
            v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            v0.record()
            for _ in range(args.steps):
                one(True)
            v1.record()
            torch.cuda.synchronize()
            vms = v0.elapsed_time(v1) / args.steps
            out = {"ms_per_step": vms, "value": alg_bytes(n, k, nr) / (vms * 1e-3) / 1e9,
                   "backward_error_N": float(spike.backward_error(band, k, k, B1, A1, "N").max()),
                   "backward_error_T": float(spike.backward_error(band, k, k, B2, A2, "T").max()),
                   "stages_ms": {key: round(float(np.mean(v)), 3) for key, v in stg.items()}}
            if use_mixed:
                out["refine_steps_N_T"] = refs[-1]
                # the FP32 block stage (block LU + fused spike sweeps) against the FP32 FMA peak
                _, po, pf = spike.plan(n, k, k, p, nrhs_hint=nr, stage_balance=True)
                bl = method_flops(po, pf, k, nr)["block_lu"] / (out["stages_ms"]["block_lu"] * 1e-3) / 1e12
                out["block_stage_fp32"] = {"tflops": bl, "frac_fp32_peak": bl / FP32_PEAK_TFLOPS,
                                           "peak_note": "derived FP32 FMA peak %.2f TFLOP/s (152 SMs x 128 FMA/clk x 2 "
                                                        "flop x 2.07 GHz)" % FP32_PEAK_TFLOPS}
            return out

        mx = variant(m, True)
        f1 = variant(1, False)
        m1 = variant(1, True)
        tres = tensor_residual_leg(band, k, torch.from_numpy(pr["xstar"]).to(dev), F1src, F2src, p)
        mixed = {"method": "FP32 block factorizations and sweeps, FP64 spike tips and reduced system, FP64 "
                           "iterative refinement to backward error <= 1e-14 (SPIKE_FLAG_MIXED), residuals "
                           "on the tensor cores to FP64 accuracy",
                 "tensor_residual": tres,
                 "unit": "GB/s",
                 "nrhs_%d" % m: dict(mx, speedup_vs_fp64=(ms / args.steps) / mx["ms_per_step"]),
                 "nrhs_1": {"fp64": f1, "mixed": m1, "speedup_vs_fp64": f1["ms_per_step"] / m1["ms_per_step"]}}

    # e2e: same metric through the C ABI with pinned host buffers
    band_h = torch.from_numpy(pr["band"]).pin_memory()
    F1h = torch.empty((m, n), dtype=torch.float64).pin_memory()
    F2hp = torch.empty((m, n), dtype=torch.float64).pin_memory()
    e2e_s, e2e_phase = 0.0, {}
    if args.no_e2e:
        args.e2e_steps = 0
    e2e_warm = max(1, args.warmup)  # the same W untimed steps as the device-timed leg
    for it in range(e2e_warm + args.e2e_steps if args.e2e_steps > 0 else 0):
        F1h.copy_(torch.from_numpy(pr["F"]))
        F2hp.copy_(torch.from_numpy(F2h))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fac = spike.Factorization(band_h.numpy(), k, k, p, nrhs_hint=m, stream=0, stage_balance=True)
        t1 = time.perf_counter()  # each call returns once its stream is idle (results read back)
        fac.solve(F1h.numpy(), "N")
        t2 = time.perf_counter()
        fac.solve(F2hp.numpy(), "T")
        t3 = time.perf_counter()
        fac.free()
        t4 = time.perf_counter()
        dt = t4 - t0
        if it >= e2e_warm:
            e2e_s += dt
            for key, v in zip(("factor", "solve_n", "solve_t", "free"), (t1 - t0, t2 - t1, t3 - t2, t4 - t3)):
                e2e_phase.setdefault(key, []).append(1e3 * v)
    e2e_step_s = e2e_s / args.e2e_steps if args.e2e_steps > 0 else float("nan")
    e2e_ms, e2e_value = e2e_step_s * 1e3, world * bytes_step / e2e_step_s / 1e9
    if dist is not None and args.e2e_steps > 0:  # max over ranks, as for the device-timed value
        e2e_ms, e2e_value, _ = aggregate_over_ranks(e2e_ms, bytes_step, 1, dist, dev)

    mixed_workload = None
    if not args.no_mixed and extras:
        mixed_workload = mixed_workload_leg(dev)
    grid = config_grid_leg(dev) if extras and not args.no_grid else None
    pivoting = pivoting_leg(dev) if extras and not args.no_pivot else None
    graphs = graphs_leg(dev) if extras and not args.no_tune else None
    tuning = None
    if not args.no_tune and extras:
        tuning = tuning_leg(band, k, m)
    cpu_serve = None
    if not args.no_serve and not args.no_cpu and extras:
        cpu_serve = cpu_serving_baseline()
    serving = None
    if not args.no_serve and extras:
        serving = serving_leg(dev, args.serve_requests, args.serve_streams, args.serve_batch, args.serve_passes,
                              batch_systems=args.serve_batch_systems, evict=args.serve_evict,
                              fp64_residual=not args.serve_tensor_residual)
        serving["cpu_baseline"] = cpu_serve

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    st = {key: float(np.mean(v)) for key, v in stage_acc.items()}
    lu_ms = st.get("block_lu", float("nan"))
    achieved = fl["block_lu"] / (lu_ms * 1e-3) / 1e12
    traffic, tinfo = load_traffic()
    step_tflops = fl["step"] / (ms / args.steps * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload, "n": n, "kl": k, "ku": k, "p": p, "nrhs": m, "dd": dd,
                   "blocks": info["leaves"], "partitions": info["P"], "pairs_2x2": info["r"],
                   "l2": "inputs larger than L2 (band %.2f GB per step)" % (8.0 * n * (2 * k + 1) / 1e9),
                   "planner": "stage-balanced sizing (SPIKE_FLAG_STAGE_BALANCE: R13 = %.3g)" % info["R13"],
                   "parallelism": "replicas x%d" % world},
        "roofline": {"bound": "alu", "kernel": "k_factor_nopiv (block LU + all spike sweeps of the block)",
                     "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic, "peak_note": FP64_PEAK_NOTE,
                     "peak_measured": peak_meas, "frac_of_measured": achieved / peak_meas if peak_meas else None,
                     "flops_per_launch": fl["block_lu"], "mean_launch_ms": lu_ms},
        "step_roofline": {"method_tflop_per_step": fl["step"] / 1e12, "achieved_tflops": step_tflops,
                          "frac_fp64": step_tflops / FP64_PEAK_TFLOPS,
                          "lu_equivalent_tflop_per_step": (2.0 * n * k * k + 3 * 4.0 * n * k * m) / 1e12},
        "stages_ms": st,
        "accuracy": {"backward_error_N": be_n, "backward_error_T": be_t},
        "e2e": {"value": e2e_value, "unit": "GB/s",
                "h2d_bytes_per_step": int(8 * n * (2 * k + 1) + 2 * 8 * n * m),
                "d2h_bytes_per_step": int(2 * 8 * n * m), "steps": args.e2e_steps, "warmup": e2e_warm,
                "ms_per_step": e2e_ms,
                "phases_ms": {key: round(float(np.mean(v)), 2) for key, v in e2e_phase.items()}},
        "variants": {"mixed_fp32_fp64_refinement": mixed, "mixed_precision_workload": mixed_workload,
                     "large_dominant_grid": grid, "pivoting_workload": pivoting,
                     "cuda_graphs_repeated_solves": graphs},
        "serving": serving,
        "tuning": tuning,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "pipes": pipes,
    }
    if not args.no_cpu and rank == 0 and world == 1:  # the CPU baseline is a single-GPU figure
        line["cpu_baseline"] = cpu_oracle_sample(k, m, dd, args.cpu_sample, seed)
        line["cpu_baseline"].pop("seconds", None)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
