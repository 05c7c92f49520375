#!/usr/bin/env python3
"""Benchmark of the downsampling hot path on GB300.

Workload (one step): MinMax and M4, n_out = 2000, over one series of
n = 10^9 float32 random-walk values (cumsum of N(0,1) steps) with int64
sorted, non-equidistant x (0 then a cumsum of geometric(0.5) gaps).  Inputs
are drawn on the device with a seeded generator and stay resident in HBM; at
4 GB of y (8 GB of x) they are far larger than the 129 MB L2, so no flush is
needed between steps.

Metric: input GB/s = algorithmic input bytes / time, where a step's bytes are
n*4 for each of the two algorithms plus the x reads of the bin-edge searches
((nb+1)*ceil(log2 n)*8 per algorithm).  The line also reports the roofline of
the dominant kernel (the streaming argmin/argmax, n*4 bytes per launch, timed
by CUDA events on its stream) against the measured copy bandwidth and against
a read-only streaming ceiling measured in the same run (tsds_read_stream over
the resident y), an end-to-end figure through the public API with pinned host
buffers, and the CPU oracle timed on a bounded sample.

--impl reference times the CPU oracle itself on the host cores (the paper's
own implementation is CPU code that is not available here).
Under torchrun each rank runs an independent series (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_DEFAULT = 10 ** 9
N_OUT = 2000
ALGOS = ("minmax", "m4")
METRIC = "input GB/s and % of GB300 HBM peak per algorithm"
WORKLOAD = ("single series n=1e9 float32 random walk with int64 sorted non-equidistant x "
            "(geometric(0.5) gaps), n_out=2000, MinMax + M4")


def workload_name(n, n_out, no_x=False, dtype="float32"):
    """The default step's workload, or the same recipe at other sizes (profiling runs)."""
    if n == N_DEFAULT and n_out == N_OUT and not no_x and dtype == "float32":
        return WORKLOAD
    values = "float32 random walk" if dtype == "float32" else f"{dtype} uniform over a quarter of its range"
    xs = "no x" if no_x else "int64 sorted non-equidistant x (geometric(0.5) gaps)"
    return f"single series n={n:.4g} {values} with {xs}, n_out={n_out}, MinMax + M4"


def l2_note(n, ysz=4, xsz=8):
    gb = n * ysz / 1e9
    if n * ysz > 129e6:
        xs = f", {n * xsz / 1e9:.4g} GB x" if xsz else ""
        return f"inputs larger than L2 ({gb:.4g} GB y{xs}); no flush"
    return f"y ({gb:.4g} GB) fits in L2: not an HBM measurement"


FALLBACK_HBM = 6800.0
DTYPE_SHORT = {"float32": "f32", "float64": "f64", "float16": "f16", "int8": "i8", "int16": "i16", "int32": "i32",
               "int64": "i64", "uint8": "u8", "uint16": "u16", "uint32": "u32", "uint64": "u64"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--cpu-sample", type=int, default=250_000_000)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--n-out", type=int, default=N_OUT, help="n_out of the default step (profiling other bin sizes)")
    ap.add_argument("--no-x", action="store_true", help="the default step without x (index bins; profiling runs)")
    ap.add_argument("--dtype", default="float32",
                    help="y dtype of the default step (float32: random walk; others: quarter-range values; profiling runs)")
    ap.add_argument("--dtypes", default=None, help="dtypes suite: a comma-separated subset of the eleven dtypes")
    ap.add_argument("--batched-plan-only", action="store_true",
                    help="batched suite: only the resident plan with its default shape (profiling runs)")
    ap.add_argument("--serve-series", type=int, default=32, help="resident series of the serve suite")
    ap.add_argument("--serve-n", type=int, default=100_000_000, help="points per resident series of the serve suite")
    ap.add_argument("--serve-algos", default="minmax,m4,minmaxlttb", help="algorithms the serve suite draws from")
    ap.add_argument("--serve-burst-only", type=int, default=0,
                    help="serve suite: only a warm-up and one burst of this many queries (profiling runs)")
    ap.add_argument("--batch-count", type=int, default=4096, help="series in the batched suite (smaller for profiling)")
    ap.add_argument("--stream-variant", default="auto", choices=["auto", "ring", "ldg", "seg", "grp"],
                    help="kernel variant of the streaming pass (tsds_stream_variant)")
    ap.add_argument("--suite", default=None, choices=["dtypes", "config1", "lttb", "batched", "serve", "values"],
                    help="instead of the headline step, measure one of the other workloads and print one JSON line")
    return ap.parse_args()


# ----------------------------------------------------------------------------- other workloads

def _timed_calls(torch, stream, fn, reps):
    """Median and mean device time (ms) of `fn()` over reps, one event pair each."""
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times), sum(times) / len(times)


def _raw_call(binding, algo, x, x_dtype, y, y_dtype, n, n_out, out, cnt, stream, nan=0, ratio=4):
    sp = binding.ctypes.c_void_p(stream.cuda_stream)
    xp = x.data_ptr() if x is not None else None
    xd = binding.DTYPES[x_dtype] if x is not None else 0
    if algo == "minmaxlttb":
        r = binding.tsds_minmaxlttb(xp, xd, y.data_ptr(), binding.DTYPES[y_dtype], n, n_out, ratio, nan,
                                    out.data_ptr(), cnt.data_ptr(), sp)
    else:
        fn = {"minmax": binding.tsds_minmax, "m4": binding.tsds_m4, "lttb": binding.tsds_lttb,
              "everynth": binding.tsds_everynth}[algo]
        r = fn(xp, xd, y.data_ptr(), binding.DTYPES[y_dtype], n, n_out, nan, out.data_ptr(), cnt.data_ptr(), sp)
    if r != 0:
        raise RuntimeError(binding.last_error())


def suite_dtypes(args):
    """Config of the paper's Table 1 at 4 GB per dtype: n*itemsize = 4e9, values uniform over a
    quarter of the dtype range, int64 geometric x, n_out = 2000, MinMax and M4."""
    import numpy as np
    import torch

    import paper_2307_05389_gb300 as pkg
    from paper_2307_05389_gb300 import binding, inputs
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    peak, peak_src = hbm_peak()
    res = {}
    x = None
    x_n = 0
    out = torch.empty(N_OUT, dtype=torch.int64, device=dev)
    cnt = torch.empty(1, dtype=torch.int64, device=dev)
    rpeak = None
    for d in (args.dtypes.split(",") if args.dtypes else inputs.DTYPES):
        size = np.dtype(d).itemsize
        n = 4_000_000_000 // size
        y = inputs.quarter_range_cuda(n, d, seed=2, device=dev)
        if x_n != n:
            x = None
            torch.cuda.empty_cache()
            x = inputs.geometric_x_cuda(n, seed=2, device=dev)
            x_n = n
        torch.cuda.synchronize()
        if rpeak is None:
            rpeak = read_peak(pkg, torch, y, stream)
        row = {"n": n}
        for algo in ALGOS:
            f = lambda: _raw_call(binding, algo, x, "int64", y, d, n, N_OUT, out, cnt, stream)
            for _ in range(2):
                f()
            pkg.tsds_timing_read()
            pkg.tsds_timing_enable(True)
            med, mean = _timed_calls(torch, stream, f, args.steps)
            pkg.tsds_timing_enable(False)
            km, kl = pkg.tsds_timing_read()
            b = step_bytes(n)[algo] - n * 4 + n * size
            kgb = n * size / (km / kl / 1e3) / 1e9
            row[algo] = {"call_ms": med, "call_GBps": b / (med / 1e3) / 1e9,
                         "kernel_GBps": kgb,
                         "pct_of_hbm_peak": 100.0 * b / (med / 1e3) / 1e9 / peak}
            if rpeak:
                row[algo]["kernel_pct_of_read_peak"] = 100.0 * kgb / rpeak
        res[d] = row
        del y
        torch.cuda.empty_cache()
    return {"suite": "dtypes", "metric": METRIC, "unit": "GB/s", "peak": peak, "peak_source": peak_src,
            "read_peak": rpeak,
            "config": {"workload": "per dtype: n*itemsize = 4e9, quarter-range uniform values, int64 geometric x, "
                                   "n_out=2000, MinMax + M4", "reps": args.steps}, "results": res}


def suite_batched(args):
    """4096 float32 random-walk series, lengths round(10**U(3,7)) (seed 3), n_out uniform in
    [200, 4000] rounded down to a multiple of 4, no x: one launch sequence per series vs the
    batched one-shot call vs a resident plan (autotuned launch shape, CUDA graph)."""
    import numpy as np
    import torch

    import paper_2307_05389_gb300 as pkg
    from paper_2307_05389_gb300 import binding, inputs
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    count = args.batch_count
    lens = inputs.batch_lengths(count, seed=3)
    n_outs = inputs.batch_n_out(count, seed=3)
    total = int(lens.sum())
    walk = inputs.random_walk_cuda(total, "float32", seed=3, device=dev)
    offs = np.concatenate([[0], np.cumsum(lens)])
    ys = [walk[int(offs[i]):int(offs[i + 1])] for i in range(count)]
    torch.cuda.empty_cache()
    res = {"series": count, "points": total, "GB": total * 4 / 1e9}
    sp = binding.ctypes.c_void_p(stream.cuda_stream)
    for algo in ALGOS:
        outs, counts = binding.batch_buffers(ys, n_outs, dev)
        fn = binding.tsds_minmax if algo == "minmax" else binding.tsds_m4

        def per_series():
            for i, y in enumerate(ys):
                r = fn(None, 0, y.data_ptr(), binding.DTYPES["float32"], y.shape[0], int(n_outs[i]), 0,
                       outs[i].data_ptr(), counts[i:i + 1].data_ptr(), sp)
                if r != 0:
                    raise RuntimeError(binding.last_error())

        def snapshot():
            torch.cuda.synchronize()
            c = counts.clone()
            return c, [o[:int(k)].clone() for o, k in zip(outs, c.tolist())]

        if args.batched_plan_only:
            # profiling runs: the resident plan alone (default launch shape, CUDA graph)
            plan = binding.Plan(algo, ys, n_outs, graph=True, autotune=False)
            plan.execute()
            t_p, _ = _timed_calls(torch, stream, plan.execute, max(3, args.steps // 10))
            res[algo] = {"plan_graph_ms": t_p, "plan_GBps": total * 4 / (t_p / 1e3) / 1e9, "plan": plan.info()}
            plan.close()
            continue
        per_series()
        ref_c, ref_o = snapshot()
        t_ps, _ = _timed_calls(torch, stream, per_series, 3)

        def batched():
            binding.downsample_batched(algo, ys, n_outs, outs=outs, counts=counts)
        counts.fill_(-1)
        batched()
        b_c, b_o = snapshot()
        t_b, _ = _timed_calls(torch, stream, batched, 5)

        plan = binding.Plan(algo, ys, n_outs, graph=True, autotune=True)
        plan.execute()
        torch.cuda.synchronize()
        p_c = plan.counts.clone()
        p_o = [o[:int(k)].clone() for o, k in zip(plan.outs, p_c.tolist())]
        t_p, _ = _timed_calls(torch, stream, plan.execute, max(5, args.steps // 10))
        same = bool(torch.equal(ref_c, b_c) and all(torch.equal(a, b) for a, b in zip(ref_o, b_o)))
        same_plan = bool(torch.equal(ref_c, p_c) and all(torch.equal(a, b) for a, b in zip(ref_o, p_o)))
        res[algo] = {"per_series_ms": t_ps, "batched_ms": t_b, "plan_graph_ms": t_p,
                     "per_series_GBps": total * 4 / (t_ps / 1e3) / 1e9,
                     "batched_GBps": total * 4 / (t_b / 1e3) / 1e9,
                     "plan_GBps": total * 4 / (t_p / 1e3) / 1e9,
                     "speedup_batched": t_ps / t_b, "speedup_plan": t_ps / t_p,
                     "identical_to_per_series": same and same_plan, "plan": plan.info()}
        plan.close()
    peak, peak_src = hbm_peak()
    return {"suite": "batched", "unit": "ms", "peak": peak, "peak_source": peak_src,
            "config": {"workload": "4096 float32 random-walk series, lengths log-uniform [1e3, 1e7] (seed 3), "
                                   "n_out uniform [200, 4000] (multiple of 4), no x; actual total reported"},
            "results": res}


def suite_values(args):
    """Fused value gather on the headline workload (1e9 float32 random walk, int64 geometric x,
    n_out = 2000) and on LTTB (1e7 float64 walk, n_out = 4000): the index-only call, the *_values
    call (indices plus x and y values from the same kernels), and the unfused alternative (the
    index call, then torch gathers of x and y by the indices over the full output buffer)."""
    import torch

    from paper_2307_05389_gb300 import binding, inputs
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    sp = binding.ctypes.c_void_p(stream.cuda_stream)
    res = {}
    cases = [("minmax", 1_000_000_000, "float32", True, 2000), ("m4", 1_000_000_000, "float32", True, 2000),
             ("everynth", 1_000_000_000, "float32", True, 2000),
             ("lttb", 10_000_000, "float64", False, 4000), ("minmaxlttb", 10_000_000, "float64", False, 4000)]
    cache = {}
    for algo, n, dt, with_x, n_out in cases:
        key = (n, dt, with_x)
        if key not in cache:
            cache.clear()
            torch.cuda.empty_cache()
            y = inputs.random_walk_cuda(n, dt, seed=2, device=dev)
            x = inputs.geometric_x_cuda(n, seed=2, device=dev) if with_x else None
            cache[key] = (y, x)
        y, x = cache[key]
        # zeros: entries past the count (empty bins) stay a valid index for the torch gathers
        out = torch.zeros(n_out, dtype=torch.int64, device=dev)
        cnt = torch.empty(1, dtype=torch.int64, device=dev)
        yo = torch.empty(n_out, dtype=y.dtype, device=dev)
        xo = torch.empty(n_out, dtype=torch.int64, device=dev) if with_x else None
        xp = x.data_ptr() if with_x else None
        xd = binding.DTYPES["int64"] if with_x else 0
        common = (xp, xd, y.data_ptr(), binding.DTYPES[dt], n, n_out)

        def plain():
            _raw_call(binding, algo, x, "int64" if with_x else None, y, dt, n, n_out, out, cnt, stream)

        def fused():
            tail = (out.data_ptr(), cnt.data_ptr(), xo.data_ptr() if with_x else None, yo.data_ptr(), sp)
            if algo == "minmaxlttb":
                r = binding.tsds_minmaxlttb_values(*common, 4, 0, *tail)
            else:
                r = {"minmax": binding.tsds_minmax_values, "m4": binding.tsds_m4_values,
                     "lttb": binding.tsds_lttb_values, "everynth": binding.tsds_everynth_values}[algo](*common, 0,
                                                                                                     *tail)
            if r != 0:
                raise RuntimeError(binding.last_error())

        def unfused():
            plain()
            torch.index_select(y, 0, out, out=yo)
            if with_x:
                torch.index_select(x, 0, out, out=xo)
        for f in (plain, fused, unfused):
            f()
        reps = max(10, args.steps // 5)
        t_plain, _ = _timed_calls(torch, stream, plain, reps)
        t_fused, _ = _timed_calls(torch, stream, fused, reps)
        t_unfused, _ = _timed_calls(torch, stream, unfused, reps)
        torch.cuda.synchronize()
        k = int(cnt.item())
        same = bool(torch.equal(yo[:k], y[out[:k]]) and (not with_x or torch.equal(xo[:k], x[out[:k]])))
        res[algo] = {"n": n, "y": dt, "x": "int64" if with_x else None, "n_out": n_out, "index_only_ms": t_plain,
                     "fused_values_ms": t_fused, "index_then_torch_gather_ms": t_unfused,
                     "fused_overhead_us": (t_fused - t_plain) * 1e3, "values_match": same}
    return {"suite": "values", "unit": "ms", "config": {"workload": "headline MinMax/M4 (1e9 float32, int64 x, "
            "n_out=2000) and LTTB/MinMaxLTTB(4) on a 1e7 float64 walk (n_out=4000)"}, "results": res}


def suite_serve(args):
    """32 resident float32 random walks of 1e8 points with float64 x (cumsum of exponential(1)).
    Poisson-arriving viewport queries: a series uniformly, a span log-uniform in [1e4, 1e8] points
    at a uniform start (sent as an x range), n_out from {500, 1000, 2000, 4000}, algorithm from
    MinMax / M4 / MinMaxLTTB(ratio 4).  Per arrival rate: p50/p99 submission-to-result latency,
    completed queries/s and GB/s of y inside the ranges; plus the same queries issued one call
    at a time through the single-series entry points for comparison."""
    import numpy as np
    import torch

    from paper_2307_05389_gb300 import binding, inputs
    dev = torch.device("cuda", 0)
    nser, n = args.serve_series, args.serve_n
    algos = args.serve_algos.split(",")
    ys = [inputs.random_walk_cuda(n, "float32", seed=500 + i, device=dev) for i in range(nser)]
    xs = [inputs.exponential_x_cuda(n, seed=600 + i, device=dev) for i in range(nser)]
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    xh = [x[::1000].cpu().numpy() for x in xs]   # coarse host copy to pick x ranges from
    rng = np.random.default_rng(5)

    def draw(k):
        qs = []
        for _ in range(k):
            s = int(rng.integers(0, nser))
            span = int(10 ** rng.uniform(4, np.log10(n)))
            start = int(rng.integers(0, n - span + 1))
            lo_x = float(xh[s][min(start // 1000, len(xh[s]) - 1)])
            hi_x = float(xh[s][min((start + span) // 1000, len(xh[s]) - 1)])
            qs.append((s, algos[int(rng.integers(0, len(algos)))],
                       int([500, 1000, 2000, 4000][int(rng.integers(0, 4))]), lo_x, hi_x))
        return qs

    srv = binding.Server("float32", "float64", streams=4, max_batch=256, memory_budget=8 << 30)
    ids = [srv.add_series(y, x) for y, x in zip(ys, xs)]
    res = {}
    # warm-up (autotune-free path; first batches allocate pinned buffers)
    for t in [srv.submit(ids[s], a, k, x_range=(l, h)) for s, a, k, l, h in draw(64)]:
        srv.result(t)
    if args.serve_burst_only:
        qs = draw(args.serve_burst_only)
        srv.reset_stats()
        tickets = [srv.submit(ids[s], a, k, x_range=(l, h)) for s, a, k, l, h in qs]
        for t in tickets:
            srv.result(t)
        st = srv.stats()
        srv.close()
        return {"suite": "serve", "unit": "ms", "config": {
            "workload": f"{nser} x {n:.3g} float32 random walks, float64 x; one burst of {len(qs)} viewport queries "
                        f"({'/'.join(algos)})"},
            "results": {"burst": {"achieved_qps": st["completed"] / st["span_s"], "p50_ms": st["p50_us"] / 1e3,
                                  "p99_ms": st["p99_us"] / 1e3, "GBps": st["bytes"] / st["span_s"] / 1e9,
                                  "batches": st["batches"]}}}
    for rate in (1e2, 1e3, 1e4, 1e5):
        count = int(min(max(200, rate * 2.0), 4000))
        qs = draw(count)
        gaps = rng.exponential(1.0 / rate, count)
        srv.reset_stats()
        t0 = time.perf_counter()
        due = t0
        tickets = []
        for (s, a, k, l, h), g in zip(qs, gaps):
            due += g
            while time.perf_counter() < due:
                pass
            tickets.append(srv.submit(ids[s], a, k, x_range=(l, h)))
        for t in tickets:
            srv.result(t)
        st = srv.stats()
        res[f"rate_{int(rate)}"] = {"queries": count, "offered_qps": rate,
                                    "achieved_qps": st["completed"] / max(st["span_s"], 1e-9),
                                    "p50_ms": st["p50_us"] / 1e3, "p99_ms": st["p99_us"] / 1e3,
                                    "mean_ms": st["mean_us"] / 1e3, "batches": st["batches"],
                                    "GBps": st["bytes"] / max(st["span_s"], 1e-9) / 1e9,
                                    "mean_points_per_query": st["points"] / max(st["completed"], 1)}
    # saturation: every query submitted at once
    qs = draw(2000)
    srv.reset_stats()
    tickets = [srv.submit(ids[s], a, k, x_range=(l, h)) for s, a, k, l, h in qs]
    for t in tickets:
        srv.result(t)
    st = srv.stats()
    res["burst_2000"] = {"achieved_qps": st["completed"] / st["span_s"], "p50_ms": st["p50_us"] / 1e3,
                         "p99_ms": st["p99_us"] / 1e3, "GBps": st["bytes"] / st["span_s"] / 1e9,
                         "batches": st["batches"]}
    srv.close()
    # the same kind of queries one call at a time (range found by searchsorted on the device)
    qs = draw(300)
    stream = torch.cuda.current_stream(dev)
    out = torch.empty(4096, dtype=torch.int64, device=dev)
    cnt = torch.empty(1, dtype=torch.int64, device=dev)
    tot_pts = 0
    t0 = time.perf_counter()
    for s, a, k, l, h in qs:
        lo = int(torch.searchsorted(xs[s], torch.tensor([l], device=dev, dtype=torch.float64)).item())
        hi = int(torch.searchsorted(xs[s], torch.tensor([h], device=dev, dtype=torch.float64), right=True).item())
        tot_pts += hi - lo
        if hi - lo <= 0:
            continue
        _raw_call(binding, a, xs[s][lo:hi], "float64", ys[s][lo:hi], "float32", hi - lo, k, out, cnt, stream)
        int(cnt.item())
    dt = time.perf_counter() - t0
    res["one_call_per_query"] = {"queries": len(qs), "qps": len(qs) / dt, "GBps": tot_pts * 4 / dt / 1e9,
                                 "mean_ms": dt / len(qs) * 1e3}
    return {"suite": "serve", "unit": "ms", "config": {
        "workload": f"{nser} x {n:.3g} float32 random walks, float64 x = cumsum(exponential(1)); Poisson viewport "
                    f"queries, span log-uniform [1e4, {n:.3g}] points, n_out in {{500,1000,2000,4000}}, "
                    f"{'/'.join(algos)} (MinMaxLTTB ratio 4)",
        "server": {"streams": 4, "max_batch": 256, "memory_budget_GiB": 8}}, "results": res}


def suite_config1(args):
    """10^6-point float32 random walk (seed 0), no x, n_out = 1000: latency of each algorithm
    (EveryNth included: the paper reports it as constant time, Section 4)."""
    import torch

    from paper_2307_05389_gb300 import binding, inputs
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    n, n_out = 1_000_000, 1000
    y = torch.from_numpy(inputs.random_walk(n, "float32", seed=0)).to(dev)
    out = torch.empty(n_out, dtype=torch.int64, device=dev)
    cnt = torch.empty(1, dtype=torch.int64, device=dev)
    res = {}
    for algo in ("minmax", "m4", "lttb", "minmaxlttb", "everynth"):
        f = lambda: _raw_call(binding, algo, None, None, y, "float32", n, n_out, out, cnt, stream)
        for _ in range(5):
            f()
        med, mean = _timed_calls(torch, stream, f, max(20, args.steps))
        res[algo] = {"median_us": med * 1e3, "mean_us": mean * 1e3, "GBps": n * 4 / (med / 1e3) / 1e9}
    return {"suite": "config1", "unit": "us", "config": {"workload": "n=1e6 float32 random walk (seed 0), no x, "
            "n_out=1000, minmax_ratio=4; 4 MB is L2-resident: latency, not % of HBM"}, "results": res}


def suite_lttb(args):
    """Plain LTTB on one float64 random walk of 1e7 points and MinMaxLTTB on 64 float64
    series of 1e8/64 points (random walk quantised to 256 levels, 1 % NaN), n_out = 4000."""
    import torch

    from paper_2307_05389_gb300 import binding, inputs
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    res = {}
    n_out = 4000
    out = torch.empty(n_out, dtype=torch.int64, device=dev)
    cnt = torch.empty(1, dtype=torch.int64, device=dev)
    for n, dt in ((10_000_000, "float64"), (10_000_000, "float32"), (1_000_000, "float32")):
        y = torch.from_numpy(inputs.random_walk(n, dt, seed=4)).to(dev)
        f = lambda: _raw_call(binding, "lttb", None, None, y, dt, n, n_out, out, cnt, stream)
        f()
        med, _ = _timed_calls(torch, stream, f, 3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f()
        issue = (time.perf_counter() - t0) * 1e3
        torch.cuda.synchronize()
        res[f"lttb_{dt}_{n}"] = {"ms": med, "GBps": n * y.element_size() / (med / 1e3) / 1e9,
                                 "us_per_bucket": med * 1e3 / (n_out - 2), "host_issue_ms": issue}
    series = [torch.from_numpy(inputs.quantised_nan(1_562_500, seed=4 + i)).to(dev) for i in range(64)]
    for nan, nm in ((0, "propagate"), (1, "ignore")):
        for r in (2, 4, 30):
            def f():
                for s in series:
                    _raw_call(binding, "minmaxlttb", None, None, s, "float64", s.numel(), n_out, out, cnt, stream,
                              nan=nan, ratio=r)
            f()
            med, _ = _timed_calls(torch, stream, f, 3)
            # host time to issue the 64 calls (no synchronisation inside): close to the
            # device time means the loop is bound by issuing launches, not by the GPU
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            f()
            issue = (time.perf_counter() - t0) * 1e3
            torch.cuda.synchronize()
            # the same 64 series as one batched call (tsds_batched_minmaxlttb)
            outs, counts = binding.batch_buffers(series, [n_out] * 64, dev)

            def fb():
                binding.downsample_batched("minmaxlttb", series, [n_out] * 64, nan=nm, outs=outs, counts=counts,
                                           minmax_ratio=r)
            fb()
            torch.cuda.synchronize()
            same = True
            c = counts.cpu().tolist()
            for k, srs in enumerate(series):
                _raw_call(binding, "minmaxlttb", None, None, srs, "float64", srs.numel(), n_out, out, cnt, stream,
                          nan=nan, ratio=r)
                torch.cuda.synchronize()
                same &= int(cnt.item()) == c[k] and torch.equal(out[:c[k]], outs[k][:c[k]])
            bmed, _ = _timed_calls(torch, stream, fb, 5)
            res[f"minmaxlttb_r{r}_{nm}"] = {"ms_64_series": med, "GBps": 1e8 * 8 / (med / 1e3) / 1e9,
                                            "host_issue_ms": issue, "batched_ms_64_series": bmed,
                                            "batched_GBps": 1e8 * 8 / (bmed / 1e3) / 1e9,
                                            "batched_identical": bool(same)}
    return {"suite": "lttb", "unit": "ms", "config": {"workload": "LTTB: float64/float32 random walks, n_out=4000; "
            "MinMaxLTTB: 64 x 1.5625e6 float64 quantised to 256 levels with 1% NaN, one call per series and "
            "one batched call for all 64"},
            "results": res}


def step_bytes(n, n_out=N_OUT, x_itemsize=8, y_itemsize=4):
    """Algorithmic input bytes of one MinMax and one M4 call: y read once, plus the x probes of the
    bin searches (x_itemsize 0: no x)."""
    per = {}
    for algo in ALGOS:
        nb = n_out // (2 if algo == "minmax" else 4)
        per[algo] = n * y_itemsize + (nb + 1) * math.ceil(math.log2(max(n, 2))) * x_itemsize
    return per


def oracle_all_cores(oracle, x, y, n_out):
    """The oracle's per-bin argmin/argmax (MinMax and M4 bins of the same sample) split over
    the host's cores by contiguous bin ranges, one thread each (the C oracle releases the
    GIL), as a second CPU line beside the single-threaded one."""
    import concurrent.futures
    cores = os.cpu_count() or 1
    n = len(y)
    t0 = time.perf_counter()
    for algo in ALGOS:
        nb = n_out // (2 if algo == "minmax" else 4)
        edges = oracle.bin_edges(x, n, nb)

        def work(b0, b1, edges=edges):
            return [oracle.argminmax(y, int(edges[b]), int(edges[b + 1])) for b in range(b0, b1) if edges[b + 1] > edges[b]]
        step = (nb + cores - 1) // cores
        with concurrent.futures.ThreadPoolExecutor(cores) as ex:
            list(ex.map(lambda b0: work(b0, min(b0 + step, nb)), range(0, nb, step)))
    dt = time.perf_counter() - t0
    return {"value": sum(step_bytes(n, n_out).values()) / dt / 1e9, "unit": "GB/s", "cores": cores,
            "kind": "oracle per-bin argmin/argmax, bins split over threads",
            "sample": f"the same {n} points, MinMax + M4 bins once each ({dt:.2f} s)"}


def aggregate_ranks(ms_local, bytes_local, dist=None, device=None):
    """Whole-job numbers of a timed region: (the slowest rank's milliseconds,
    the bytes all ranks processed, GB/s of the whole job).  Every rank must
    call it (collectives); with dist None it is the single-rank case."""
    import torch
    ms = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    by = torch.tensor([float(bytes_local)], dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(ms, op=dist.ReduceOp.MAX)
        dist.all_reduce(by, op=dist.ReduceOp.SUM)
    ms_max, total = float(ms.item()), float(by.item())
    return ms_max, total, total / (ms_max / 1e3) / 1e9


def stream_kernel_name(n, n_out, forced, itemsize=4, has_x=True):
    """The streaming kernel a MinMax launch of this shape runs (the library's automatic rule for a
    single series: up to 256 MB a warp per bin with bins of at least 8 KB or at most 4096 bins of
    at most 64 KB, else lane groups below 8 KB mean bins; beyond 256 MB lane groups below 64 KB
    mean bins; register streaming above)."""
    v = forced
    nb = max(n_out // 2, 1)
    bytes_ = n * itemsize
    if v == "auto":
        big = bytes_ > 256 << 20
        small = (not big) and bytes_ <= nb * 65536 and (nb <= 4096 or bytes_ >= 8192 * nb)
        limit = 65536 if big else 8192
        v = "small" if small else "grp" if bytes_ / nb < limit else "ldg"
    return {"ldg": "tsds::k_argminmax_ldg (register streaming)", "seg": "tsds::k_argminmax_seg (segmented)",
            "ring": "tsds::k_argminmax (shared-memory ring)", "grp": "tsds::k_argminmax_grp (lane groups)",
            "small": "tsds::k_small (a warp per bin)"}[v] + " — streaming per-bin argmin/argmax"


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


def kernel_traffic():
    """DRAM bytes per launch from the committed ncu summary, only while the
    kernel source still matches the one profiled."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "argminmax_traffic.json")) as f:
            rec = json.load(f)
        h = hashlib.sha256()
        for s in rec["sources"]:
            h.update(open(os.path.join(ROOT, s), "rb").read())
        if h.hexdigest() != rec.get("sources_sha256"):
            return None
        return rec.get("dram_bytes_per_launch_full_size")
    except Exception:
        return None


def read_peak(pkg, torch, y, stream, reps=10):
    """Read-only streaming ceiling: median GB/s of the library's read probe
    (tsds_read_stream: every byte once, 16-byte loads) over the resident y."""
    per16 = max(1, 16 // y.element_size())
    buf = y[: (y.numel() // per16) * per16]
    nbytes = buf.numel() * buf.element_size()
    if nbytes == 0:
        return None
    sink = torch.zeros(1, dtype=torch.int64, device=y.device)
    for _ in range(2):
        pkg.read_stream(buf, sink, stream)
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pkg.read_stream(buf, sink, stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return nbytes / (statistics.median(times) / 1e3) / 1e9


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        import torch
        self.path = tempfile.mktemp(prefix="tsds_clocks_", suffix=".csv")
        sel = []
        try:
            u = str(torch.cuda.get_device_properties(device_index).uuid)
            sel = ["--id=" + (u if u.startswith("GPU-") else "GPU-" + u)]
        except Exception:
            sel = []
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", *sel, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [t.strip() for t in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
                power.append(float(p[3]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


# ----------------------------------------------------------------------------- reference arm

def run_reference(args, rank):
    import numpy as np

    import oracle
    from paper_2307_05389_gb300 import inputs
    if rank != 0:
        return
    n = min(args.cpu_sample, args.n) // 5          # one step of the reference: a bounded sample
    y = inputs.random_walk(n, "float32", seed=2)
    x = inputs.geometric_x(n, seed=2)
    oracle.build()
    for _ in range(args.warmup):
        for algo in ALGOS:
            oracle.downsample(algo, x, y, args.n_out)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for algo in ALGOS:
            oracle.downsample(algo, x, y, args.n_out)
    dt = time.perf_counter() - t0
    per = step_bytes(n, args.n_out)
    gbs = sum(per.values()) * args.steps / dt / 1e9
    sample = f"first {n} points of the workload (numpy default_rng seed 2), MinMax + M4, single-threaded C oracle"
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n_sample": n, "n_out": args.n_out},
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- native arm

def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.suite:
        import paper_2307_05389_gb300 as pkg
        pkg.load()
        fn = {"dtypes": suite_dtypes, "config1": suite_config1, "lttb": suite_lttb, "batched": suite_batched,
              "serve": suite_serve, "values": suite_values}[args.suite]
        clocks = ClockSampler(0)
        out = fn(args)
        out["clocks"] = clocks.stop()
        print(json.dumps(out), flush=True)
        return

    import numpy as np
    import torch

    import paper_2307_05389_gb300 as pkg
    from paper_2307_05389_gb300 import binding, inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    pkg.load()
    if args.stream_variant != "auto":
        binding.tsds_stream_variant(args.stream_variant)

    n = args.n
    if np.dtype(args.dtype).kind == "u":
        args.no_e2e = True   # the host-buffer API takes torch tensors, which have no unsigned 16-64-bit types
    if args.dtype == "float32":
        y = inputs.random_walk_cuda(n, "float32", seed=2 + rank, device=dev)
    else:
        y = inputs.quarter_range_cuda(n, args.dtype, seed=2 + rank, device=dev)
    x = None if args.no_x else inputs.geometric_x_cuda(n, seed=2 + rank, device=dev)
    outs = {a: torch.empty(args.n_out, dtype=torch.int64, device=dev) for a in ALGOS}
    cnts = {a: torch.empty(1, dtype=torch.int64, device=dev) for a in ALGOS}
    torch.cuda.synchronize()
    torch.cuda.empty_cache()               # drop the generators' temporaries
    stream = torch.cuda.current_stream(dev)
    sp = binding.ctypes.c_void_p(stream.cuda_stream)
    fns = {"minmax": binding.tsds_minmax, "m4": binding.tsds_m4}

    def call(algo):
        r = fns[algo](x.data_ptr() if x is not None else None, binding.DTYPES["int64"] if x is not None else 0,
                      y.data_ptr(), binding.DTYPES[args.dtype], n, args.n_out,
                      0, outs[algo].data_ptr(), cnts[algo].data_ptr(), sp)
        if r != 0:
            raise RuntimeError(binding.last_error())

    def step():
        for a in ALGOS:
            call(a)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, CUDA events on the launching stream
    clocks = ClockSampler(local)
    time.sleep(0.2)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    pkg.tsds_timing_read()                 # drop anything recorded before
    pkg.tsds_timing_enable(True)
    launches0 = pkg.tsds_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = pkg.tsds_kernel_launches() - launches0
    pkg.tsds_timing_enable(False)
    ms = ev0.elapsed_time(ev1)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    kern_ms, kern_launches = pkg.tsds_timing_read()
    ysz = np.dtype(args.dtype).itemsize
    xsz = 0 if x is None else 8
    per = step_bytes(n, args.n_out, xsz, ysz)
    ms_max, total_bytes, value = aggregate_ranks(ms, sum(per.values()) * args.steps, dist, dev)
    peak, peak_src = hbm_peak()
    kern_avg_ms = kern_ms / max(kern_launches, 1)
    achieved = n * ysz / (kern_avg_ms / 1e3) / 1e9

    # ---- per-algorithm breakdown (whole call and streaming kernel)
    per_algo = {}
    for a in ALGOS:
        reps = max(10, args.steps // 4)
        pkg.tsds_timing_read()
        pkg.tsds_timing_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            call(a)
        e1.record(stream)
        torch.cuda.synchronize()
        pkg.tsds_timing_enable(False)
        km, kl = pkg.tsds_timing_read()
        call_ms = e0.elapsed_time(e1) / reps
        per_algo[a] = {"call_ms": call_ms, "call_GBps": per[a] / (call_ms / 1e3) / 1e9,
                       "kernel_ms": km / max(kl, 1), "kernel_GBps": n * ysz / (km / max(kl, 1) / 1e3) / 1e9,
                       "pct_of_hbm_peak": 100.0 * per[a] / (call_ms / 1e3) / 1e9 / peak}

    rpeak = read_peak(pkg, torch, y, stream)

    # ---- end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        yh = y.cpu().pin_memory()
        xh = x.cpu().pin_memory() if x is not None else None
        yd, xd = torch.empty_like(y), (torch.empty_like(x) if x is not None else None)
        pkg.downsample_host(ALGOS, yh, args.n_out, x=xh, y_dev=yd, x_dev=xd)   # warm-up
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        d2h = 0
        for _ in range(args.e2e_steps):
            res = pkg.downsample_host(ALGOS, yh, args.n_out, x=xh, y_dev=yd, x_dev=xd)
            d2h = sum(r.numel() * 8 + 8 for r in res)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        tt = torch.tensor([dt], device=dev)
        if dist:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        dt = float(tt.item())
        # y is copied to the device every step; the pinned x stays in host memory and the
        # bin search reads its probes in place ((nb+1) * ceil(log2 n) elements per call)
        probes = sum(per.values()) - 2 * n * ysz
        e2e = {"value": sum(per.values()) * args.e2e_steps * world / dt / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": int(yh.numel() * ysz), "d2h_bytes_per_step": int(d2h),
               "x_read_in_place_bytes_per_step": int(probes),
               "api": "paper_2307_05389_gb300.downsample_host -> tsds_downsample_host (pinned y copied in chunks that overlap the reduction, pinned x searched in place)"}
        del yh, xh, yd, xd

    # ---- CPU oracle on a bounded sample (rank 0)
    cpu = None
    if rank == 0 and not args.no_cpu:
        import oracle
        oracle.build()
        ns = min(args.cpu_sample, n)
        ys = y[:ns].cpu().numpy()
        if args.dtype != "float32" and np.dtype(args.dtype).kind == "u":
            ys = ys.view(np.dtype(args.dtype))
        xs = x[:ns].cpu().numpy() if x is not None else None
        t0 = time.perf_counter()
        for a in ALGOS:
            oracle.downsample(a, xs, ys, args.n_out)
        dt = time.perf_counter() - t0
        cpu = {"value": sum(step_bytes(ns, args.n_out, xsz, ysz).values()) / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"first {ns} points of the same series and x, MinMax + M4 once each ({dt:.1f} s)"}
        cpu["all_cores"] = oracle_all_cores(oracle, xs, ys, args.n_out)

    # ---- output check of the timed results against each other (counts)
    counts = {a: int(cnts[a].item()) for a in ALGOS}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_SHORT.get(args.dtype, args.dtype),
            "data": "synthetic",
            "impl": "native",
            "config": {"workload": workload_name(n, args.n_out, x is None, args.dtype), "n": n, "n_out": args.n_out,
                       "algorithms": list(ALGOS), "x": None if x is None else "int64", "y": args.dtype,
                       "l2": l2_note(n, ysz, xsz),
                       "parallelism": f"{world} independent series (one per GPU)" if world > 1 else "single GPU"},
            "pct_of_hbm_peak": 100.0 * value / world / peak,
            "per_algo": per_algo,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": kernel_traffic(),
                         "kernel": stream_kernel_name(n, args.n_out, args.stream_variant, ysz, x is not None),
                         "bytes_per_launch": n * ysz, "launches_timed": kern_launches,
                         "peak_source": f"{peak_src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                         "read_peak": None if rpeak is None else {
                             "value": rpeak, "frac": achieved / rpeak,
                             "source": "tsds_read_stream over the resident y (each byte read once, "
                                       "16-byte loads), median of 10 launches, same call"}},
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "gpu_launches": launches,
            "selected": counts,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
