"""Parity at the benchmark's full sizes, in the launch configurations bench.py
times, on outputs the oracle computes one by one.

* The headline workload (10^9 float32 random walk, int64 geometric x, n_out =
  2000, MinMax and M4) and the per-dtype workloads (4 GB of y each, all eleven
  dtypes): whole outputs against the oracle on host copies of the same bytes.
* The served workload's shape (resident 10^8-point float32 series with float64
  x, viewport queries spanning 10^6 to 10^8 points, every served algorithm,
  both NaN modes): every query's whole result against the oracle on its range.
* The batched workload (4096 series, 17.7 GB, a resident autotuned plan with a
  CUDA graph): sampled series against the oracle, whole outputs.
* Plain LTTB on 10^7 points and MinMaxLTTB on the 64 quantised NaN series of
  1.5625e6 points, one call per series and one batched call for all 64: whole
  outputs against the oracle.

Inputs are generated exactly as bench.py generates them (same seeds)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2307_05389_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

N_OUT = 2000


def _host(t, dtype):
    """Device tensor -> numpy array of `dtype` (unsigned dtypes are stored signed on the device)."""
    return t.cpu().numpy().view(np.dtype(dtype))


def _raw(algo, x, y, y_dtype, n, n_out, nan="propagate", x_dtype="int64"):
    import torch
    out = torch.full((n_out + 8,), -7, dtype=torch.int64, device=y.device)
    cnt = torch.full((1,), -1, dtype=torch.int64, device=y.device)
    st = torch.cuda.current_stream(y.device)
    fn = {"minmax": binding.tsds_minmax, "m4": binding.tsds_m4}[algo]
    r = fn(x.data_ptr() if x is not None else None, binding.DTYPES[x_dtype] if x is not None else 0,
           y.data_ptr(), binding.DTYPES[y_dtype], n, n_out, binding.NAN_MODES[nan], out.data_ptr(),
           cnt.data_ptr(), ctypes.c_void_p(st.cuda_stream))
    assert r == 0, binding.last_error()
    torch.cuda.synchronize()
    k = int(cnt.item())
    res = out.cpu().numpy()
    assert 0 < k <= n_out and np.all(res[k:] == -7)
    return res[:k]


def _whole_outputs_match(x, y, y_dtype, n, seed_note):
    """MinMax and M4 at n_out = 2000 on the device, then the oracle on host copies of
    the same bytes (its bins split over host threads, each part the single-threaded
    oracle), compared index for index."""
    import torch
    got = {algo: _raw(algo, x, y, y_dtype, n, N_OUT) for algo in ("minmax", "m4")}
    yh = _host(y, y_dtype)
    xh = _host(x, "int64")
    for algo, g in got.items():
        want = oracle.binned_threads(algo, xh, yh, N_OUT)
        assert len(want) == len(g), f"{algo} {seed_note}: {len(g)} indices, oracle {len(want)}"
        bad = np.flatnonzero(g != want)
        assert bad.size == 0, f"{algo} {seed_note}: first difference at output {bad[:1]}"
    del yh, xh
    torch.cuda.empty_cache()


def test_headline_workload_whole_output():
    """10^9 float32 random walk (seed 2), int64 geometric x (seed 2), n_out = 2000: every
    index of both outputs."""
    import torch
    n = 10 ** 9
    y = inputs.random_walk_cuda(n, "float32", seed=2)
    x = inputs.geometric_x_cuda(n, seed=2)
    torch.cuda.synchronize()
    _whole_outputs_match(x, y, "float32", n, "1e9 float32 random walk")
    del x, y
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", inputs.DTYPES)
def test_dtype_workloads_whole_output(dtype):
    """4 GB of quarter-range y per dtype (seed 2; float32 here is the uniform case) with int64
    geometric x (seed 2), n_out = 2000: every index of both outputs."""
    import torch
    n = 4_000_000_000 // np.dtype(dtype).itemsize
    y = inputs.quarter_range_cuda(n, dtype, seed=2)
    x = inputs.geometric_x_cuda(n, seed=2)
    torch.cuda.synchronize()
    _whole_outputs_match(x, y, dtype, n, f"4 GB {dtype}")
    del x, y
    torch.cuda.empty_cache()


@pytest.mark.parametrize("bin_bytes", [1024, 16384, 49152, 131072])
@pytest.mark.parametrize("with_x", [False, True])
def test_automatic_choice_beyond_256mb_whole_output(bin_bytes, with_x):
    """1 GB of float32 random walk (seed 2), index bins or x-space bins over int64 geometric x:
    beyond 256 MB the automatic choice runs lane groups below 64 KB mean bins and register
    streaming above; every index of both outputs at bins of 1, 16, 48 and 128 KB."""
    import torch
    n = 250_000_000
    y = inputs.random_walk_cuda(n, "float32", seed=2)
    x = inputs.geometric_x_cuda(n, seed=2) if with_x else None
    torch.cuda.synchronize()
    yh = _host(y, "float32")
    xh = _host(x, "int64") if with_x else None
    for algo, per in (("minmax", 2), ("m4", 4)):
        n_out = per * (n * 4 // bin_bytes)
        g = _raw(algo, x, y, "float32", n, n_out)
        want = oracle.binned_threads(algo, xh, yh, n_out)
        assert len(want) == len(g), f"{algo} {bin_bytes} B bins: {len(g)} indices, oracle {len(want)}"
        bad = np.flatnonzero(g != want)
        assert bad.size == 0, f"{algo} {bin_bytes} B bins: first difference at output {bad[:1]}"
    del x, y, xh, yh
    torch.cuda.empty_cache()


def test_batched_workload_sampled_series():
    """4096 float32 series, lengths round(10**U(3,7)) and n_out in [200, 4000] (seed 3), as a
    resident autotuned plan with a CUDA graph, MinMax and M4."""
    import torch
    count = 4096
    lens = inputs.batch_lengths(count, seed=3)
    n_outs = inputs.batch_n_out(count, seed=3)
    walk = inputs.random_walk_cuda(int(lens.sum()), "float32", seed=3)
    offs = np.concatenate([[0], np.cumsum(lens)])
    ys = [walk[int(offs[i]):int(offs[i + 1])] for i in range(count)]
    rng = np.random.default_rng(13)
    pick = sorted({int(np.argmax(lens)), int(np.argmin(lens)), *rng.choice(count, 22, replace=False).tolist()})
    for algo in ("minmax", "m4"):
        plan = binding.Plan(algo, ys, n_outs, graph=True, autotune=True)
        try:
            outs, counts = plan.execute()
            torch.cuda.synchronize()
            c = counts.cpu().numpy()
            for i in pick:
                want = oracle.downsample(algo, None, _host(ys[i], "float32"), int(n_outs[i]))
                got = outs[i][:int(c[i])].cpu().numpy()
                assert np.array_equal(got, want), f"{algo} series {i} (n={lens[i]}, n_out={n_outs[i]})"
        finally:
            plan.close()
    del ys, walk
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_plain_lttb_1e7(dtype):
    """LTTB on a 10^7-point random walk (seed 4), n_out = 4000: the whole output."""
    import torch
    y = inputs.random_walk(10_000_000, dtype, seed=4)
    got = binding.downsample("lttb", torch.from_numpy(y).cuda(), 4000).cpu().numpy()
    assert np.array_equal(got, oracle.lttb(None, y, 4000))


@pytest.mark.parametrize("nan", ["propagate", "ignore"])
def test_minmaxlttb_quantised_nan_series(nan):
    """MinMaxLTTB on the 64 quantised series with 1 % NaN (seeds 4..67), n_out = 4000,
    ratios 2, 4 and 30: eight sampled series, whole outputs."""
    import torch
    rng = np.random.default_rng(14)
    for i in sorted(rng.choice(64, 8, replace=False).tolist()):
        y = inputs.quantised_nan(1_562_500, seed=4 + i)
        dy = torch.from_numpy(y).cuda()
        for r in (2, 4, 30):
            got = binding.downsample("minmaxlttb", dy, 4000, nan=nan, minmax_ratio=r).cpu().numpy()
            want = oracle.minmaxlttb(None, y, 4000, r, nan)
            assert np.array_equal(got, want), f"series {i} ratio {r}"


@pytest.mark.parametrize("nan", ["propagate", "ignore"])
def test_batched_minmaxlttb_quantised_nan_series(nan):
    """The same 64 series as one tsds_batched_minmaxlttb call per ratio: eight sampled
    series against the oracle, whole outputs."""
    import torch
    series = [inputs.quantised_nan(1_562_500, seed=4 + i) for i in range(64)]
    dev = [torch.from_numpy(y).cuda() for y in series]
    rng = np.random.default_rng(15)
    pick = sorted(rng.choice(64, 8, replace=False).tolist())
    for r in (2, 4, 30):
        outs, counts = binding.downsample_batched("minmaxlttb", dev, [4000] * 64, nan=nan, minmax_ratio=r)
        torch.cuda.synchronize()
        c = counts.cpu().numpy()
        for i in pick:
            want = oracle.minmaxlttb(None, series[i], 4000, r, nan)
            assert np.array_equal(outs[i][:int(c[i])].cpu().numpy(), want), f"series {i} ratio {r}"


def test_served_workload_resident_1e8_series():
    """The served workload's shape: four resident 10^8-point float32 random walks (the
    serving benchmark's first four, seeds 500..503) with float64 x = cumsum(exponential(1))
    (seeds 600..603), one of them with 1 % of its points set to NaN so that the two NaN modes
    differ.  48 viewport queries spanning 10^6 to 10^8 points (log-uniform; 36 as x ranges,
    12 as index ranges), n_out in {500, 1000, 2000, 4000}, MinMax / M4 / MinMaxLTTB(4), both
    NaN modes, all submitted at once to a server shaped like the benchmark's (4 streams,
    batches of up to 256, 8 GiB budget).  Each whole result must equal the oracle on the range
    its query selects, shifted to the whole series."""
    import concurrent.futures as cf

    import torch
    nser, n = 4, 100_000_000
    ys = [inputs.random_walk_cuda(n, "float32", seed=500 + i) for i in range(nser)]
    xs = [inputs.exponential_x_cuda(n, seed=600 + i) for i in range(nser)]
    torch.cuda.synchronize()
    yh = [_host(y, "float32") for y in ys]
    xh = [_host(x, "float64") for x in xs]
    rng = np.random.default_rng(16)
    nan_at = rng.choice(n, size=n // 100, replace=False)
    yh[3] = yh[3].copy()
    yh[3][nan_at] = np.nan
    ys[3].copy_(torch.from_numpy(yh[3]))
    srv = binding.Server("float32", "float64", streams=4, max_batch=256, memory_budget=8 << 30)
    try:
        ids = [srv.add_series(y, x) for y, x in zip(ys, xs)]
        qs = []
        for k in range(48):
            s = int(rng.integers(0, nser))
            span = int(10 ** rng.uniform(6, 8))
            start = int(rng.integers(0, n - span + 1))
            q = dict(sid=s, algo=("minmax", "m4", "minmaxlttb")[k % 3], n_out=int(rng.choice([500, 1000, 2000, 4000])),
                     nan=("propagate", "ignore")[(k // 3) % 2])
            if k % 4 == 3:
                q["index_range"] = (start, start + span)
            else:
                q["x_range"] = (float(xh[s][start]), float(xh[s][start + span - 1]))
            qs.append(q)
        tickets = [srv.submit(ids[q["sid"]], q["algo"], q["n_out"], x_range=q.get("x_range"),
                              index_range=q.get("index_range"), nan=q["nan"]) for q in qs]
        got = [srv.result(t)[0] for t in tickets]
    finally:
        srv.close()

    def want(q):
        x, y = xh[q["sid"]], yh[q["sid"]]
        if "x_range" in q:
            lo = int(np.searchsorted(x, q["x_range"][0], "left"))
            hi = int(np.searchsorted(x, q["x_range"][1], "right"))
        else:
            lo, hi = q["index_range"]
        return oracle.downsample(q["algo"], x[lo:hi], y[lo:hi], q["n_out"], nan=q["nan"], minmax_ratio=4) + lo

    with cf.ThreadPoolExecutor(16) as ex:
        wants = list(ex.map(want, qs))
    for q, g, w in zip(qs, got, wants):
        assert np.array_equal(g, w), f"query {q}: {len(g)} indices, oracle {len(w)}"
    del ys, xs
    torch.cuda.empty_cache()
