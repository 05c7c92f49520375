"""Parity at the benchmark's full sizes, in the launch configurations bench.py
times, on outputs the oracle computes one by one.

* The headline workload (10^9 float32 random walk, int64 geometric x, n_out =
  2000, MinMax and M4) and the per-dtype workloads (4 GB of y each): sampled
  bins.  The oracle places each sampled bin (its own bin rule, Section 2.3,
  evaluated on x_0, x_{n-1} and a window of x around the bin start, the window
  checked to contain the answer) and takes its argmin/argmax (Section 2.1);
  the GPU's indices inside that bin must be exactly the oracle's.  The whole
  output must be strictly increasing, in range and at most n_out long.
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
WINDOW = 1 << 20          # x elements on each side of a sampled bin start


def _host(t, dtype):
    """Device tensor -> numpy array of `dtype` (unsigned dtypes are stored signed on the device)."""
    return t.cpu().numpy().view(np.dtype(dtype))


def _raw(algo, x, y, y_dtype, n, n_out, nan="propagate"):
    import torch
    out = torch.full((n_out + 8,), -7, dtype=torch.int64, device=y.device)
    cnt = torch.full((1,), -1, dtype=torch.int64, device=y.device)
    st = torch.cuda.current_stream(y.device)
    fn = {"minmax": binding.tsds_minmax, "m4": binding.tsds_m4}[algo]
    r = fn(x.data_ptr() if x is not None else None, binding.DTYPES["int64"] if x is not None else 0,
           y.data_ptr(), binding.DTYPES[y_dtype], n, n_out, binding.NAN_MODES[nan], out.data_ptr(),
           cnt.data_ptr(), ctypes.c_void_p(st.cuda_stream))
    assert r == 0, binding.last_error()
    torch.cuda.synchronize()
    k = int(cnt.item())
    res = out.cpu().numpy()
    assert 0 < k <= n_out and np.all(res[k:] == -7)
    return res[:k]


def _bin_start(x_dev, n, nb, i):
    """Start of bin i by the oracle's bin rule, from x_0, x_{n-1} and a window of x."""
    if i == 0:
        return 0
    if i == nb:
        return n
    c = int(round(i * n / nb))
    a, b = max(1, c - WINDOW), min(n - 1, c + WINDOW)
    sub = np.concatenate([_host(x_dev[:1], "int64"), _host(x_dev[a:b], "int64"), _host(x_dev[n - 1:], "int64")])
    p = int(oracle.bin_edges(sub, len(sub), nb)[i])
    # the answer lies strictly inside the window: x[a] is below the edge and some
    # element of the window reaches it, so the global first index is a + p - 1
    assert 1 < p <= b - a, f"bin {i}: edge outside the sampled window"
    return a + p - 1


def _check_sampled_bins(algo, out, x_dev, y_dev, y_dtype, n, n_out, bins, nan="propagate"):
    nb = n_out // (2 if algo == "minmax" else 4)
    assert np.all(np.diff(out) > 0) and out[0] >= 0 and out[-1] < n
    for i in bins:
        if x_dev is None:
            e = oracle.bin_edges(None, n, nb)
            lo, hi = int(e[i]), int(e[i + 1])
        else:
            lo, hi = _bin_start(x_dev, n, nb, i), _bin_start(x_dev, n, nb, i + 1)
        got = out[(out >= lo) & (out < hi)]
        if hi == lo:
            assert got.size == 0
            continue
        a, b = oracle.argminmax(_host(y_dev[lo:hi], y_dtype), 0, hi - lo, nan)
        want = {lo + a, lo + b}
        if algo == "m4":
            want |= {lo, hi - 1}
        assert list(got) == sorted(want), f"{algo} bin {i} [{lo}, {hi})"


def _sample(nb, seed, k=14):
    rng = np.random.default_rng(seed)
    return sorted({0, nb - 1, *rng.choice(nb, size=k, replace=False).tolist()})


def test_headline_workload_sampled_bins():
    """10^9 float32 random walk (seed 2), int64 geometric x (seed 2), n_out = 2000."""
    import torch
    n = 10 ** 9
    y = inputs.random_walk_cuda(n, "float32", seed=2)
    x = inputs.geometric_x_cuda(n, seed=2)
    torch.cuda.synchronize()
    for algo in ("minmax", "m4"):
        out = _raw(algo, x, y, "float32", n, N_OUT)
        nb = N_OUT // (2 if algo == "minmax" else 4)
        _check_sampled_bins(algo, out, x, y, "float32", n, N_OUT, _sample(nb, seed=11))
    del x, y
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", ["int8", "uint16", "float16", "float64"])
def test_dtype_workloads_sampled_bins(dtype):
    """4 GB of quarter-range y per dtype (seed 2) with int64 geometric x (seed 2)."""
    import torch
    n = 4_000_000_000 // np.dtype(dtype).itemsize
    y = inputs.quarter_range_cuda(n, dtype, seed=2)
    x = inputs.geometric_x_cuda(n, seed=2)
    torch.cuda.synchronize()
    for algo in ("minmax", "m4"):
        out = _raw(algo, x, y, dtype, n, N_OUT)
        nb = N_OUT // (2 if algo == "minmax" else 4)
        _check_sampled_bins(algo, out, x, y, dtype, n, N_OUT, _sample(nb, seed=12, k=6))
    del x, y
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
