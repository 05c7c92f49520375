"""Fused value gather: the *_values entry points return the oracle's indices
and, beside them, the raw x and y elements at those indices (compared as
bytes, so NaN payloads, -0 and every dtype count).  Cases reach every kernel
that writes indices: the small one-launch path, the windowed streaming pass
with the per-series and the tiled emit, n_out >= n, the LTTB table and hull
modes, and MinMaxLTTB with and without a full preselection."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2307_05389_gb300 import binding, inputs

from gpu_util import DevArray

pytestmark = pytest.mark.gpu

FNS = {"minmax": binding.tsds_minmax_values, "m4": binding.tsds_m4_values, "lttb": binding.tsds_lttb_values,
       "everynth": binding.tsds_everynth_values}


def call_values(algo, x, y, n_out, nan="propagate", ratio=4, want_x=True):
    import torch
    yd = DevArray(y)
    xd = DevArray(x) if x is not None else None
    n = len(y)
    cap = max(n if n_out >= n else n_out, 1)
    out = torch.full((cap,), -7, dtype=torch.int64, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    yo = torch.zeros(cap * y.dtype.itemsize + 8, dtype=torch.uint8, device="cuda")
    xo = torch.zeros(cap * x.dtype.itemsize + 8, dtype=torch.uint8, device="cuda") if x is not None and want_x else None
    st = torch.cuda.current_stream()
    sp = ctypes.c_void_p(st.cuda_stream)
    common = (xd.ptr if xd else None, binding.DTYPES[xd.dtype] if xd else 0, yd.ptr, binding.DTYPES[yd.dtype], n,
              n_out)
    tail = (out.data_ptr(), cnt.data_ptr(), xo.data_ptr() if xo is not None else None, yo.data_ptr(), sp)
    nm = binding.NAN_MODES[nan]
    if algo == "minmaxlttb":
        r = binding.tsds_minmaxlttb_values(*common, ratio, nm, *tail)
    else:
        r = FNS[algo](*common, nm, *tail)
    assert r == 0, binding.last_error()
    st.synchronize()
    k = int(cnt.item())
    idx = out.cpu().numpy()[:k]
    yv = yo.cpu().numpy()[:k * y.dtype.itemsize].view(y.dtype)
    xv = xo.cpu().numpy()[:k * x.dtype.itemsize].view(x.dtype) if xo is not None else None
    return idx, xv, yv


def check(algo, x, y, n_out, nan="propagate", ratio=4, want_x=True):
    idx, xv, yv = call_values(algo, x, y, n_out, nan, ratio, want_x)
    exp = oracle.downsample(algo, x, y, n_out, nan=nan, minmax_ratio=ratio)
    np.testing.assert_array_equal(idx, exp)
    assert yv.tobytes() == np.ascontiguousarray(y[exp]).tobytes(), f"{algo} y values"
    if x is not None and want_x:
        assert xv.tobytes() == np.ascontiguousarray(x[exp]).tobytes(), f"{algo} x values"


@pytest.mark.parametrize("dtype", ["int8", "uint16", "float16", "int32", "float32", "float64", "uint64"])
@pytest.mark.parametrize("algo", ["minmax", "m4"])
def test_binned_values_every_path(dtype, algo):
    big = 2_000_003
    y_small = inputs.ties_and_specials(30_011, dtype, 1) if np.dtype(dtype).kind == "f" else \
        inputs.quarter_range(30_011, dtype, 1)
    y_big = inputs.random_walk(big, dtype, 2) if np.dtype(dtype).kind == "f" else inputs.quarter_range(big, dtype, 2)
    check(algo, None, y_small, 400)                      # one-launch small path
    check(algo, None, y_big, 2000)                       # windowed pass, per-series emit
    check(algo, None, y_big, 80_000)                     # tiled emit (>= 4096 bins)
    check(algo, None, y_small[:300], 400)                # n_out >= n
    if np.dtype(dtype).kind == "f":
        check(algo, None, y_small, 400, nan="ignore")


@pytest.mark.parametrize("x_dtype", ["int64", "float64", "uint32", "float16"])
def test_binned_values_with_x(x_dtype):
    n = 500_009
    y = inputs.random_walk(n, "float32", 3)
    if x_dtype == "float16":
        x = np.sort(np.random.default_rng(3).uniform(0, 60000, n)).astype(np.float16)
    elif x_dtype == "float64":
        x = inputs.exponential_x(n, 3)
    else:
        x = inputs.geometric_x(n, 3).astype(x_dtype)
    for algo in ("minmax", "m4"):
        check(algo, x, y, 2000)
        check(algo, x, y, 2000, want_x=False)            # y values only
    check("minmax", x[:1000], y[:1000], 40)               # small path with x


@pytest.mark.parametrize("dtype", ["float32", "float64", "int16"])
def test_lttb_values(dtype):
    y = inputs.random_walk(200_003, dtype, 4) if np.dtype(dtype).kind == "f" else inputs.quarter_range(200_003, dtype, 4)
    check("lttb", None, y, 1000)                         # hull mode (about 200 points per bucket)
    check("lttb", None, y, 20_000)                       # table mode (10 per bucket)
    check("lttb", None, y[:500], 800)                    # n_out >= n
    x = inputs.geometric_x(len(y), 4)
    check("lttb", x, y, 1000)


def test_minmaxlttb_values():
    n = 1_000_003
    y = inputs.quantised_nan(n, 5)
    x = inputs.exponential_x(n, 5)
    for nan in ("propagate", "ignore"):
        check("minmaxlttb", None, y, 1000, nan=nan, ratio=4)
        check("minmaxlttb", x, y, 1000, nan=nan, ratio=30)
    check("minmaxlttb", None, y[:3000], 1000, ratio=4)    # the preselection keeps every point


def test_downsample_values_helper():
    import torch
    y = torch.from_numpy(inputs.random_walk(100_000, "float32", 6)).cuda()
    x = torch.from_numpy(inputs.geometric_x(100_000, 6)).cuda()
    idx, xv, yv = binding.downsample_values("m4", y, 400, x=x)
    assert torch.equal(yv, y[idx]) and torch.equal(xv, x[idx])
    idx, xv, yv = binding.downsample_values("minmaxlttb", y, 400)
    assert xv is None and torch.equal(yv, y[idx])


@pytest.mark.parametrize("dtype", ["uint8", "float16", "float64"])
def test_everynth_values(dtype):
    n = 400_003
    y = inputs.random_walk(n, dtype, 8) if np.dtype(dtype).kind == "f" else inputs.quarter_range(n, dtype, 8)
    x = inputs.exponential_x(n, 8)
    for n_out in (1000, 30_000):
        check("everynth", None, y, n_out)
        check("everynth", x, y, n_out)
    check("everynth", x[:100], y[:100], 100)


def test_downsample_host_pinned_x_read_in_place():
    """downsample_host with page-locked host buffers: y is copied, a pinned x
    is searched in place; the indices equal the oracle's."""
    import torch
    n = 400_003
    y = inputs.random_walk(n, "float32", 9)
    x = inputs.geometric_x(n, 9)
    yh = torch.from_numpy(y).pin_memory()
    xh = torch.from_numpy(x).pin_memory()
    res = binding.downsample_host(["minmax", "m4", "everynth"], yh, 2000, x=xh)
    for algo, got in zip(["minmax", "m4", "everynth"], res):
        np.testing.assert_array_equal(got.numpy(), oracle.downsample(algo, x, y, 2000))
    res = binding.downsample_host(["minmaxlttb", "lttb"], yh, 2000, x=xh)   # x copied for the LTTB family
    for algo, got in zip(["minmaxlttb", "lttb"], res):
        np.testing.assert_array_equal(got.numpy(), oracle.downsample(algo, x, y, 2000))
