"""tsds_downsample_host (through binding.downsample_host): y in host memory, copied in
chunks that overlap the reduction of the bins already on the device, indices back in host
memory.  Every result against the oracle on the same bytes (Section 2.3's
downsample([x], y, n_out) semantics), over several chunks, with and without x, both NaN
modes, pinned and pageable y, x in page-locked host memory and on the device, and an n_out
that covers every index."""
import numpy as np
import pytest

import oracle
import paper_2307_05389_gb300 as pkg
from paper_2307_05389_gb300 import inputs

pytestmark = pytest.mark.gpu


def _check(algos, yh, n_out, x=None, nan="propagate", y_dev=None):
    import torch
    got = pkg.downsample_host(algos, yh, n_out, x=x, nan=nan, y_dev=y_dev)
    xn = x.cpu().numpy() if x is not None else None
    yn = yh.numpy()
    for algo, g in zip(algos, got):
        want = oracle.downsample(algo, xn, yn, n_out, nan)
        g = g.numpy()
        assert len(g) == len(want), f"{algo} n_out={n_out}: {len(g)} indices, oracle {len(want)}"
        bad = np.flatnonzero(g != want)
        assert bad.size == 0, f"{algo} n_out={n_out}: first difference at output {bad[:1]}"
    torch.cuda.synchronize()


@pytest.mark.parametrize("n_out", [2000, 40_000, 400_000])
@pytest.mark.parametrize("with_x", [False, True])
def test_chunks_overlap_and_match_the_oracle(n_out, with_x):
    """12.5e6 float32 points (50 MB: four chunks of 16 MB or less), pinned y and pinned int64
    x, MinMax and M4 in one call, bins of 500 B to 100 KB."""
    import torch
    n = 12_500_000
    yh = torch.from_numpy(inputs.random_walk(n, "float32", seed=11)).pin_memory()
    x = torch.from_numpy(inputs.geometric_x(n, seed=12)).pin_memory() if with_x else None
    _check(("minmax", "m4"), yh, n_out, x=x)


def test_pageable_y_device_x_float64_nan_ignore():
    """Pageable y with 1 % NaN, float64 x on the device, NaN-ignore and NaN-propagate, a
    caller-supplied y_dev (which holds y afterwards)."""
    import torch
    n = 6_000_001
    y = inputs.random_walk(n, "float32", seed=13)
    rng = np.random.default_rng(14)
    y[rng.random(n) < 0.01] = np.nan
    yh = torch.from_numpy(y)
    x = torch.from_numpy(inputs.exponential_x(n, seed=15)).cuda()
    y_dev = torch.empty(n, dtype=torch.float32, device="cuda")
    for nan in ("ignore", "propagate"):
        _check(("m4", "minmax"), yh, 8000, x=x, nan=nan, y_dev=y_dev)
    assert torch.equal(y_dev.cpu().view(torch.int32), yh.view(torch.int32))   # bit for bit (NaN != NaN)


@pytest.mark.parametrize("dtype", ["uint16", "int64", "float64", "int8"])
def test_other_dtypes(dtype):
    import torch
    n = 3_000_003
    yn = inputs.quarter_range(n, dtype, seed=16)
    yh = torch.from_numpy(yn)
    got = pkg.downsample_host(("minmax", "m4"), yh, 4000)
    for algo, g in zip(("minmax", "m4"), got):
        want = oracle.downsample(algo, None, yn, 4000)
        assert np.array_equal(g.numpy(), want), (dtype, algo)


def test_every_index_and_small_series():
    """n_out >= n returns every index; a series smaller than one chunk."""
    import torch
    n = 1001
    yh = torch.from_numpy(inputs.random_walk(n, "float32", seed=17)).pin_memory()
    got = pkg.downsample_host(("minmax", "m4"), yh, 2000)
    for g in got:
        assert np.array_equal(g.numpy(), np.arange(n))
    _check(("minmax", "m4"), yh, 100)
    _check(("m4",), yh, 8)


def test_pageable_x_is_refused():
    import torch
    n = 100_000
    yh = torch.from_numpy(inputs.random_walk(n, "float32", seed=18))
    x = torch.from_numpy(inputs.geometric_x(n, seed=19))
    from paper_2307_05389_gb300 import binding
    import ctypes
    codes = (ctypes.c_int * 1)(0)
    n_outs = (ctypes.c_int64 * 1)(1000)
    out = torch.empty(1000, dtype=torch.int64)
    ptrs = (ctypes.c_void_p * 1)(out.data_ptr())
    counts = (ctypes.c_int64 * 1)()
    r = binding.tsds_downsample_host(1, codes, n_outs, x.data_ptr(), binding.DTYPES["int64"], yh.data_ptr(),
                                     binding.DTYPES["float32"], n, 0, None, ptrs, counts, None)
    assert r == 1 and "page-locked" in pkg.last_error()
