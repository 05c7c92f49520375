"""tsds_minmax_noalloc: MinMax for callers that cannot allocate device memory
while the call runs (their memory is owned by another allocator, or they sit
in a latency-bound redraw loop where an allocation could stall the device).
Its scratch is a fixed array inside the library, shared by every call.

These GPU tests call it through the C ABI and compare it with tsds_minmax
index for index, twice in a row (so the second call runs on the array the
first one left behind), and check that a call too large for the array is
refused before any device work.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2307_05389_gb300 import binding, inputs

from gpu_util import DevArray

pytestmark = pytest.mark.gpu


def _run(fn, x, y, n_out, nan="propagate"):
    import torch
    yd = DevArray(y)
    xd = DevArray(x) if x is not None else None
    out = torch.full((max(len(y), n_out, 1),), -7, dtype=torch.int64, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream()
    r = fn(xd.ptr if xd else None, binding.DTYPES[xd.dtype] if xd else 0, yd.ptr, binding.DTYPES[yd.dtype],
           len(y), n_out, binding.NAN_MODES[nan], out.data_ptr(), cnt.data_ptr(), ctypes.c_void_p(st.cuda_stream))
    assert r == 0, binding.last_error()
    st.synchronize()
    k = int(cnt.item())
    return out[:k].cpu().numpy()


CASES = [
    # (y, x, n_out, nan): two different series so the second call sees leftovers of the first
    (lambda: inputs.random_walk(3_000_003, "float32", seed=41), None, 2000, "propagate"),
    (lambda: inputs.quarter_range(1_000_001, "int16", seed=42), None, 500, "propagate"),
    (lambda: inputs.random_walk(400_000, "float64", seed=43), lambda: inputs.geometric_x(400_000, seed=44), 4000, "ignore"),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_noalloc_matches_tsds_minmax_on_two_calls_in_a_row(case):
    make_y, make_x, n_out, nan = CASES[case]
    y = make_y()
    x = make_x() if make_x else None
    ref = _run(binding.tsds_minmax, x, y, n_out, nan)
    first = _run(binding.tsds_minmax_noalloc, x, y, n_out, nan)
    second = _run(binding.tsds_minmax_noalloc, x, y, n_out, nan)
    np.testing.assert_array_equal(first, ref)
    np.testing.assert_array_equal(second, ref)


def test_noalloc_back_to_back_different_inputs():
    a = inputs.random_walk(2_000_000, "float32", seed=45)
    b = inputs.random_walk(777_777, "float32", seed=46)
    ra, rb = _run(binding.tsds_minmax, None, a, 1000), _run(binding.tsds_minmax, None, b, 3000)
    np.testing.assert_array_equal(_run(binding.tsds_minmax_noalloc, None, a, 1000), ra)
    np.testing.assert_array_equal(_run(binding.tsds_minmax_noalloc, None, b, 3000), rb)


@pytest.mark.parametrize("case", ["segmented", "two_level_int64_x", "two_level_float64_x"])
def test_noalloc_paths_with_many_bins(case):
    """Calls with many bins, twice in a row against tsds_minmax: sub-KB float32 bins (the
    segmented streaming kernel), and 8192 x-space bins of about 244 points (the two-level bin
    search; tsds_minmax emits them with its tiled emit, this call with one CTA)."""
    if case == "segmented":
        y, x, n_out = inputs.random_walk(4_000_000, "float32", seed=47), None, 40_000
    elif case == "two_level_int64_x":
        y, x, n_out = inputs.random_walk(2_000_000, "float32", seed=48), inputs.geometric_x(2_000_000, seed=49), 2 * 8192
    else:
        y, x, n_out = inputs.random_walk(2_000_000, "float32", seed=50), inputs.exponential_x(2_000_000, seed=51), 2 * 8192
    ref = _run(binding.tsds_minmax, x, y, n_out)
    np.testing.assert_array_equal(_run(binding.tsds_minmax_noalloc, x, y, n_out), ref)
    np.testing.assert_array_equal(_run(binding.tsds_minmax_noalloc, x, y, n_out), ref)


def test_noalloc_every_index_and_empty_input():
    """n_out >= n returns every index; n == 0 returns a count of 0."""
    y = inputs.random_walk(5000, "float32", seed=52)
    np.testing.assert_array_equal(_run(binding.tsds_minmax_noalloc, None, y, 6000), _run(binding.tsds_minmax, None, y, 6000))
    np.testing.assert_array_equal(_run(binding.tsds_minmax_noalloc, None, y, 5000), np.arange(5000))
    assert _run(binding.tsds_minmax_noalloc, None, y[:0], 10).size == 0


def _scratch_bytes(nb, windows):
    """The static-scratch layout of one call: edges, results, counters, work counter,
    two piece slots per window, each part rounded up to 256 bytes."""
    up = lambda v: (v + 255) // 256 * 256
    o = up((nb + 1) * 8)
    o = up(o + nb * 16)
    o = up(o + nb * 4)
    o = up(o + 64)
    o = up(o + windows * 32)
    return up(o + windows * 32)


def test_noalloc_largest_accepted_call():
    """At n_out = 2000, the largest float32 series whose scratch fits the 8 MiB array is
    accepted and matches tsds_minmax (twice); one more 64 KB window of y is refused."""
    import torch
    welems = 65536 // 4
    windows = 1
    while _scratch_bytes(1000, windows + 1) <= 8 << 20:
        windows += 1
    n = windows * welems
    y = inputs.random_walk_cuda(n, "float32", seed=53)
    out = torch.full((2008,), -7, dtype=torch.int64, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream()
    sp = ctypes.c_void_p(st.cuda_stream)

    def call(fn, n_):
        return fn(None, 0, y.data_ptr(), binding.DTYPES["float32"], n_, 2000, 0, out.data_ptr(), cnt.data_ptr(), sp)

    r = call(binding.tsds_minmax_noalloc, n + 1)   # refused on the host: y is not read
    assert r == 1 and "static scratch" in binding.last_error()
    outs = []
    for fn in (binding.tsds_minmax, binding.tsds_minmax_noalloc, binding.tsds_minmax_noalloc):
        out.fill_(-7)
        assert call(fn, n) == 0, binding.last_error()
        st.synchronize()
        k = int(cnt.item())
        assert 0 < k <= 2000
        outs.append(out[:k].cpu().numpy())
    np.testing.assert_array_equal(outs[1], outs[0])
    np.testing.assert_array_equal(outs[2], outs[0])
    del y
    torch.cuda.empty_cache()


def test_noalloc_refuses_calls_larger_than_its_array():
    # 2e6 bins need 56 MB of scratch: refused on the host with the sizes in the message
    import torch
    y = torch.zeros(8_000_000, dtype=torch.float32, device="cuda")
    out = torch.empty(4_000_000, dtype=torch.int64, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    r = binding.tsds_minmax_noalloc(None, 0, y.data_ptr(), binding.DTYPES["float32"], 8_000_000, 4_000_000, 0,
                                    out.data_ptr(), cnt.data_ptr(), None)
    assert r == 1
    assert "static scratch" in binding.last_error()
    torch.cuda.synchronize()
    assert int(cnt.item()) == -1
