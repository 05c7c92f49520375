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
