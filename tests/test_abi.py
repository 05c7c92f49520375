"""The C ABI library loads and exports every entry point include/tsds.h
declares; host-side argument checks answer without a GPU (CPU only)."""
import ctypes
import os
import re

import pytest

import paper_2307_05389_gb300 as pkg
from paper_2307_05389_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(tsds_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    return pkg.load()


def test_header_declares_the_core_entry_points():
    names = declared_functions()
    for n in ("tsds_minmax", "tsds_m4", "tsds_lttb", "tsds_minmaxlttb", "tsds_last_error", "tsds_shutdown"):
        assert n in names


@pytest.mark.parametrize("name", declared_functions())
def test_symbol_exported(lib, name):
    assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_names_match_abi():
    for n in ("tsds_minmax", "tsds_m4", "tsds_lttb", "tsds_minmaxlttb", "tsds_shutdown", "tsds_version"):
        assert callable(getattr(pkg, n))


def test_version(lib):
    assert re.match(r"^\d+\.\d+\.\d+$", pkg.tsds_version())


def _call(fn, n, n_out, y=1 << 20, out=1 << 21, cnt=1 << 22, x=None, x_dtype=0, y_dtype=9, nan=0):
    return fn(x, x_dtype, y, y_dtype, n, n_out, nan, out, cnt, None)


@pytest.mark.parametrize("fn,n_out", [(binding.tsds_minmax, 3), (binding.tsds_minmax, 0), (binding.tsds_m4, 6),
                                      (binding.tsds_m4, 2), (binding.tsds_lttb, 2)])
def test_invalid_n_out_is_rejected_on_the_host(lib, fn, n_out):
    assert _call(fn, 100, n_out) == 1
    assert "n_out" in pkg.last_error()


def test_other_invalid_arguments(lib):
    assert _call(binding.tsds_minmax, -1, 10) == 1                   # n < 0
    assert _call(binding.tsds_minmax, 10, 10, y=None) == 1           # y NULL
    assert _call(binding.tsds_minmax, 10, 10, y_dtype=11) == 1       # unknown dtype
    assert _call(binding.tsds_minmax, 10, 10, x=1 << 20, x_dtype=-1) == 1
    assert _call(binding.tsds_minmax, 10, 10, nan=2) == 1
    assert _call(binding.tsds_minmax, 10, 10, cnt=None) == 1
    assert _call(binding.tsds_minmax, 10, 10, y=(1 << 20) + 2) == 1  # misaligned float32
    assert binding.tsds_minmaxlttb(None, 0, 1 << 20, 9, 100, 10, 0, 0, 1 << 21, 1 << 22, None) == 1
    assert "minmax_ratio" in pkg.last_error()


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError):
        binding_path = str(tmp_path / "nope.so")
        saved = binding._lib
        binding._lib = None
        try:
            binding.load(binding_path)
        finally:
            binding._lib = saved


def test_series_array_matches_the_struct_layout():
    """The batch descriptor array built column-wise has the tsds_series layout
    (six 8-byte fields in header order), without touching device memory."""
    import numpy as np

    class FakeTensor:
        def __init__(self, ptr, n):
            self.ptr, self.shape = ptr, (n,)

        def data_ptr(self):
            return self.ptr

    ys = [FakeTensor(0x1000 * (i + 1), 100 + i) for i in range(3)]
    xs = [FakeTensor(0x9000 + 0x100 * i, 100 + i) for i in range(3)]
    outs = [FakeTensor(0x20000 + 0x40 * i, 8) for i in range(3)]
    counts = FakeTensor(0x30000, 3)
    a = binding._series_array(ys, [8, 12, 16], xs, outs, counts)
    assert a.dtype == np.uint64 and a.shape == (3, 6)
    assert ctypes.sizeof(binding.tsds_series) == a.itemsize * a.shape[1]
    s = binding.tsds_series.from_buffer_copy(a.tobytes(), ctypes.sizeof(binding.tsds_series))
    assert (s.x, s.y, s.n, s.n_out, s.out, s.out_count) == (0x9100, 0x2000, 101, 12, 0x20040, 0x30008)
    a = binding._series_array(ys, [8, 12, 16], None, outs, counts)
    assert (a[:, 0] == 0).all()


def test_value_outputs_are_checked_on_the_host(lib):
    """x_out without x, and value buffers not aligned to their elements, are
    rejected before anything runs."""
    y, out, cnt = 1 << 20, 1 << 21, 1 << 22
    for fn in (binding.tsds_minmax_values, binding.tsds_m4_values, binding.tsds_lttb_values):
        assert fn(None, 0, y, 9, 100, 8, 0, out, cnt, 1 << 23, None, None) == 1      # x_out, no x
        assert "x_out" in pkg.last_error()
        assert fn(None, 0, y, 9, 100, 8, 0, out, cnt, None, (1 << 23) + 2, None) == 1  # float32 y_out
        assert "aligned" in pkg.last_error()
        assert fn(1 << 24, 3, y, 9, 100, 8, 0, out, cnt, (1 << 23) + 4, None, None) == 1  # int64 x_out
    assert binding.tsds_minmaxlttb_values(None, 0, y, 9, 100, 8, 4, 0, out, cnt, 1 << 23, None, None) == 1


def test_read_stream_arguments_are_checked_on_the_host(lib):
    """The read-only streaming probe rejects bad sizes and pointers before any
    launch; zero bytes launch nothing."""
    buf, sink = 1 << 20, 1 << 21
    assert binding.tsds_read_stream(buf, -16, sink, None) == 1
    assert binding.tsds_read_stream(buf, 24, sink, None) == 1           # not a multiple of 16
    assert "multiple of 16" in pkg.last_error()
    assert binding.tsds_read_stream(buf, 32, None, None) == 1           # no sink
    assert binding.tsds_read_stream(buf + 8, 32, sink, None) == 1       # misaligned
    assert binding.tsds_read_stream(None, 32, sink, None) == 1
    assert "aligned" in pkg.last_error()
    before = pkg.tsds_kernel_launches()
    assert binding.tsds_read_stream(None, 0, sink, None) == 0
    assert pkg.tsds_kernel_launches() == before


def test_checked_mode_toggle(lib):
    """tsds_checked sets and reports the mode; negative arguments only query."""
    prev = pkg.tsds_checked(-1)
    try:
        assert pkg.tsds_checked(1) == prev
        assert pkg.tsds_checked(-1) == 1
        assert pkg.tsds_checked(0) == 1
        assert pkg.tsds_checked(-5) == 0
    finally:
        pkg.tsds_checked(prev)


@pytest.mark.parametrize("value,want", [("1", 1), ("yes", 1), ("0", 0), ("", 0)])
def test_checked_mode_from_environment(value, want):
    """TSDS_CHECKED turns the mode on at load for any value but "0" (and empty)."""
    import subprocess
    import sys
    code = ("import paper_2307_05389_gb300 as p; p.load(); print(p.tsds_checked(-1))")
    env = dict(os.environ, TSDS_CHECKED=value)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120,
                       cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    assert r.returncode == 0, r.stderr
    assert int(r.stdout.strip().splitlines()[-1]) == want


def test_batched_minmaxlttb_arguments_are_checked_on_the_host(lib):
    """tsds_batched_minmaxlttb rejects bad batches before anything runs and names the series."""
    import numpy as np
    y, out, cnt = 1 << 20, 1 << 24, 1 << 28

    def arr(rows):
        a = np.zeros((len(rows), 6), dtype=np.uint64)
        for i, r in enumerate(rows):
            a[i] = r
        return a

    good = [0, y, 1000, 100, out, cnt]
    f = binding.tsds_batched_minmaxlttb
    a = arr([good, good])
    assert f(binding._array_ptr(a), 0, 0, 9, 4, 0, None) == 1                       # count 0
    assert f(None, 2, 0, 9, 4, 0, None) == 1                                         # no series
    assert f(binding._array_ptr(a), 2, 0, 9, 0, 0, None) == 1                        # ratio 0
    assert "minmax_ratio" in pkg.last_error()
    assert f(binding._array_ptr(a), 2, 0, 11, 4, 0, None) == 1                       # y dtype
    assert f(binding._array_ptr(a), 2, 0, 9, 4, 2, None) == 1                        # NaN mode
    b = arr([good, [0, y, 1000, 2, out, cnt]])
    assert f(binding._array_ptr(b), 2, 0, 9, 4, 0, None) == 1                        # n_out < 3
    assert "series 1" in pkg.last_error()
    b = arr([good, [0, y, 1000, 100, out, 0]])
    assert f(binding._array_ptr(b), 2, 0, 9, 4, 0, None) == 1                        # no count word
    b = arr([good, [1 << 30, y, 1000, 100, out, cnt]])
    assert f(binding._array_ptr(b), 2, 3, 9, 4, 0, None) == 1                        # x on one series only
    b = arr([good, [0, y + 2, 1000, 100, out, cnt]])
    assert f(binding._array_ptr(b), 2, 0, 9, 4, 0, None) == 1                        # misaligned float32 y
    b = arr([good, [0, y, 1000, 1 << 40, out, cnt]])
    assert f(binding._array_ptr(b), 2, 0, 9, 1 << 40, 0, None) == 1                  # n_out * ratio overflows
    assert "overflows" in pkg.last_error()


def test_binding_rejects_host_tensors_and_bad_shapes_before_any_call(lib):
    """The torch-facing helpers check their tensors on the host: CPU tensors, 2-D tensors, an x
    of another length and unknown names raise before anything reaches the library."""
    torch = pytest.importorskip("torch")
    y = torch.zeros(100, dtype=torch.float32)
    before = pkg.tsds_kernel_launches()
    for algo in ("minmax", "m4", "lttb", "minmaxlttb", "everynth"):
        with pytest.raises(ValueError):
            binding.downsample(algo, y, 10)                       # host tensor
        with pytest.raises(ValueError):
            binding.downsample_values(algo, y, 10)
    with pytest.raises(ValueError):
        binding.downsample("minmax", y.reshape(10, 10), 4)
    with pytest.raises(ValueError):
        binding.read_stream(y, torch.zeros(1, dtype=torch.int64))
    with pytest.raises(ValueError):
        binding.tsds_stream_variant("fastest")
    with pytest.raises(TypeError):
        binding.MinMaxDownsampler().downsample(y, y, y, n_out=4)
    assert pkg.tsds_kernel_launches() == before


@pytest.mark.parametrize("fn", [binding.tsds_minmax_bins, binding.tsds_m4_bins])
def test_bin_range_arguments_are_checked_on_the_host(lib, fn):
    """tsds_minmax_bins / tsds_m4_bins refuse a range outside [0, nb), a reversed range, an n_out
    that covers every index and an invalid n_out, before anything reaches the device."""
    before = pkg.tsds_kernel_launches()
    y, out, cnt = 1 << 20, 1 << 21, 1 << 22
    nb = 400 // (2 if fn is binding.tsds_minmax_bins else 4)
    for n_out, lo, hi in ((400, -1, 3), (400, 5, 4), (400, 0, nb + 1), (1000, 0, 1), (5, 0, 1), (0, 0, 0)):
        assert fn(None, 0, y, 9, 1000, n_out, lo, hi, 0, out, cnt, None) == 1, (n_out, lo, hi)
        assert pkg.last_error()
    assert pkg.tsds_kernel_launches() == before


def test_host_entry_arguments_are_checked_on_the_host(lib):
    """tsds_downsample_host refuses a bad count, an unknown algorithm, an invalid n_out, a NULL
    output and a misaligned y_dev before anything reaches the device."""
    import ctypes
    before = pkg.tsds_kernel_launches()
    y = (ctypes.c_float * 1000)()
    out = (ctypes.c_int64 * 1000)()
    counts = (ctypes.c_int64 * 2)()
    outs = (ctypes.c_void_p * 2)(ctypes.addressof(out), ctypes.addressof(out))
    null_outs = (ctypes.c_void_p * 2)(None, None)

    def call(count, algos, n_outs, outs_=outs, y_dev=None):
        a = (ctypes.c_int * max(len(algos), 1))(*algos)
        k = (ctypes.c_int64 * max(len(n_outs), 1))(*n_outs)
        return binding.tsds_downsample_host(count, a, k, None, 0, ctypes.addressof(y), 9, 1000, 0, y_dev, outs_,
                                            counts, None)

    cases = [(0, [0], [100]), (17, [0], [100]), (1, [2], [100]), (1, [0], [101]), (1, [1], [102]),
             (1, [1], [0]), (2, [0, 1], [100, 6])]
    for count, algos, n_outs in cases:
        assert call(count, algos, n_outs) == 1, (count, algos, n_outs)
        assert pkg.last_error()
    assert call(1, [0], [100], outs_=null_outs) == 1
    assert call(1, [0], [100], y_dev=1 << 20 | 2) == 1
    assert pkg.tsds_kernel_launches() == before
