"""ctypes binding of libtsds.so (the C ABI in include/tsds.h).

The functions named like the C entry points take raw device pointers and
return the tsds_status code; ``downsample`` and the ``*Downsampler`` classes
marshal torch tensors onto them.  Every step of the computation runs in the
library's CUDA kernels; there is no CPU path, and a missing library raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtsds.so")

DTYPES = {
    "int8": 0, "int16": 1, "int32": 2, "int64": 3,
    "uint8": 4, "uint16": 5, "uint32": 6, "uint64": 7,
    "float16": 8, "float32": 9, "float64": 10,
}
NAN_MODES = {"propagate": 0, "ignore": 1}
STATUS = {0: "TSDS_OK", 1: "TSDS_EINVAL", 2: "TSDS_ENOMEM", 3: "TSDS_ECUDA", 4: "TSDS_ETIMEOUT",
          5: "TSDS_EINTERNAL"}

ENTRY_POINTS = ["tsds_minmax", "tsds_m4", "tsds_lttb", "tsds_minmaxlttb", "tsds_last_error",
                "tsds_shutdown", "tsds_version"]

_lib = None


class TsdsError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load libtsds.so (built by paper_2307_05389_gb300.build) and declare its symbols."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2307_05389_gb300.build`")
    lib = ctypes.CDLL(path)
    p, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    for name in ("tsds_minmax", "tsds_m4", "tsds_lttb", "tsds_everynth"):
        f = getattr(lib, name)
        f.argtypes = [p, c_int, p, c_int, i64, i64, c_int, p, p, p]
        f.restype = c_int
    lib.tsds_minmaxlttb.argtypes = [p, c_int, p, c_int, i64, i64, i64, c_int, p, p, p]
    lib.tsds_minmaxlttb.restype = c_int
    for name in ("tsds_minmax_bins", "tsds_m4_bins"):
        f = getattr(lib, name)
        f.argtypes = [p, c_int, p, c_int, i64, i64, i64, i64, c_int, p, p, p]
        f.restype = c_int
    lib.tsds_downsample_host.argtypes = [c_int, ctypes.POINTER(c_int), ctypes.POINTER(i64), p, c_int, p, c_int, i64,
                                         c_int, p, ctypes.POINTER(p), ctypes.POINTER(i64), p]
    lib.tsds_downsample_host.restype = c_int
    lib.tsds_last_error.argtypes = []
    lib.tsds_last_error.restype = ctypes.c_char_p
    lib.tsds_shutdown.argtypes = []
    lib.tsds_shutdown.restype = None
    lib.tsds_version.argtypes = []
    lib.tsds_version.restype = ctypes.c_char_p
    lib.tsds_batched.argtypes = [c_int, p, i64, c_int, c_int, c_int, p]
    lib.tsds_batched_minmaxlttb.argtypes = [p, i64, c_int, c_int, i64, c_int, p]
    lib.tsds_batched_minmaxlttb.restype = c_int
    lib.tsds_batched.restype = c_int
    lib.tsds_plan_create.argtypes = [ctypes.POINTER(p), c_int, p, i64, c_int, c_int, c_int, c_int, p]
    lib.tsds_plan_create.restype = c_int
    lib.tsds_plan_execute.argtypes = [p, p]
    lib.tsds_plan_execute.restype = c_int
    lib.tsds_plan_info.argtypes = [p, ctypes.POINTER(i64), ctypes.POINTER(c_int), ctypes.POINTER(i64),
                                   ctypes.POINTER(i64), ctypes.POINTER(c_int)]
    lib.tsds_plan_info.restype = c_int
    lib.tsds_plan_destroy.argtypes = [p]
    lib.tsds_plan_destroy.restype = c_int
    lib.tsds_minmax_noalloc.argtypes = [p, c_int, p, c_int, i64, i64, c_int, p, p, p]
    lib.tsds_minmax_noalloc.restype = c_int
    lib.tsds_check_wait_timeout.argtypes = [ctypes.c_uint, p]
    lib.tsds_check_wait_timeout.restype = c_int
    lib.tsds_kernel_launches.argtypes = []
    lib.tsds_kernel_launches.restype = i64
    lib.tsds_timing_enable.argtypes = [c_int]
    lib.tsds_timing_enable.restype = None
    lib.tsds_timing_read.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
    lib.tsds_timing_read.restype = c_int
    lib.tsds_stream_variant.argtypes = [c_int]
    lib.tsds_stream_variant.restype = c_int
    lib.tsds_lttb_means.argtypes = [p, c_int, p, c_int, i64, i64, c_int, p, p]
    lib.tsds_lttb_means.restype = c_int
    for name in ("tsds_minmax_values", "tsds_m4_values", "tsds_lttb_values", "tsds_everynth_values"):
        f = getattr(lib, name)
        f.argtypes = [p, c_int, p, c_int, i64, i64, c_int, p, p, p, p, p]
        f.restype = c_int
    lib.tsds_minmaxlttb_values.argtypes = [p, c_int, p, c_int, i64, i64, i64, c_int, p, p, p, p, p]
    lib.tsds_minmaxlttb_values.restype = c_int
    lib.tsds_read_stream.argtypes = [p, i64, p, p]
    lib.tsds_read_stream.restype = c_int
    lib.tsds_checked.argtypes = [c_int]
    lib.tsds_checked.restype = c_int
    lib.tsds_inject_alloc_failures.argtypes = [c_int]
    lib.tsds_inject_alloc_failures.restype = None
    _lib = lib
    return lib


def tsds_kernel_launches() -> int:
    return int(load().tsds_kernel_launches())


def tsds_timing_enable(on: bool) -> None:
    load().tsds_timing_enable(1 if on else 0)


STREAM_VARIANTS = {"auto": 0, "ring": 1, "ldg": 2, "seg": 3, "grp": 4}


def tsds_stream_variant(variant) -> str:
    """Sets the streaming-pass kernel variant ("auto", "ring", "ldg", "seg", "grp" or 0..4)
    for later calls; returns the previous one by name."""
    if isinstance(variant, str) and variant not in STREAM_VARIANTS:
        raise ValueError(f"unknown stream variant {variant!r}")
    v = STREAM_VARIANTS[variant] if isinstance(variant, str) else int(variant)
    prev = load().tsds_stream_variant(v)
    if prev < 0:
        raise ValueError(f"unknown stream variant {variant!r}")
    return {b: a for a, b in STREAM_VARIANTS.items()}[prev]


def tsds_timing_read():
    """(total device milliseconds, launches) of the timed streaming launches since the last read."""
    ms = ctypes.c_double()
    k = ctypes.c_int64()
    r = load().tsds_timing_read(ctypes.byref(ms), ctypes.byref(k))
    if r != 0:
        raise TsdsError(r, last_error())
    return ms.value, k.value


def tsds_checked(on: int = -1) -> int:
    """Checked mode (x sortedness verified on the device before each call that takes x):
    on = 0/1 sets it, on < 0 only queries; returns the previous mode."""
    return int(load().tsds_checked(int(on)))


def tsds_inject_alloc_failures(count: int) -> None:
    """Failure injection for tests: the next `count` device allocations of the library fail
    (the calls return TSDS_ENOMEM); count <= 0 clears it."""
    load().tsds_inject_alloc_failures(int(count))


def tsds_read_stream(buf, nbytes, sink, stream):
    return load().tsds_read_stream(buf, nbytes, sink, stream)


def read_stream(buf, sink, stream=None) -> None:
    """Reads every byte of the CUDA tensor `buf` once (the read-only streaming ceiling) and
    XORs the XOR of its 8-byte words into the one-element int64 CUDA tensor `sink`."""
    import torch
    if not buf.is_cuda or not buf.is_contiguous():
        raise ValueError("buf must be a contiguous CUDA tensor")
    if sink.dtype != torch.int64 or sink.numel() < 1 or sink.device != buf.device:
        raise ValueError("sink must be an int64 tensor on buf's device")
    nbytes = buf.numel() * buf.element_size()
    st = stream if stream is not None else torch.cuda.current_stream(buf.device)
    with torch.cuda.device(buf.device):
        r = tsds_read_stream(buf.data_ptr(), nbytes, sink.data_ptr(), ctypes.c_void_p(st.cuda_stream))
    if r != 0:
        raise TsdsError(r, last_error())


def last_error() -> str:
    return load().tsds_last_error().decode()


# ----------------------------------------------------------------------------- raw entry points

def tsds_minmax(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, stream):
    return load().tsds_minmax(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, stream)


def tsds_m4(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, stream):
    return load().tsds_m4(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, stream)


def tsds_lttb(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, stream):
    return load().tsds_lttb(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, stream)


def tsds_everynth(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, stream):
    return load().tsds_everynth(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, stream)


def tsds_everynth_values(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, x_out, y_out, stream):
    return load().tsds_everynth_values(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, x_out, y_out, stream)


def tsds_lttb_means(x, x_dtype, y, y_dtype, n, n_out, nan, means, stream):
    return load().tsds_lttb_means(x, x_dtype, y, y_dtype, n, n_out, nan, means, stream)


def tsds_minmax_values(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, x_out, y_out, stream):
    return load().tsds_minmax_values(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, x_out, y_out, stream)


def tsds_m4_values(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, x_out, y_out, stream):
    return load().tsds_m4_values(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, x_out, y_out, stream)


def tsds_lttb_values(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, x_out, y_out, stream):
    return load().tsds_lttb_values(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, x_out, y_out, stream)


def tsds_minmaxlttb_values(x, x_dtype, y, y_dtype, n, n_out, minmax_ratio, nan, out, out_count, x_out, y_out,
                           stream):
    return load().tsds_minmaxlttb_values(x, x_dtype, y, y_dtype, n, n_out, minmax_ratio, nan, out, out_count,
                                         x_out, y_out, stream)


def tsds_minmaxlttb(x, x_dtype, y, y_dtype, n, n_out, minmax_ratio, nan, out, out_count, stream):
    return load().tsds_minmaxlttb(x, x_dtype, y, y_dtype, n, n_out, minmax_ratio, nan, out, out_count, stream)


def tsds_minmax_bins(x, x_dtype, y, y_dtype, n, n_out, bin_lo, bin_hi, nan, out, out_count, stream):
    return load().tsds_minmax_bins(x, x_dtype, y, y_dtype, n, n_out, bin_lo, bin_hi, nan, out, out_count, stream)


def tsds_m4_bins(x, x_dtype, y, y_dtype, n, n_out, bin_lo, bin_hi, nan, out, out_count, stream):
    return load().tsds_m4_bins(x, x_dtype, y, y_dtype, n, n_out, bin_lo, bin_hi, nan, out, out_count, stream)


def tsds_downsample_host(count, algos, n_outs, x, x_dtype, y_host, y_dtype, n, nan, y_dev, outs_host, counts_host,
                         stream):
    """algos, n_outs: ctypes int / int64 arrays; outs_host: ctypes array of host pointers;
    counts_host: ctypes int64 array (see tsds.h)."""
    return load().tsds_downsample_host(count, algos, n_outs, x, x_dtype, y_host, y_dtype, n, nan, y_dev, outs_host,
                                       counts_host, stream)


def tsds_minmax_noalloc(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, stream):
    """MinMax for callers that cannot allocate device memory during a call:
    scratch comes from a fixed 8 MiB array inside the library (see tsds.h for
    the size limit and the rule that overlapping calls must be serialised)."""
    return load().tsds_minmax_noalloc(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, stream)


class tsds_series(ctypes.Structure):
    """One series of a batch (include/tsds.h); pointers are device addresses."""
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("n", ctypes.c_int64), ("n_out", ctypes.c_int64),
                ("out", ctypes.c_void_p), ("out_count", ctypes.c_void_p)]


ALGO_CODES = {"minmax": 0, "m4": 1}
PLAN_GRAPH = 1
PLAN_AUTOTUNE = 2


def tsds_batched(algo, series, count, x_dtype, y_dtype, nan, stream):
    return load().tsds_batched(algo, series, count, x_dtype, y_dtype, nan, stream)


def tsds_plan_create(plan_ref, algo, series, count, x_dtype, y_dtype, nan, flags, stream):
    return load().tsds_plan_create(plan_ref, algo, series, count, x_dtype, y_dtype, nan, flags, stream)


def tsds_plan_execute(plan, stream):
    return load().tsds_plan_execute(plan, stream)


def tsds_plan_info(plan, window_bytes, ctas_per_sm, windows, scratch_bytes, variant):
    return load().tsds_plan_info(plan, window_bytes, ctas_per_sm, windows, scratch_bytes, variant)


def tsds_plan_destroy(plan):
    return load().tsds_plan_destroy(plan)


def _series_array(ys, n_outs, xs, outs, counts):
    """The tsds_series array of a batch, built column-wise with numpy (48-byte
    records: x, y, n, n_out, out, out_count); returns the array, which owns
    the memory the pointer refers to."""
    import numpy as np
    k = len(ys)
    a = np.zeros((k, 6), dtype=np.uint64)
    if xs is not None:
        a[:, 0] = [x.data_ptr() for x in xs]
    a[:, 1] = [y.data_ptr() for y in ys]
    a[:, 2] = [y.shape[0] for y in ys]
    a[:, 3] = np.asarray(n_outs, dtype=np.int64).astype(np.uint64)
    a[:, 4] = [o.data_ptr() for o in outs]
    a[:, 5] = counts.data_ptr() + 8 * np.arange(k, dtype=np.uint64)
    return a


def _array_ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def batch_buffers(ys, n_outs, device):
    """Output buffers for a batch: one int64 tensor per series and one count tensor."""
    import torch
    outs = [torch.empty(out_capacity("", y.shape[0], int(k)), dtype=torch.int64, device=device)
            for y, k in zip(ys, n_outs)]
    counts = torch.empty(len(ys), dtype=torch.int64, device=device)
    return outs, counts


def tsds_batched_minmaxlttb(series, count, x_dtype, y_dtype, minmax_ratio, nan, stream):
    return load().tsds_batched_minmaxlttb(series, count, x_dtype, y_dtype, minmax_ratio, nan, stream)


def downsample_batched(algo, ys, n_outs, xs=None, nan="propagate", stream=None, outs=None, counts=None,
                       y_dtype=None, x_dtype=None, minmax_ratio=4):
    """MinMax, M4 or MinMaxLTTB of every CUDA tensor in `ys` in one launch sequence.
    Returns (outs, counts) device tensors (outs[i][:counts[i]] are series i's indices)."""
    import torch
    dev = ys[0].device
    if outs is None or counts is None:
        outs, counts = batch_buffers(ys, n_outs, dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    arr = _series_array(ys, n_outs, xs, outs, counts)
    yd = DTYPES[y_dtype or _torch_dtype_name(ys[0])]
    xd = DTYPES[x_dtype or _torch_dtype_name(xs[0])] if xs is not None else 0
    with torch.cuda.device(dev):
        if algo == "minmaxlttb":
            r = tsds_batched_minmaxlttb(_array_ptr(arr), len(ys), xd, yd, int(minmax_ratio), NAN_MODES[nan],
                                        ctypes.c_void_p(st.cuda_stream))
        else:
            r = tsds_batched(ALGO_CODES[algo], _array_ptr(arr), len(ys), xd, yd, NAN_MODES[nan],
                             ctypes.c_void_p(st.cuda_stream))
    if r != 0:
        raise TsdsError(r, last_error())
    return outs, counts


class Plan:
    """A resident batch (tsds_plan_*): create once, execute many times."""

    def __init__(self, algo, ys, n_outs, xs=None, nan="propagate", graph=True, autotune=False, stream=None,
                 y_dtype=None, x_dtype=None):
        import torch
        self.device = ys[0].device
        self.outs, self.counts = batch_buffers(ys, n_outs, self.device)
        self._keep = (ys, xs)
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        arr = _series_array(ys, n_outs, xs, self.outs, self.counts)
        yd = DTYPES[y_dtype or _torch_dtype_name(ys[0])]
        xd = DTYPES[x_dtype or _torch_dtype_name(xs[0])] if xs is not None else 0
        self.handle = ctypes.c_void_p()
        flags = (PLAN_GRAPH if graph else 0) | (PLAN_AUTOTUNE if autotune else 0)
        with torch.cuda.device(self.device):
            r = tsds_plan_create(ctypes.byref(self.handle), ALGO_CODES[algo], _array_ptr(arr), len(ys), xd, yd,
                                 NAN_MODES[nan], flags, ctypes.c_void_p(st.cuda_stream))
        if r != 0:
            raise TsdsError(r, last_error())

    def execute(self, stream=None):
        import torch
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        r = tsds_plan_execute(self.handle, ctypes.c_void_p(st.cuda_stream))
        if r != 0:
            raise TsdsError(r, last_error())
        return self.outs, self.counts

    def info(self):
        wb, cp, w, sb, var = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        r = tsds_plan_info(self.handle, ctypes.byref(wb), ctypes.byref(cp), ctypes.byref(w), ctypes.byref(sb),
                           ctypes.byref(var))
        if r != 0:
            raise TsdsError(r, last_error())
        names = {b: a for a, b in STREAM_VARIANTS.items()}
        return {"window_bytes": wb.value, "ctas_per_sm": cp.value, "windows": w.value, "scratch_bytes": sb.value,
                "variant": names.get(var.value, var.value)}

    def close(self):
        if self.handle:
            tsds_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class tsds_query(ctypes.Structure):
    _fields_ = [("series", ctypes.c_int64), ("algo", ctypes.c_int32), ("nan", ctypes.c_int32),
                ("by_x", ctypes.c_int32), ("reserved", ctypes.c_int32), ("x_lo", ctypes.c_double),
                ("x_hi", ctypes.c_double), ("lo", ctypes.c_int64), ("hi", ctypes.c_int64),
                ("n_out", ctypes.c_int64), ("minmax_ratio", ctypes.c_int64)]


class tsds_server_config(ctypes.Structure):
    _fields_ = [("streams", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("memory_budget", ctypes.c_int64)]


class tsds_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("points", ctypes.c_int64), ("bytes", ctypes.c_int64), ("span_s", ctypes.c_double),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("max_us", ctypes.c_double)]


SERVER_ALGOS = {"minmax": 0, "m4": 1, "minmaxlttb": 2}


def _declare_server(lib):
    p, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.tsds_server_create.argtypes = [ctypes.POINTER(p), ctypes.POINTER(tsds_server_config), c_int, c_int]
    lib.tsds_server_create.restype = c_int
    lib.tsds_server_add_series.argtypes = [p, p, p, i64, ctypes.POINTER(i64)]
    lib.tsds_server_add_series.restype = c_int
    lib.tsds_server_submit.argtypes = [p, ctypes.POINTER(tsds_query), ctypes.POINTER(i64)]
    lib.tsds_server_submit.restype = c_int
    lib.tsds_server_result.argtypes = [p, i64, i64, p, i64, ctypes.POINTER(i64), ctypes.POINTER(c_int),
                                       ctypes.POINTER(ctypes.c_double)]
    lib.tsds_server_result.restype = c_int
    lib.tsds_server_stats_get.argtypes = [p, ctypes.POINTER(tsds_server_stats)]
    lib.tsds_server_stats_get.restype = c_int
    lib.tsds_server_reset_stats.argtypes = [p]
    lib.tsds_server_reset_stats.restype = c_int
    lib.tsds_server_destroy.argtypes = [p]
    lib.tsds_server_destroy.restype = c_int


class Server:
    """Continuous-batching server over resident series (tsds_server_*)."""

    def __init__(self, y_dtype, x_dtype=None, streams=2, max_batch=256, memory_budget=1 << 30):
        lib = load()
        if not hasattr(lib, "_server_declared"):
            _declare_server(lib)
            lib._server_declared = True
        self.lib = lib
        cfg = tsds_server_config(streams, max_batch, memory_budget)
        self.handle = ctypes.c_void_p()
        r = lib.tsds_server_create(ctypes.byref(self.handle), ctypes.byref(cfg),
                                   DTYPES[x_dtype] if x_dtype else 0, DTYPES[y_dtype])
        if r != 0:
            raise TsdsError(r, last_error())
        self._keep = []
        self.n_out = {}

    def add_series(self, y, x=None):
        sid = ctypes.c_int64()
        r = self.lib.tsds_server_add_series(self.handle, x.data_ptr() if x is not None else None, y.data_ptr(),
                                            y.shape[0], ctypes.byref(sid))
        if r != 0:
            raise TsdsError(r, last_error())
        self._keep.append((y, x))
        return sid.value

    def submit(self, series, algo, n_out, x_range=None, index_range=None, nan="propagate", minmax_ratio=4):
        q = tsds_query()
        q.series = series
        q.algo = SERVER_ALGOS[algo]
        q.nan = NAN_MODES[nan]
        if x_range is not None:
            q.by_x = 1
            q.x_lo, q.x_hi = float(x_range[0]), float(x_range[1])
        else:
            q.by_x = 0
            q.lo, q.hi = (0, 2 ** 62) if index_range is None else (int(index_range[0]), int(index_range[1]))
        q.n_out = n_out
        q.minmax_ratio = minmax_ratio
        t = ctypes.c_int64()
        r = self.lib.tsds_server_submit(self.handle, ctypes.byref(q), ctypes.byref(t))
        if r != 0:
            raise TsdsError(r, last_error())
        self.n_out[t.value] = n_out
        return t.value

    def result(self, ticket, timeout_us=-1):
        """(indices as numpy int64, latency in µs), or None if not done within the timeout."""
        import numpy as np
        cap = self.n_out.get(ticket, 1)
        out = np.empty(max(cap, 1), dtype=np.int64)
        cnt, done, lat = ctypes.c_int64(), ctypes.c_int(), ctypes.c_double()
        r = self.lib.tsds_server_result(self.handle, ticket, timeout_us, out.ctypes.data_as(ctypes.c_void_p), cap,
                                        ctypes.byref(cnt), ctypes.byref(done), ctypes.byref(lat))
        if r != 0:
            raise TsdsError(r, last_error())
        if not done.value:
            return None
        self.n_out.pop(ticket, None)
        return out[:cnt.value].copy(), lat.value

    def stats(self):
        s = tsds_server_stats()
        r = self.lib.tsds_server_stats_get(self.handle, ctypes.byref(s))
        if r != 0:
            raise TsdsError(r, last_error())
        return {f: getattr(s, f) for f, _ in tsds_server_stats._fields_}

    def reset_stats(self):
        self.lib.tsds_server_reset_stats(self.handle)

    def close(self):
        if self.handle:
            self.lib.tsds_server_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tsds_shutdown():
    load().tsds_shutdown()


def tsds_version() -> str:
    return load().tsds_version().decode()


# ----------------------------------------------------------------------------- torch marshalling

def _torch_dtype_name(t) -> str:
    name = str(t.dtype).replace("torch.", "")
    if name not in DTYPES:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return name


def out_capacity(algo: str, n: int, n_out: int) -> int:
    return max(1, n if n_out >= n else n_out)


def lttb_means(y, n_out, x=None, nan="propagate"):
    """The (x, y) averages of LTTB buckets 1 .. n_out-3 on a CUDA tensor y (and x), as a
    (n_out-3, 2) float64 device tensor (tsds_lttb_means)."""
    import torch
    n = y.shape[0]
    means = torch.empty((max(n_out - 3, 0), 2), dtype=torch.float64, device=y.device)
    st = torch.cuda.current_stream(y.device)
    xp = x.data_ptr() if x is not None else None
    xd = DTYPES[_torch_dtype_name(x)] if x is not None else 0
    with torch.cuda.device(y.device):
        r = tsds_lttb_means(xp, xd, y.data_ptr(), DTYPES[_torch_dtype_name(y)], n, n_out, NAN_MODES[nan],
                            means.data_ptr(), ctypes.c_void_p(st.cuda_stream))
    if r != 0:
        raise TsdsError(r, last_error())
    return means


def downsample_values(algo, y, n_out, x=None, nan="propagate", minmax_ratio=4):
    """Indices selected by `algo` with the selected points' values gathered in the same
    launch: returns (indices, x_values or None, y_values), CUDA tensors trimmed to the count
    (one device-to-host read of the count)."""
    import torch
    if not (y.is_cuda and y.dim() == 1 and y.is_contiguous()):
        raise ValueError("y must be a contiguous 1-D CUDA tensor")
    n = y.shape[0]
    if x is not None and not (x.is_cuda and x.dim() == 1 and x.is_contiguous() and x.shape[0] == n):
        raise ValueError("x must be a contiguous 1-D CUDA tensor as long as y")
    dev = y.device
    cap = out_capacity(algo, n, n_out)
    out = torch.empty(cap, dtype=torch.int64, device=dev)
    cnt = torch.empty(1, dtype=torch.int64, device=dev)
    y_out = torch.empty(cap, dtype=y.dtype, device=dev)
    x_out = torch.empty(cap, dtype=x.dtype, device=dev) if x is not None else None
    st = torch.cuda.current_stream(dev)
    xp = x.data_ptr() if x is not None else None
    xd = DTYPES[_torch_dtype_name(x)] if x is not None else 0
    args = (xp, xd, y.data_ptr(), DTYPES[_torch_dtype_name(y)], n, n_out)
    tail = (out.data_ptr(), cnt.data_ptr(), x_out.data_ptr() if x_out is not None else None, y_out.data_ptr(),
            ctypes.c_void_p(st.cuda_stream))
    with torch.cuda.device(dev):
        if algo == "minmax":
            r = tsds_minmax_values(*args, NAN_MODES[nan], *tail)
        elif algo == "m4":
            r = tsds_m4_values(*args, NAN_MODES[nan], *tail)
        elif algo == "lttb":
            r = tsds_lttb_values(*args, NAN_MODES[nan], *tail)
        elif algo == "everynth":
            r = tsds_everynth_values(*args, NAN_MODES[nan], *tail)
        elif algo == "minmaxlttb":
            r = tsds_minmaxlttb_values(*args, minmax_ratio, NAN_MODES[nan], *tail)
        else:
            raise ValueError(f"unknown algorithm {algo!r}")
    if r != 0:
        raise TsdsError(r, last_error())
    k = int(cnt.item())
    if k < 0:
        raise TsdsError(-k, "the streaming pass reported a device-side failure")
    return out[:k], (x_out[:k] if x_out is not None else None), y_out[:k]


def downsample(algo, y, n_out, x=None, nan="propagate", minmax_ratio=4, out=None, out_count=None,
               stream=None, sync=True):
    """Indices selected by `algo` ("minmax", "m4", "lttb", "minmaxlttb", "everynth") on y (and x).

    y and x are 1-D CUDA tensors (contiguous).  With sync=True the result is
    trimmed to the selected count (one device-to-host read of the count);
    with sync=False the call only enqueues work and returns (out, out_count)
    device tensors.  Errors raise TsdsError with the library's message."""
    import torch
    if not (y.is_cuda and y.dim() == 1 and y.is_contiguous()):
        raise ValueError("y must be a contiguous 1-D CUDA tensor")
    n = y.shape[0]
    if x is not None:
        if not (x.is_cuda and x.dim() == 1 and x.is_contiguous() and x.shape[0] == n):
            raise ValueError("x must be a contiguous 1-D CUDA tensor as long as y")
    dev = y.device
    if out is None:
        out = torch.empty(out_capacity(algo, n, n_out), dtype=torch.int64, device=dev)
    if out_count is None:
        out_count = torch.empty(1, dtype=torch.int64, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    xp = x.data_ptr() if x is not None else None
    xd = DTYPES[_torch_dtype_name(x)] if x is not None else 0
    args = (xp, xd, y.data_ptr(), DTYPES[_torch_dtype_name(y)], n, n_out)
    tail = (NAN_MODES[nan], out.data_ptr(), out_count.data_ptr(), ctypes.c_void_p(st.cuda_stream))
    with torch.cuda.device(dev):
        if algo == "minmax":
            r = tsds_minmax(*args, *tail)
        elif algo == "m4":
            r = tsds_m4(*args, *tail)
        elif algo == "lttb":
            r = tsds_lttb(*args, *tail)
        elif algo == "everynth":
            r = tsds_everynth(*args, *tail)
        elif algo == "minmaxlttb":
            r = tsds_minmaxlttb(*args, minmax_ratio, *tail)
        else:
            raise ValueError(f"unknown algorithm {algo!r}")
    if r != 0:
        raise TsdsError(r, last_error())
    if not sync:
        return out, out_count
    k = int(out_count.item())
    if k < 0:
        raise TsdsError(-k, "the streaming pass reported a device-side failure")
    return out[:k]


def downsample_bins(algo, y, n_out, bin_lo, bin_hi, x=None, nan="propagate", stream=None):
    """What bins [bin_lo, bin_hi) of MinMax or M4 select (tsds_minmax_bins / tsds_m4_bins),
    the bins laid out over the whole series; a device int64 tensor of global indices."""
    import torch
    if algo not in ("minmax", "m4"):
        raise ValueError(f"bin ranges cover MinMax and M4, not {algo!r}")
    if not (y.is_cuda and y.dim() == 1 and y.is_contiguous()):
        raise ValueError("y must be a contiguous 1-D CUDA tensor")
    n = y.shape[0]
    if x is not None and not (x.is_cuda and x.dim() == 1 and x.is_contiguous() and x.shape[0] == n):
        raise ValueError("x must be a contiguous 1-D CUDA tensor as long as y")
    per = 2 if algo == "minmax" else 4
    dev = y.device
    out = torch.empty(max(per * (bin_hi - bin_lo), 1), dtype=torch.int64, device=dev)
    cnt = torch.empty(1, dtype=torch.int64, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    fn = tsds_minmax_bins if algo == "minmax" else tsds_m4_bins
    with torch.cuda.device(dev):
        r = fn(x.data_ptr() if x is not None else None, DTYPES[_torch_dtype_name(x)] if x is not None else 0,
               y.data_ptr(), DTYPES[_torch_dtype_name(y)], n, n_out, bin_lo, bin_hi, NAN_MODES[nan], out.data_ptr(),
               cnt.data_ptr(), ctypes.c_void_p(st.cuda_stream))
    if r != 0:
        raise TsdsError(r, last_error())
    k = int(cnt.item())
    if k < 0:
        raise TsdsError(-k, "the streaming pass reported a device-side failure")
    return out[:k]


def downsample_host(algos, y, n_out, x=None, nan="propagate", minmax_ratio=4, device="cuda",
                    y_dev=None, x_dev=None):
    """Host-buffer form: y (a CPU tensor) goes to the device, each algorithm in
    `algos` runs on the GPU and each index list comes back as a CPU int64
    tensor.  When every algorithm is MinMax or M4 this is one
    tsds_downsample_host call: y is copied in chunks that overlap the
    reduction of the bins already on the device.  Otherwise y is copied once
    and the single-series calls run on the copy.  A pinned (or device) x is
    read in place by the bin search of MinMax, M4 and EveryNth (which probes
    only about log2(n) values per bin); otherwise x is copied too.  y_dev /
    x_dev may supply preallocated device buffers to copy into."""
    import torch
    st = torch.cuda.current_stream(device)
    if (not y.is_cuda and y.is_contiguous() and len(algos) > 0
            and all(a in ("minmax", "m4") for a in algos)):
        return _downsample_host_native(algos, y, n_out, x, nan, device, y_dev, x_dev, st)
    yd = y_dev if y_dev is not None else torch.empty_like(y, device=device)
    yd.copy_(y, non_blocking=True)
    xp, xd = None, 0
    if x is not None:
        if x.is_pinned() and all(a in ("minmax", "m4", "everynth") for a in algos):
            # page-locked x is read in place: the bin search probes about log2(n)
            # elements per bin, so x is not copied (the device reads pinned host
            # memory through its unified address)
            xp = x.data_ptr()
        else:
            xdev = x_dev if x_dev is not None else torch.empty_like(x, device=device)
            xdev.copy_(x, non_blocking=True)
            xp = xdev.data_ptr()
        xd = DTYPES[_torch_dtype_name(x)]
    fns = {"minmax": tsds_minmax, "m4": tsds_m4, "lttb": tsds_lttb, "everynth": tsds_everynth}
    n = yd.shape[0]
    res = []
    for algo in algos:
        out = torch.empty(out_capacity(algo, n, n_out), dtype=torch.int64, device=yd.device)
        cnt = torch.empty(1, dtype=torch.int64, device=yd.device)
        args = (xp, xd, yd.data_ptr(), DTYPES[_torch_dtype_name(yd)], n, n_out)
        tail = (NAN_MODES[nan], out.data_ptr(), cnt.data_ptr(), ctypes.c_void_p(st.cuda_stream))
        with torch.cuda.device(yd.device):
            if algo == "minmaxlttb":
                r = tsds_minmaxlttb(*args, minmax_ratio, *tail)
            elif algo in fns:
                r = fns[algo](*args, *tail)
            else:
                raise ValueError(f"unknown algorithm {algo!r}")
        if r != 0:
            raise TsdsError(r, last_error())
        k = int(cnt.item())
        if k < 0:
            raise TsdsError(-k, "the streaming pass reported a device-side failure")
        res.append(out[:k].cpu())
    return res


def _downsample_host_native(algos, y, n_out, x, nan, device, y_dev, x_dev, st):
    import torch
    n = y.shape[0]
    xp, xd = None, 0
    if x is not None:
        if x.is_cuda or x.is_pinned():
            xp = x.data_ptr()
        else:
            xdev = x_dev if x_dev is not None else torch.empty_like(x, device=device)
            xdev.copy_(x, non_blocking=False)
            xp = xdev.data_ptr()
        xd = DTYPES[_torch_dtype_name(x)]
    k = len(algos)
    codes = (ctypes.c_int * k)(*[{"minmax": 0, "m4": 1}[a] for a in algos])
    n_outs = (ctypes.c_int64 * k)(*([int(n_out)] * k))
    outs = [torch.empty(max(min(int(n_out), n), 1), dtype=torch.int64) for _ in algos]
    ptrs = (ctypes.c_void_p * k)(*[o.data_ptr() for o in outs])
    counts = (ctypes.c_int64 * k)()
    with torch.cuda.device(device):
        r = tsds_downsample_host(k, codes, n_outs, xp, xd, y.data_ptr(), DTYPES[_torch_dtype_name(y)], n,
                                 NAN_MODES[nan], y_dev.data_ptr() if y_dev is not None else None, ptrs, counts,
                                 ctypes.c_void_p(st.cuda_stream))
    if r != 0:
        raise TsdsError(r, last_error())
    return [o[:int(c)] for o, c in zip(outs, counts)]


class _Downsampler:
    """Class interface in the shape of the paper's (Section 2.3):
    ``Downsampler().downsample([x], y, n_out=..., **kwargs)``."""
    algo = ""

    def downsample(self, *args, n_out, nan="propagate", **kw):
        if len(args) == 1:
            x, y = None, args[0]
        elif len(args) == 2:
            x, y = args
        else:
            raise TypeError("downsample([x], y, n_out=...)")
        return downsample(self.algo, y, n_out, x=x, nan=nan, **kw)


class MinMaxDownsampler(_Downsampler):
    algo = "minmax"


class EveryNthDownsampler(_Downsampler):
    algo = "everynth"


class M4Downsampler(_Downsampler):
    algo = "m4"


class LTTBDownsampler(_Downsampler):
    algo = "lttb"


class MinMaxLTTBDownsampler(_Downsampler):
    algo = "minmaxlttb"

    def downsample(self, *args, n_out, minmax_ratio=4, nan="propagate", **kw):
        return super().downsample(*args, n_out=n_out, nan=nan, minmax_ratio=minmax_ratio, **kw)
