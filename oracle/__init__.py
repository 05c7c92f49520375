"""CPU oracle for MinMax, M4, LTTB and MinMaxLTTB (arXiv 2307.05389).

TEST INFRASTRUCTURE ONLY.  This package wraps ``tsds_oracle.c``, a plain,
slow, single-threaded C restatement of the algorithms (see the header of that
file for the readings it follows).  The test suite, the smoke check and the
benchmark's CPU-baseline leg are its only users; the CUDA library never
imports, links or calls it, and the two share no code.

Arrays are numpy arrays on the host.  ``build()`` compiles the shared library
in place with ``-O2 -ffp-contract=off``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsds_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libtsds_oracle.so")

# Element type codes of tsds_oracle.h (the oracle's own numbering).
DTYPE_CODES = {
    "int8": 0, "int16": 1, "int32": 2, "int64": 3,
    "uint8": 4, "uint16": 5, "uint32": 6, "uint64": 7,
    "float16": 8, "float32": 9, "float64": 10,
}
NAN_MODES = {"propagate": 0, "ignore": 1}
EINVAL = -1

_lib = None


def build(force: bool = False) -> str:
    """Compile libtsds_oracle.so next to its source; return its path."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(os.path.join(_HERE, "tsds_oracle.h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
           "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    # TSDS_ORACLE_LIB loads another build of the same source instead (the
    # mutation test compiles copies with one planted mistake each)
    lib = ctypes.CDLL(os.environ.get("TSDS_ORACLE_LIB") or build())
    p, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.orc_f16_to_f64.argtypes = [ctypes.c_uint16]
    lib.orc_f16_to_f64.restype = ctypes.c_double
    lib.orc_bin_edges.argtypes = [p, c_int, i64, i64, p]
    lib.orc_bin_edges.restype = i64
    lib.orc_argminmax.argtypes = [p, c_int, i64, i64, c_int, p, p]
    lib.orc_argminmax.restype = c_int
    for name in ("orc_minmax", "orc_m4", "orc_lttb", "orc_everynth"):
        f = getattr(lib, name)
        f.argtypes = [p, c_int, p, c_int, i64, i64, c_int, p]
        f.restype = i64
    lib.orc_binned_range.argtypes = [c_int, p, c_int, p, c_int, i64, i64, c_int, i64, i64, p]
    lib.orc_binned_range.restype = i64
    lib.orc_minmaxlttb.argtypes = [p, c_int, p, c_int, i64, i64, i64, c_int, p]
    lib.orc_minmaxlttb.restype = i64
    lib.orc_lttb_points.argtypes = [p, p, i64, i64, c_int, p]
    lib.orc_lttb_points.restype = i64
    lib.orc_lttb_means.argtypes = [p, c_int, p, c_int, i64, i64, c_int, p]
    lib.orc_lttb_means.restype = i64
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _prep(x, y):
    y = np.ascontiguousarray(y)
    if y.dtype.name not in DTYPE_CODES:
        raise TypeError(f"unsupported y dtype {y.dtype}")
    if x is not None:
        x = np.ascontiguousarray(x)
        if x.dtype.name not in DTYPE_CODES:
            raise TypeError(f"unsupported x dtype {x.dtype}")
        if x.shape[0] != y.shape[0]:
            raise ValueError("x and y differ in length")
    return x, y


class OracleError(ValueError):
    pass


def _call(name, x, y, n_out, nan, extra=()):
    lib = _load()
    x, y = _prep(x, y)
    n = y.shape[0]
    cap = max(n, n_out, 1)
    out = np.empty(cap, dtype=np.int64)
    xc = DTYPE_CODES[x.dtype.name] if x is not None else 0
    args = [_ptr(x), xc, _ptr(y), DTYPE_CODES[y.dtype.name], n, n_out]
    if name == "orc_minmaxlttb":
        args += list(extra)
    args += [NAN_MODES[nan], _ptr(out)]
    r = getattr(lib, name)(*args)
    if r < 0:
        raise OracleError(f"{name}: invalid arguments (n={n}, n_out={n_out})")
    return out[:r].copy()


def minmax(x, y, n_out, nan="propagate"):
    return _call("orc_minmax", x, y, n_out, nan)


def m4(x, y, n_out, nan="propagate"):
    return _call("orc_m4", x, y, n_out, nan)


def lttb(x, y, n_out, nan="propagate"):
    return _call("orc_lttb", x, y, n_out, nan)


def everynth(x, y, n_out, nan="propagate"):
    return _call("orc_everynth", x, y, n_out, nan)


def minmaxlttb(x, y, n_out, minmax_ratio=4, nan="propagate"):
    return _call("orc_minmaxlttb", x, y, n_out, nan, extra=(minmax_ratio,))


def downsample(algo, x, y, n_out, nan="propagate", minmax_ratio=4):
    if algo == "minmax":
        return minmax(x, y, n_out, nan)
    if algo == "m4":
        return m4(x, y, n_out, nan)
    if algo == "lttb":
        return lttb(x, y, n_out, nan)
    if algo == "minmaxlttb":
        return minmaxlttb(x, y, n_out, minmax_ratio, nan)
    if algo == "everynth":
        return everynth(x, y, n_out, nan)
    raise ValueError(algo)


def binned_range(algo, x, y, n_out, b0, b1, nan="propagate"):
    """What bins [b0, b1) of MinMax or M4 select, the bins laid out over the whole
    series (n_out < len(y)); the whole output is the concatenation over
    consecutive bin ranges."""
    lib = _load()
    x, y = _prep(x, y)
    per_bin = {"minmax": 2, "m4": 4}[algo]
    out = np.empty(max(per_bin * (b1 - b0), 1), dtype=np.int64)
    xc = DTYPE_CODES[x.dtype.name] if x is not None else 0
    r = lib.orc_binned_range(per_bin, _ptr(x), xc, _ptr(y), DTYPE_CODES[y.dtype.name], y.shape[0], n_out,
                             NAN_MODES[nan], b0, b1, _ptr(out))
    if r < 0:
        raise OracleError(f"binned_range: invalid arguments (n={y.shape[0]}, n_out={n_out}, bins [{b0}, {b1}))")
    return out[:r].copy()


def binned_threads(algo, x, y, n_out, nan="propagate", threads=None):
    """MinMax or M4 of a large series as the concatenation of binned_range over
    consecutive bin ranges run on host threads (each call is the single-threaded
    oracle; the C calls release the GIL).  Equal to minmax/m4 by bin
    independence, which the tests pin on small inputs."""
    import concurrent.futures as cf
    n = np.asarray(y).shape[0]
    if n_out >= n:
        return downsample(algo, x, y, n_out, nan)
    nb = n_out // {"minmax": 2, "m4": 4}[algo]
    k = max(1, min(nb, threads or os.cpu_count() or 1))
    cuts = [nb * i // k for i in range(k + 1)]
    x, y = _prep(x, y)
    with cf.ThreadPoolExecutor(k) as ex:
        parts = list(ex.map(lambda i: binned_range(algo, x, y, n_out, cuts[i], cuts[i + 1], nan), range(k)))
    return np.concatenate(parts)


def bin_edges(x, n, nb):
    lib = _load()
    s = np.empty(nb + 1, dtype=np.int64)
    if x is not None:
        x = np.ascontiguousarray(x)
    r = lib.orc_bin_edges(_ptr(x), DTYPE_CODES[x.dtype.name] if x is not None else 0, n, nb, _ptr(s))
    if r < 0:
        raise OracleError("bin_edges: invalid arguments")
    return s


def argminmax(y, lo, hi, nan="propagate"):
    lib = _load()
    y = np.ascontiguousarray(y)
    a = ctypes.c_int64()
    b = ctypes.c_int64()
    r = lib.orc_argminmax(_ptr(y), DTYPE_CODES[y.dtype.name], lo, hi, NAN_MODES[nan],
                          ctypes.byref(a), ctypes.byref(b))
    if r < 0:
        raise OracleError("argminmax: invalid arguments")
    return a.value, b.value


def lttb_points(px, py, n_out, nan="propagate"):
    lib = _load()
    py = np.ascontiguousarray(py, dtype=np.float64)
    if px is not None:
        px = np.ascontiguousarray(px, dtype=np.float64)
    m = py.shape[0]
    out = np.empty(max(m, n_out, 1), dtype=np.int64)
    r = lib.orc_lttb_points(_ptr(px), _ptr(py), m, n_out, NAN_MODES[nan], _ptr(out))
    if r < 0:
        raise OracleError("lttb_points: invalid arguments")
    return out[:r].copy()


def lttb_means(x, y, n_out, nan="propagate"):
    """(n_out-3, 2) array: the (x, y) average of LTTB buckets 1 .. n_out-3."""
    lib = _load()
    x, y = _prep(x, y)
    n = y.shape[0]
    out = np.empty((max(n_out - 3, 0), 2), dtype=np.float64)
    xc = DTYPE_CODES[x.dtype.name] if x is not None else 0
    r = lib.orc_lttb_means(_ptr(x), xc, _ptr(y), DTYPE_CODES[y.dtype.name], n, n_out, NAN_MODES[nan], _ptr(out))
    if r < 0:
        raise OracleError(f"lttb_means: invalid arguments (n={n}, n_out={n_out})")
    return out


def f16_to_f64(bits: int) -> float:
    return _load().orc_f16_to_f64(bits)
