"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws numbers: it holds none of the downsampling arithmetic,
so both the CUDA path and the CPU oracle can be fed from it.  The paper
measures on arrays of random values of each dtype (Section 4, Table 1) and
downsamples a random series in its example (Section 3, Listing 2); the
recipes below follow those shapes:

* ``random_walk``     -- cumulative sum of N(0, 1) steps, cast to the dtype.
* ``quarter_range``   -- values uniform over one quarter of the dtype's range
                         (signed ints [min/4, max/4], uints [0, max/4],
                         floats [-max/4, max/4]).
* ``geometric_x``     -- sorted int64 timestamps: 0 then a cumulative sum of
                         geometric(p) gaps (gaps >= 1).
* ``exponential_x``   -- sorted float64 x: cumulative sum of exponential(1).
* ``quantised_nan``   -- a float64 random walk quantised to 256 levels, with a
                         given fraction of positions set to NaN.

Host generators use numpy's ``default_rng(seed)``; the ``*_cuda`` variants
draw the same distributions with torch's CUDA generator for sizes where host
generation would dominate the run.
"""
from __future__ import annotations

import numpy as np

DTYPES = ["int8", "int16", "int32", "int64", "uint8", "uint16", "uint32", "uint64",
          "float16", "float32", "float64"]


def random_walk(n: int, dtype="float32", seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.standard_normal(n)).astype(dtype)


def quarter_range(n: int, dtype: str, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    dt = np.dtype(dtype)
    if dt.kind == "f":
        hi = float(np.finfo(dt).max) / 4
        return rng.uniform(-hi, hi, n).astype(dt)
    info = np.iinfo(dt)
    if dt.kind == "i":
        lo, hi = info.min // 4, info.max // 4
    else:
        lo, hi = 0, info.max // 4
    return rng.integers(lo, hi, size=n, endpoint=True, dtype=dt)


def geometric_x(n: int, seed: int = 0, p: float = 0.5) -> np.ndarray:
    rng = np.random.default_rng(seed)
    x = np.zeros(n, dtype=np.int64)
    if n > 1:
        np.cumsum(rng.geometric(p, n - 1), out=x[1:])
    return x


def exponential_x(n: int, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0, n))


def quantised_nan(n: int, seed: int = 0, levels: int = 256, nan_frac: float = 0.01) -> np.ndarray:
    rng = np.random.default_rng(seed)
    w = np.cumsum(rng.standard_normal(n))
    lo, hi = w.min(), w.max()
    q = np.floor((w - lo) / (hi - lo if hi > lo else 1.0) * (levels - 1e-3))
    k = int(round(n * nan_frac))
    if k:
        q[rng.choice(n, size=k, replace=False)] = np.nan
    return q


def ties_and_specials(n: int, dtype: str, seed: int = 0) -> np.ndarray:
    """Few distinct values (heavy ties); floats also get -0, +0, +-inf and NaN."""
    rng = np.random.default_rng(seed)
    dt = np.dtype(dtype)
    if dt.kind == "f":
        pool = np.array([0.0, -0.0, 1.0, -1.0, 2.5, -2.5, np.inf, -np.inf, np.nan], dtype=np.float64)
        v = pool[rng.integers(0, len(pool), n)]
        return v.astype(dt)
    info = np.iinfo(dt)
    pool = np.array([info.min, info.min + 1, 0, 1, info.max - 1, info.max], dtype=object)
    return np.array(pool[rng.integers(0, len(pool), n)].tolist(), dtype=dt)


def batch_lengths(count: int, seed: int = 3, lo_exp: float = 3.0, hi_exp: float = 7.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.round(10.0 ** rng.uniform(lo_exp, hi_exp, count)).astype(np.int64)


def batch_n_out(count: int, seed: int = 3, lo: int = 200, hi: int = 4000, multiple: int = 4) -> np.ndarray:
    rng = np.random.default_rng(seed + 1)
    v = rng.integers(lo, hi, size=count, endpoint=True)
    return (v // multiple) * multiple


# ----------------------------------------------------------------------------- device-side draws
# Drawn in chunks of 2^27 elements, each chunk from its own generator seeded
# with (seed, chunk), so temporaries stay small for 4*10^9-element inputs.
# Unsigned dtypes come back in the signed dtype of the same width (their
# values are below the signed maximum, so the bytes are identical); pass the
# unsigned dtype code to the library.

_CHUNK = 1 << 27


def _gen(device, seed, chunk):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 1_000_003 + int(chunk))
    return g


def _signed_torch_dtype(dtype):
    import torch
    dt = np.dtype(dtype)
    if dt.kind == "u":
        return getattr(torch, f"int{8 * dt.itemsize}") if dt.itemsize > 1 else torch.uint8
    return getattr(torch, dtype)


def random_walk_cuda(n: int, dtype="float32", seed: int = 0, device="cuda"):
    import torch
    out = torch.empty(n, dtype=_signed_torch_dtype(dtype), device=device)
    carry = torch.zeros((), dtype=torch.float64, device=device)
    for c, lo in enumerate(range(0, n, _CHUNK)):
        hi = min(n, lo + _CHUNK)
        steps = torch.randn(hi - lo, generator=_gen(device, seed, c), device=device, dtype=torch.float32)
        w = torch.cumsum(steps, 0, dtype=torch.float64) + carry
        carry = w[-1].clone()
        out[lo:hi] = w.to(out.dtype)
    return out


def geometric_x_cuda(n: int, seed: int = 0, p: float = 0.5, device="cuda"):
    import torch
    out = torch.empty(n, dtype=torch.int64, device=device)
    carry = torch.zeros((), dtype=torch.int64, device=device)
    for c, lo in enumerate(range(0, n, _CHUNK)):
        hi = min(n, lo + _CHUNK)
        gaps = torch.empty(hi - lo, dtype=torch.float32, device=device).geometric_(p, generator=_gen(device, seed, c))
        gaps = gaps.to(torch.int64)
        if lo == 0:
            gaps[0] = 0
        w = torch.cumsum(gaps, 0) + carry
        carry = w[-1].clone()
        out[lo:hi] = w
    return out


def exponential_x_cuda(n: int, seed: int = 0, device="cuda"):
    import torch
    out = torch.empty(n, dtype=torch.float64, device=device)
    carry = torch.zeros((), dtype=torch.float64, device=device)
    for c, lo in enumerate(range(0, n, _CHUNK)):
        hi = min(n, lo + _CHUNK)
        gaps = torch.empty(hi - lo, dtype=torch.float64, device=device).exponential_(1.0, generator=_gen(device, seed, c))
        w = torch.cumsum(gaps, 0) + carry
        carry = w[-1].clone()
        out[lo:hi] = w
    return out


def quarter_range_cuda(n: int, dtype: str, seed: int = 0, device="cuda"):
    import torch
    dt = np.dtype(dtype)
    out = torch.empty(n, dtype=_signed_torch_dtype(dtype), device=device)
    for c, lo in enumerate(range(0, n, _CHUNK)):
        hi = min(n, lo + _CHUNK)
        g = _gen(device, seed, c)
        if dt.kind == "f":
            top = float(np.finfo(dt).max) / 4
            u = torch.rand(hi - lo, generator=g, device=device, dtype=torch.float64)
            out[lo:hi] = (u * (2 * top) - top).to(out.dtype)
            continue
        info = np.iinfo(dt)
        a, b = (info.min // 4, info.max // 4) if dt.kind == "i" else (0, info.max // 4)
        if dt.itemsize < 8:
            v = torch.randint(a, b + 1, (hi - lo,), generator=g, device=device, dtype=torch.int64)
        else:
            r = torch.randint(0, 2 ** 62, (hi - lo,), generator=g, device=device, dtype=torch.int64)
            v = (r.to(torch.float64) / float(2 ** 62) * float(b - a)).to(torch.int64) + a
        out[lo:hi] = v.to(out.dtype)
    return out
