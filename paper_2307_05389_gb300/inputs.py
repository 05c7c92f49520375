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

def random_walk_cuda(n: int, dtype="float32", seed: int = 0, device="cuda"):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    steps = torch.randn(n, generator=g, device=device, dtype=torch.float32)
    return torch.cumsum(steps, 0, dtype=torch.float64).to(getattr(torch, dtype))


def geometric_x_cuda(n: int, seed: int = 0, p: float = 0.5, device="cuda"):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    gaps = torch.empty(n, dtype=torch.float32, device=device).geometric_(p, generator=g)
    gaps = gaps.to(torch.int64)
    gaps[0] = 0
    return torch.cumsum(gaps, 0)


def quarter_range_cuda(n: int, dtype: str, seed: int = 0, device="cuda"):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    dt = np.dtype(dtype)
    tdt = getattr(torch, dtype)
    if dt.kind == "f":
        hi = float(np.finfo(dt).max) / 4
        u = torch.rand(n, generator=g, device=device, dtype=torch.float64)
        return (u * (2 * hi) - hi).to(tdt)
    info = np.iinfo(dt)
    lo, hi = (info.min // 4, info.max // 4) if dt.kind == "i" else (0, info.max // 4)
    if dt.itemsize < 8:
        v = torch.randint(lo, hi + 1, (n,), generator=g, device=device, dtype=torch.int64)
        return v.to(tdt) if dt.kind == "i" or dt.itemsize < 8 else v
    # 64-bit: draw 63 random bits and scale into [lo, hi] (uniform up to 2^-63 bias)
    r = torch.randint(0, 2 ** 62, (n,), generator=g, device=device, dtype=torch.int64)
    span = hi - lo
    v = (r.to(torch.float64) / float(2 ** 62) * float(span)).to(torch.int64)
    if dt.kind == "i":
        return v + lo
    return v.view(torch.uint64) if hasattr(torch, "uint64") else v
