"""LTTB bucket averages on the GPU vs the oracle, bit for bit.

Buckets above 32 points take one of two routes on the GPU: an exact integer
sum, used only where no addition of the index-order sum can round, or the
sequential binary64 chain.  Either way the averages must carry the oracle's
bits.  The cases put buckets on both routes, and on each side of the bound
that chooses between them; small buckets (32 points or fewer) cover the
table-mode averages."""
import numpy as np
import pytest

import oracle
from paper_2307_05389_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_means(x, y, n_out, nan):
    import torch
    m = binding.lttb_means(dev(y), n_out, x=dev(x) if x is not None else None, nan=nan)
    torch.cuda.synchronize()
    return m.cpu().numpy()


def same_bits(got, exp):
    """Equal as binary64 bit patterns, except that any NaN matches any NaN."""
    g, e = got.view(np.uint64), exp.view(np.uint64)
    both_nan = np.isnan(got) & np.isnan(exp)
    bad = np.flatnonzero(((g != e) & ~both_nan).reshape(-1))
    return bad


def check(x, y, n_out, nan="propagate"):
    got = gpu_means(x, y, n_out, nan)
    exp = oracle.lttb_means(x, y, n_out, nan=nan)
    assert got.shape == exp.shape
    bad = same_bits(got, exp)
    if bad.size:
        k = int(bad[0])
        raise AssertionError(f"n={len(y)} n_out={n_out} nan={nan}: {bad.size} averages differ, first at bucket "
                             f"{k // 2 + 1} ({'xy'[k % 2]}): got {got.reshape(-1)[k]!r} exp {exp.reshape(-1)[k]!r}")


def bucket(j, n, n_out):
    B = n_out - 2
    return 1 + (j * (n - 2)) // B, 1 + ((j + 1) * (n - 2)) // B


@pytest.mark.parametrize("dtype", ["float32", "float64", "float16", "int16", "uint8", "int64", "uint32"])
@pytest.mark.parametrize("n_out", [1000, 7000, 40, 20000])
def test_means_random_data(dtype, n_out):
    n = 300_007
    y = inputs.random_walk(n, dtype, 5) if np.dtype(dtype).kind == "f" else inputs.quarter_range(n, dtype, 5)
    for nan in (("propagate", "ignore") if np.dtype(dtype).kind == "f" else ("propagate",)):
        check(None, y, n_out, nan)


@pytest.mark.parametrize("x_kind", ["int64", "float64", "float32"])
def test_means_with_x(x_kind):
    n = 200_003
    y = inputs.random_walk(n, "float32", 6)
    if x_kind == "int64":
        x = inputs.geometric_x(n, 6)
    elif x_kind == "float64":
        x = inputs.exponential_x(n, 6)
    else:
        x = np.arange(n, dtype=np.float32) * np.float32(0.25)
    for n_out in (500, 3000):
        check(x, y, n_out)


def test_means_specials_and_quantised_nan():
    n = 100_000
    check(None, inputs.ties_and_specials(n, "float64", 7), 800, "propagate")
    check(None, inputs.ties_and_specials(n, "float64", 7), 800, "ignore")
    check(None, inputs.ties_and_specials(n, "float32", 8), 300, "ignore")
    check(None, inputs.quantised_nan(n, 9), 900, "propagate")
    check(None, inputs.quantised_nan(n, 9), 900, "ignore")
    # table mode (buckets of at most 32 points): warp sums and the sequential fallback
    for nan in ("propagate", "ignore"):
        check(None, inputs.ties_and_specials(n, "float64", 11), 20_000, nan)
        check(None, inputs.quantised_nan(n, 12), 5_000, nan)


def test_means_at_the_exactness_bound():
    """Integer-valued binary64 buckets of c points whose largest value has
    exponent T: the exact route needs T + 1 + ceil(log2 c) <= 53.  Bucket 3
    sits just inside the bound; bucket 5 just outside, where the index-order
    sum really rounds ((2^53 - 1) + 1 + 1 + ... loses the later ones); bucket 7
    mixes 1.0 with the smallest subnormal, bucket 9 has tiny values only, and
    bucket 11 is all zeros of both signs."""
    n, n_out = 4001, 50                       # 48 buckets of 83-84 points
    y = np.zeros(n)
    rng = np.random.default_rng(10)
    lo, hi = bucket(3, n, n_out)
    c = hi - lo
    lg = int(np.ceil(np.log2(c)))
    top = 53 - 1 - lg                          # T + 1 + lg == 53
    y[lo:hi] = rng.integers(-(2 ** top), 2 ** top, size=c).astype(np.float64)
    y[lo] = float(2 ** top + 12345)
    lo, hi = bucket(5, n, n_out)
    y[lo:hi] = 1.0
    y[lo] = float(2 ** 53 - 1)
    lo, hi = bucket(7, n, n_out)
    y[lo:hi] = 1.0
    y[lo + 3] = 5e-324
    lo, hi = bucket(9, n, n_out)
    y[lo:hi] = rng.integers(1, 1000, size=hi - lo) * 5e-324
    lo, hi = bucket(11, n, n_out)
    y[lo:hi] = np.where(rng.random(hi - lo) < 0.5, -0.0, 0.0)
    check(None, y, n_out)
    exp = oracle.lttb_means(None, y, n_out)
    b5 = bucket(5, n, n_out)
    assert exp[4, 1] * (b5[1] - b5[0]) != float(2 ** 53 - 1 + (b5[1] - b5[0] - 1))   # the sum rounded


def test_means_mixed_routes_in_one_warp():
    """A float32 walk where a few scattered buckets hold values of very
    different binary exponents (forced onto the sequential chain) among
    buckets that take the exact route."""
    n, n_out = 500_000, 2000
    y = inputs.random_walk(n, "float32", 12).astype(np.float64)
    rng = np.random.default_rng(12)
    for j in rng.choice(np.arange(1, n_out - 3), size=40, replace=False):
        lo, hi = bucket(int(j), n, n_out)
        y[lo + int(rng.integers(0, hi - lo))] = 1e-30 * rng.standard_normal()
    check(None, y, n_out)
    check(None, y.astype(np.float32), n_out)


def test_means_rejects_undefined_shapes():
    import torch
    y = torch.zeros(10, dtype=torch.float32, device="cuda")
    for n_out in (2, 10, 11):
        with pytest.raises(binding.TsdsError):
            binding.lttb_means(y, n_out)
