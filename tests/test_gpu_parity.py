"""CUDA path vs the CPU oracle, index for index, on seeded inputs.

Sizes span many 64 KB windows (so bins are cut across windows and rejoined)
and end in ragged tails; cases cover all eleven dtypes, both NaN modes,
no x / integer x / floating x, unaligned starts, empty bins and the
degenerate shapes (n = 0, 1, n_out >= n, one bin, one point per bin).
The bar is bit-exact equality of the int64 index lists."""
import numpy as np
import pytest

import oracle
from paper_2307_05389_gb300 import inputs

from gpu_util import call, run

pytestmark = pytest.mark.gpu

INT_DTYPES = ["int8", "int16", "int32", "int64", "uint8", "uint16", "uint32", "uint64"]
FLOAT_DTYPES = ["float16", "float32", "float64"]
ALL_DTYPES = INT_DTYPES + FLOAT_DTYPES


def check(algo, x, y, n_out, nan="propagate", ratio=4, **kw):
    got = run(algo, x, y, n_out, nan, ratio, **kw)
    exp = oracle.downsample(algo, x, y, n_out, nan=nan, minmax_ratio=ratio)
    if not np.array_equal(got, exp):
        d = np.flatnonzero(got[:min(len(got), len(exp))] != exp[:min(len(got), len(exp))])
        first = int(d[0]) if d.size else min(len(got), len(exp))
        raise AssertionError(f"{algo} n={len(y)} n_out={n_out} nan={nan}: {len(got)} vs {len(exp)} indices, "
                             f"first difference at {first}: got {got[first:first + 4]} exp {exp[first:first + 4]}")


def series(dtype, n, seed, kind="walk"):
    if kind == "walk":
        if np.dtype(dtype).kind == "f":
            return inputs.random_walk(n, dtype, seed)
        return inputs.quarter_range(n, dtype, seed)
    if kind == "ties":
        return inputs.ties_and_specials(n, dtype, seed)
    raise ValueError(kind)


@pytest.mark.parametrize("dtype", ALL_DTYPES)
@pytest.mark.parametrize("algo", ["minmax", "m4"])
def test_binned_dtypes_no_x(dtype, algo):
    n = 1_000_003 if np.dtype(dtype).itemsize == 1 else 300_007
    for kind in ("walk", "ties"):
        y = series(dtype, n, seed=11, kind=kind)
        for n_out in (4, 200, 2000, 40_000):
            for nan in (("propagate", "ignore") if np.dtype(dtype).kind == "f" else ("propagate",)):
                check(algo, None, y, n_out, nan)


@pytest.mark.parametrize("x_dtype", ["int64", "float64", "int32", "uint64", "float32", "int16", "float16", "uint8"])
@pytest.mark.parametrize("algo", ["minmax", "m4"])
def test_binned_with_x(x_dtype, algo):
    n = 250_001
    y = inputs.random_walk(n, "float32", seed=3)
    if x_dtype in ("int16", "float16", "uint8"):
        # narrow x: sorted values with long runs of equal x (many empty bins)
        rng = np.random.default_rng(5)
        hi = 250 if x_dtype == "uint8" else 2000
        x = np.sort(rng.integers(0, hi, n)).astype(x_dtype)
    elif np.dtype(x_dtype).kind == "f":
        x = inputs.exponential_x(n, seed=4).astype(x_dtype)
        x = np.maximum.accumulate(x)
    else:
        x = inputs.geometric_x(n, seed=4).astype(x_dtype)
        if x_dtype == "uint64":
            x = x + np.uint64(2 ** 63)
    for n_out in (4, 400, 4000, 100_000):
        check(algo, x, y, n_out)


def test_equal_x_equals_no_x_on_gpu():
    y = inputs.random_walk(400_000, "float32", seed=8)
    for algo in ("minmax", "m4"):
        ref = run(algo, None, y, 2000)
        for xd in ("int64", "float64", "uint32"):
            np.testing.assert_array_equal(run(algo, np.arange(len(y)).astype(xd), y, 2000), ref)


@pytest.mark.parametrize("dtype", ["int8", "int16", "float16", "float32", "float64", "uint64"])
@pytest.mark.parametrize("offset", [1, 3, 7])
def test_unaligned_start(dtype, offset):
    y = series(dtype, 123_457, seed=2)
    for algo in ("minmax", "m4"):
        check(algo, None, y, 1000, offset=offset)


@pytest.mark.parametrize("dtype", FLOAT_DTYPES)
@pytest.mark.parametrize("nan", ["propagate", "ignore"])
def test_nan_rich(dtype, nan):
    rng = np.random.default_rng(9)
    y = inputs.random_walk(200_000, dtype, seed=9)
    y[rng.choice(len(y), 3000, replace=False)] = np.nan
    y[50_000:120_000] = np.nan                     # bins that are all NaN
    y[rng.choice(len(y), 500, replace=False)] = np.inf
    y[rng.choice(len(y), 500, replace=False)] = -np.inf
    for algo in ("minmax", "m4"):
        for n_out in (8, 100, 3000):
            check(algo, None, y, n_out, nan)


@pytest.mark.parametrize("algo", ["minmax", "m4", "lttb", "minmaxlttb"])
def test_degenerate_sizes(algo):
    for n in (0, 1, 2, 3, 4, 5, 7, 8, 9, 17, 33, 100):
        y = inputs.random_walk(n, "float32", seed=n) if n else np.zeros(0, np.float32)
        for n_out in (4, 8, 12, 16, 36, 100, 200):
            check(algo, None, y, n_out)


def test_single_bin_and_one_point_bins():
    y = inputs.random_walk(3_000_001, "float32", seed=1)
    check("minmax", None, y, 2)          # one bin over 3M points (many windows)
    check("m4", None, y, 4)
    y = inputs.random_walk(20_001, "float64", seed=2)
    check("minmax", None, y, 20_000)     # bins of one or two points
    check("m4", None, y, 20_000)


def test_constant_and_monotone():
    for dtype in ("int32", "float32", "uint8"):
        y = np.full(300_000, 7, dtype=dtype)
        check("minmax", None, y, 100)
        check("m4", None, y, 100)
    y = np.arange(300_000, dtype=np.float32)
    check("minmax", None, y, 100)
    check("minmax", None, y[::-1].copy(), 100)


@pytest.mark.parametrize("nb", [4095, 4096, 4097, 4096 + 31, 4096 + 33, 65 * 32, 20_000])
@pytest.mark.parametrize("x_kind", ["int64", "float64", "gap", "runs"])
def test_many_x_bins_two_level_edges(nb, x_kind):
    """From 4096 x-space bins of at most 512 points on, a single series' edges come from a
    coarse search for every 32nd edge and a fine search between coarse neighbours: bin counts
    around that threshold and around group ends, with uniform, gapped and run-heavy x."""
    n = 200_003
    y = inputs.random_walk(n, "float32", seed=21)
    if x_kind == "int64":
        x = inputs.geometric_x(n, seed=22)
    elif x_kind == "float64":
        x = inputs.exponential_x(n, seed=22)
    elif x_kind == "gap":
        x = np.concatenate([np.arange(n // 3), np.arange(n - n // 3) + 10 ** 12]).astype(np.int64)
    else:
        x = np.sort(np.random.default_rng(23).integers(0, 3000, n)).astype(np.int64)
    check("minmax", x, y, 2 * nb)
    check("m4", x, y, 4 * nb)


def test_x_all_equal_and_gaps():
    n = 100_000
    y = inputs.random_walk(n, "float32", seed=5)
    check("minmax", np.zeros(n, np.int64), y, 100)       # one non-empty bin
    x = np.concatenate([np.arange(n // 2), np.arange(n // 2) + 10 ** 9]).astype(np.int64)
    check("m4", x, y, 400)                               # a huge gap: most bins empty


@pytest.mark.parametrize("dtype", ["float32", "float64", "int16", "uint8", "int64", "float16"])
@pytest.mark.parametrize("nan", ["propagate", "ignore"])
def test_lttb(dtype, nan):
    n = 60_001
    y = series(dtype, n, seed=21)
    if np.dtype(dtype).kind == "f":
        y[::997] = np.nan
    for n_out in (3, 4, 100, 1000, 30_000):
        check("lttb", None, y, n_out, nan)


@pytest.mark.parametrize("x_dtype", ["int64", "float64", "float32"])
def test_lttb_with_x(x_dtype):
    n = 40_000
    y = inputs.random_walk(n, "float32", seed=22)
    x = inputs.exponential_x(n, seed=23).astype(x_dtype) if x_dtype != "int64" else inputs.geometric_x(n, seed=23)
    for n_out in (3, 500, 5000):
        check("lttb", x, y, n_out)


@pytest.mark.parametrize("ratio", [1, 2, 4, 30])
@pytest.mark.parametrize("nan", ["propagate", "ignore"])
def test_minmaxlttb(ratio, nan):
    y = inputs.quantised_nan(156_250, seed=4)
    for n_out in (3, 100, 4000):
        check("minmaxlttb", None, y, n_out, nan, ratio)
    x = inputs.geometric_x(len(y), seed=6)
    check("minmaxlttb", x, y, 1000, nan, ratio)


@pytest.mark.parametrize("n_out", [3, 60, 2000, 9000])
def test_lttb_filter_stress(n_out):
    """Inputs chosen against the FP32 pre-filter of the LTTB chain: exact area
    ties (small integers), near-collinear points, timestamps ~1e15 (FP32 cannot
    resolve them), magnitudes beyond its accepted range, and both chain modes
    (n_out 9000 gives buckets of <= 32 points: the transition table)."""
    rng = np.random.default_rng(51)
    n = 40_000
    cases = []
    cases.append((None, rng.integers(-3, 4, n).astype(np.float64)))                    # many exact ties
    t = np.arange(n, dtype=np.float64)
    cases.append((None, 2.5 * t + 1e-9 * rng.standard_normal(n)))                       # near-collinear
    cases.append((1e15 + np.cumsum(rng.integers(1, 5, n)).astype(np.float64),
                  inputs.random_walk(n, "float64", seed=52)))                           # huge x, fine gaps
    cases.append((None, inputs.random_walk(n, "float64", seed=53) * 1e25))              # beyond the filter range
    cases.append((None, inputs.random_walk(n, "float64", seed=54) * 1e-25))             # tiny magnitudes
    y = inputs.random_walk(n, "float64", seed=55)
    y[rng.choice(n, 50, replace=False)] = np.inf
    cases.append((None, y))                                                             # infinities
    for x, y in cases:
        check("lttb", x, y, n_out)
        check("lttb", x, y, n_out, "ignore")


def test_config1_shape_all_algorithms():
    y = inputs.random_walk(1_000_000, "float32", seed=0)
    for algo in ("minmax", "m4", "lttb", "minmaxlttb"):
        check(algo, None, y, 1000)


def test_repeatable_and_stream_ordered():
    import torch
    y = inputs.random_walk(500_000, "float32", seed=12)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = run("m4", None, y, 4000, stream=s)
        b = run("m4", None, y, 4000, stream=s)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, oracle.m4(None, y, 4000))


def test_invalid_arguments_on_gpu():
    y = inputs.random_walk(1000, "float32", seed=0)
    assert call("minmax", None, y, 5)[0] == 1
    assert call("m4", None, y, 6)[0] == 1
    assert call("lttb", None, y, 2)[0] == 1
    assert call("minmaxlttb", None, y, 10, ratio=0)[0] == 1


def test_bounded_wait_reports_timeout_and_context_survives():
    """Failure detection without a fault: a barrier wait nothing satisfies
    gives up after its bound and reports TSDS_ETIMEOUT; later calls work."""
    import torch
    from paper_2307_05389_gb300 import binding
    lib = binding.load()
    assert lib.tsds_check_wait_timeout(2000, None) == 4          # TSDS_ETIMEOUT
    y = inputs.random_walk(100_000, "float32", seed=90)
    check("minmax", None, y, 100)
    torch.cuda.synchronize()


@pytest.mark.parametrize("n", [8191, 65_537, 400_003, 2_000_001])
@pytest.mark.parametrize("offset", [0, 3])
def test_ring_window_and_chunk_boundaries(n, offset):
    """Sizes around the window / 4 KB chunk structure of the streaming ring,
    bins far smaller and far larger than a chunk, unaligned starts."""
    for dtype in ("float32", "int8", "float64"):
        y = series(dtype, n, seed=n % 97)
        for n_out in (2, 8, 1000, n // 3 - (n // 3) % 4):
            if n_out >= 2:
                check("minmax", None, y, n_out, offset=offset)
                if n_out % 4 == 0:
                    check("m4", None, y, n_out, offset=offset)


@pytest.fixture
def stream_variant():
    """Forces one kernel variant of the streaming pass for a test, then restores."""
    from paper_2307_05389_gb300 import binding
    prev = []

    def force(v):
        prev.append(binding.tsds_stream_variant(v))
    yield force
    if prev:
        binding.tsds_stream_variant(prev[0])


@pytest.mark.parametrize("variant", ["ring", "ldg", "seg", "grp"])
@pytest.mark.parametrize("dtype", ALL_DTYPES)
def test_each_stream_variant(variant, dtype, stream_variant):
    """Each variant on its own over bins far below and far above the automatic
    threshold, with ties, unaligned starts and both NaN modes."""
    stream_variant(variant)
    n = 700_001 if np.dtype(dtype).itemsize <= 2 else 260_003
    for kind in ("walk", "ties"):
        y = series(dtype, n, seed=31, kind=kind)
        for n_out in (4, 40, 4000, 60_000):
            for nan in (("propagate", "ignore") if np.dtype(dtype).kind == "f" else ("propagate",)):
                check("minmax", None, y, n_out, nan, offset=1 if kind == "ties" else 0)
                check("m4", None, y, n_out, nan)


@pytest.mark.parametrize("variant", ["ring", "ldg", "seg", "grp"])
def test_each_variant_with_x_and_lttb_preselection(variant, stream_variant):
    stream_variant(variant)
    y = inputs.quantised_nan(300_000, seed=33)
    x = inputs.geometric_x(len(y), seed=34)
    for n_out in (8, 1000):
        check("minmax", x, y, n_out, "ignore")
        check("minmaxlttb", x, y, n_out, "propagate", 4)


@pytest.mark.parametrize("variant", ["seg", "grp"])
@pytest.mark.parametrize("dtype", ["float32", "int8", "uint16", "float16", "int32", "float64", "int64", "uint64"])
@pytest.mark.parametrize("nan", ["propagate", "ignore"])
def test_segmented_tiny_and_mixed_bins(variant, dtype, nan, stream_variant):
    """The segmented and lane-group variants where bins are one to a few
    elements (many bin starts per 512-byte sub-step, several refills of the
    prefetched starts; lane groups of one lane), around the sub-step size, and
    with x making empty bins, long runs of equal bin starts and bins far above
    the lane-group size limit (the register-streaming pass takes those)."""
    stream_variant(variant)
    rng = np.random.default_rng(61)
    n = 300_001
    y = series(dtype, n, seed=62, kind="ties")
    if np.dtype(dtype).kind == "f":
        y[rng.choice(n, 400, replace=False)] = np.nan
        y[1000:1700] = np.nan
    for n_out in (n // 2 - (n // 2) % 4, n // 5 - (n // 5) % 4, 4 * (n // 130), 4 * (n // 1100)):
        check("minmax", None, y, n_out, nan, offset=3)
        check("m4", None, y, n_out, nan)
    # x with clusters and gaps: runs of empty bins (equal bin starts)
    x = np.sort(np.concatenate([rng.integers(0, 1000, n // 2), rng.integers(10 ** 6, 10 ** 6 + 50, n - n // 2)]))
    for n_out in (400, 4000, 40_000):
        check("minmax", x.astype(np.int64), y, n_out, nan)
        check("m4", x.astype(np.int64), y, n_out, nan)


@pytest.mark.parametrize("x_dtype", [None, "int64", "float64", "uint8", "float16", "int32"])
def test_everynth(x_dtype):
    """EveryNth: index-space and x-space bins, a single bin, the tiled emit
    (>= 4096 bins), n_out >= n, n = 0, and x with long runs of equal values
    (empty bins)."""
    n = 300_007
    y = inputs.random_walk(n, "float32", 7)
    if x_dtype is None:
        x = None
    elif x_dtype in ("uint8", "float16"):
        x = np.sort(np.random.default_rng(7).integers(0, 200, n)).astype(x_dtype)
    elif x_dtype == "float64":
        x = inputs.exponential_x(n, 7)
    else:
        x = inputs.geometric_x(n, 7).astype(x_dtype) if x_dtype == "int64" else \
            np.sort(np.random.default_rng(7).integers(-10**9, 10**9, n)).astype(np.int32)
    for n_out in (1, 7, 2000, 40_000):
        check("everynth", x, y, n_out)
    check("everynth", None if x is None else x[:500], y[:500], 500)
    check("everynth", None if x is None else x[:500], y[:500], 501)
    check("everynth", None if x is None else x[:0], y[:0], 10)


@pytest.mark.parametrize("algo", ["minmax", "m4"])
@pytest.mark.parametrize("xkind", ["none", "int64_gaps", "float64_skewed"])
def test_bin_ranges_concatenate_to_the_whole_call(algo, xkind):
    """tsds_minmax_bins / tsds_m4_bins over consecutive bin ranges (the split a set of ranks
    uses, shard.shard_bins) concatenate to the single call's output and the oracle's.  The
    skewed x puts most points in a few bins, far above the lane-group size limit."""
    from paper_2307_05389_gb300 import binding, shard
    import torch
    rng = np.random.default_rng(71)
    n = 600_001
    y = inputs.random_walk(n, "float32", seed=72)
    y[rng.choice(n, 50, replace=False)] = np.nan
    if xkind == "none":
        x = None
    elif xkind == "int64_gaps":
        x = np.concatenate([[0], np.cumsum(rng.choice([0, 1, 2, 40], size=n - 1))]).astype(np.int64)
    else:
        x = np.sort(np.concatenate([rng.uniform(0, 1, n - 1000), rng.uniform(0, 1e6, 1000)]))
    dy = torch.from_numpy(y).cuda()
    dx = torch.from_numpy(x).cuda() if x is not None else None
    per = 2 if algo == "minmax" else 4
    for n_out in (per * 7, per * 3000, per * 60_000):
        for nan in ("propagate", "ignore"):
            whole = oracle.downsample(algo, x, y, n_out, nan)
            nb = n_out // per
            for world in (1, 3, 8):
                parts = [binding.downsample_bins(algo, dy, n_out, *shard.shard_bins(nb, r, world), x=dx, nan=nan)
                         for r in range(world)]
                got = torch.cat(parts).cpu().numpy()
                np.testing.assert_array_equal(got, whole, err_msg=f"{algo} n_out={n_out} world={world} {nan}")
            assert binding.downsample_bins(algo, dy, n_out, 3, 3, x=dx, nan=nan).numel() == 0
