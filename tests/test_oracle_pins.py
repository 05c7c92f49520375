"""Pins the CPU oracle to things other than itself (CPU only).

Each check uses an independent route to the answer: hand-derived fixtures,
brute-force enumeration with exact integers or rationals, numpy's own argmin /
argmax / nanargmin / nanargmax, numpy's float16 decoding, and identities the
paper states (equal x gives the same output as no x, uint/int and f16/f32
consistency, Section 2.2 unit tests and Section 2.1.2 mappings).
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from golden_util import all_cases
from paper_2307_05389_gb300 import inputs

INT_DTYPES = ["int8", "int16", "int32", "int64", "uint8", "uint16", "uint32", "uint64"]
FLOAT_DTYPES = ["float16", "float32", "float64"]


# ----------------------------------------------------------------------------- brute force helpers

def bf_edges_index(n, nb):
    """Bin i starts at the least j with j*nb >= i*(n-1): scan every j."""
    s = []
    for i in range(nb):
        j = 0
        while j * nb < i * (n - 1):
            j += 1
        s.append(j)
    return s + [n]


def bf_edges_int_x(xs, nb):
    """Least j with (x_j - x_0)*nb >= i*(x_last - x_0), scanning j, exact Python ints."""
    n = len(xs)
    span = xs[-1] - xs[0]
    s = []
    for i in range(nb):
        j = 0
        while (xs[j] - xs[0]) * nb < i * span:
            j += 1
        s.append(j)
    return s + [n]


def np_argminmax(y, lo, hi, nan):
    seg = y[lo:hi]
    if nan == "propagate":
        return lo + int(np.argmin(seg)), lo + int(np.argmax(seg))
    if seg.dtype.kind != "f":
        return lo + int(np.argmin(seg)), lo + int(np.argmax(seg))
    # numpy's nanargmin/nanargmax substitute +-inf for NaN and can return a
    # NaN's index when the extremum is itself infinite, so mask NaNs instead.
    keep = np.flatnonzero(~np.isnan(seg))
    if keep.size == 0:
        return lo, lo
    vals = seg[keep]
    return lo + int(keep[np.argmin(vals)]), lo + int(keep[np.argmax(vals)])


def bf_binned(y, s, per_bin, nan):
    out = []
    for b in range(len(s) - 1):
        lo, hi = s[b], s[b + 1]
        if lo >= hi:
            continue
        mn, mx = np_argminmax(y, lo, hi, nan)
        sel = {mn, mx} if per_bin == 2 else {lo, mn, mx, hi - 1}
        out += sorted(sel)
    return np.array(out, dtype=np.int64)


def bf_lttb_exact(px, py, n_out):
    """LTTB in exact rationals with the shoelace form of the doubled area.

    Returns the picks and the smallest relative gap between the winning area
    and the best loser over all steps (0 when an exact tie decided a step)."""
    m = len(py)
    if n_out >= m:
        return list(range(m)), float("inf")
    B = n_out - 2

    def start(j):
        return 1 + (j * (m - 2)) // B

    a = 0
    out = [0]
    gap = float("inf")
    for j in range(B):
        lo, hi = start(j), start(j + 1)
        if j == B - 1:
            xc, yc = px[m - 1], py[m - 1]
        else:
            nlo, nhi = hi, start(j + 2)
            xc = sum(px[nlo:nhi], Fraction(0)) / (nhi - nlo)
            yc = sum(py[nlo:nhi], Fraction(0)) / (nhi - nlo)
        areas = []
        for b in range(lo, hi):
            # shoelace: x_a(y_b - y_c) + x_b(y_c - y_a) + x_c(y_a - y_b)
            areas.append(abs(px[a] * (py[b] - yc) + px[b] * (yc - py[a]) + xc * (py[a] - py[b])))
        best = max(areas)
        k = areas.index(best)
        rest = [v for i, v in enumerate(areas) if i != k]
        if rest:
            second = max(rest)
            scale = max(best, Fraction(1, 10 ** 30))
            gap = min(gap, float((best - second) / scale))
        a = lo + k
        out.append(a)
    out.append(m - 1)
    return out, gap


def frac_list(v):
    return [Fraction(float(t)) for t in v]


# ----------------------------------------------------------------------------- golden fixtures

@pytest.mark.parametrize("case", all_cases(), ids=lambda c: c["id"])
def test_golden_hand_derived(case):
    got = oracle.downsample(case["algo"], case["x"], case["y"], case["n_out"], nan=case["nan"],
                            minmax_ratio=case["minmax_ratio"])
    np.testing.assert_array_equal(got, case["expected"], err_msg=case["derivation"])


# ----------------------------------------------------------------------------- float16 decoding

def test_f16_decode_matches_numpy_for_every_bit_pattern():
    bits = np.arange(1 << 16, dtype=np.uint16)
    ref = bits.view(np.float16).astype(np.float64)
    got = np.array([oracle.f16_to_f64(int(b)) for b in bits])
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan], ref[~nan])
    assert np.array_equal(np.signbit(got[~nan]), np.signbit(ref[~nan]))


# ----------------------------------------------------------------------------- bins

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13, 31, 40])
def test_index_edges_brute_force(n):
    for nb in range(1, n + 3):
        assert list(oracle.bin_edges(None, n, nb)) == bf_edges_index(n, nb)


@pytest.mark.parametrize("dtype", INT_DTYPES)
def test_int_x_edges_brute_force(dtype):
    rng = np.random.default_rng(7)
    info = np.iinfo(dtype)
    for trial in range(12):
        n = int(rng.integers(2, 40))
        # sorted values spanning a wide slice of the dtype range, with repeats
        lo = info.min if trial % 2 else info.min // 3 + 5
        hi = info.max if trial % 3 else info.max // 3
        v = np.sort(rng.integers(lo, hi, size=n, endpoint=True, dtype=dtype))
        if trial % 4 == 0:
            v[n // 2:] = v[n // 2]                     # long run of equal x
        xs = [int(t) for t in v]
        for nb in (1, 2, 3, max(1, n // 2), n, n + 1):
            got = list(oracle.bin_edges(v, n, nb))
            assert got == bf_edges_int_x(xs, nb), (dtype, n, nb)


@pytest.mark.parametrize("x_dtype", ["float64", "float32", "float16"])
def test_float_x_edges_agree_with_exact_rule_on_integer_valued_x(x_dtype):
    """For integer-valued x the binary64 edge formula meets the exact rule:
    every quotient i*span/nb is either an integer or at least 1/nb away from
    one, far more than the rounding error, so lower_bound cannot differ."""
    rng = np.random.default_rng(11)
    for trial in range(20):
        n = int(rng.integers(2, 60))
        xs = np.sort(rng.integers(-1000, 1000, size=n))
        xf = xs.astype(x_dtype)
        for nb in (1, 2, 3, 7, n, n + 5):
            assert list(oracle.bin_edges(xf, n, nb)) == bf_edges_int_x([int(t) for t in xs], nb)


def test_float_x_edges_only_differ_from_exact_rule_at_near_ties():
    """Random binary64 x: the edges equal the exact-rational rule except where
    some x lies within a few ulps of the exact edge value."""
    rng = np.random.default_rng(12)
    for trial in range(40):
        n = int(rng.integers(3, 80))
        x = np.sort(rng.uniform(-1e3, 1e3, n))
        fx = frac_list(x)
        span = fx[-1] - fx[0]
        for nb in (2, 3, 5, 11):
            got = oracle.bin_edges(x, n, nb)
            for i in range(1, nb):
                e = fx[0] + span * i / nb
                exact = next(j for j in range(n) if fx[j] >= e)
                if got[i] != exact:
                    lo, hi = sorted((got[i], exact))
                    tol = Fraction(abs(float(e))) * Fraction(2) ** -50 + Fraction(2) ** -1000
                    assert all(abs(fx[j] - e) <= tol for j in range(lo, hi)), (trial, nb, i)


@pytest.mark.parametrize("x_dtype", ["int64", "uint64", "int8", "uint16", "float16", "float32", "float64"])
def test_edges_never_decrease_with_the_bin_index(x_dtype):
    """Bin starts are non-decreasing in the bin index under both the exact integer rule and the
    rounded binary64 rule (each operation is monotone), for sorted x of every kind: long runs of
    equal values, spans near the dtype's limits, rounding-heavy float steps.  So edge i lies
    between the edges of any two bin indices around it, which lets a search for it start from
    coarser edges."""
    rng = np.random.default_rng(61)
    dt = np.dtype(x_dtype)
    for trial in range(6):
        n = int(rng.integers(2, 5000))
        if dt.kind == "f":
            hi = float(np.finfo(dt).max) / (4 if trial % 2 else 1e6)
            x = np.sort(rng.uniform(-hi, hi, n)).astype(dt)
            if trial == 5:
                x = np.sort(rng.integers(0, 7, n)).astype(dt)     # runs of equal values
        else:
            info = np.iinfo(dt)
            lo, top = (int(info.min), int(info.max)) if trial % 2 else (0, int(info.max) // 3)
            x = np.sort(rng.integers(lo, top, n, endpoint=True, dtype=dt))
            if trial == 5:
                x = np.sort(rng.integers(lo, lo + 5, n, dtype=dt))
        x = np.sort(x)
        for nb in (1, 2, 31, 32, 33, 1000, 5000):
            e = oracle.bin_edges(x, n, nb)
            assert e[0] == 0 and e[-1] == n
            assert np.all(np.diff(e) >= 0), f"{x_dtype} n={n} nb={nb}"


@pytest.mark.parametrize("x_dtype", ["int64", "int32", "uint32", "uint64", "float64", "float32"])
def test_equal_x_matches_no_x_edges(x_dtype):
    """Section 2.2: an equally sampled x gives the same output as no x."""
    for n in (2, 3, 10, 97, 1000, 12345):
        x = np.arange(n).astype(x_dtype)
        for nb in (1, 2, 3, 50, 499):
            np.testing.assert_array_equal(oracle.bin_edges(x, n, nb), oracle.bin_edges(None, n, nb))


# ----------------------------------------------------------------------------- argmin / argmax

@pytest.mark.parametrize("dtype", INT_DTYPES + FLOAT_DTYPES)
@pytest.mark.parametrize("nan", ["propagate", "ignore"])
def test_argminmax_matches_numpy(dtype, nan):
    rng = np.random.default_rng(3)
    y = inputs.ties_and_specials(400, dtype, seed=5)
    for _ in range(150):
        lo = int(rng.integers(0, 399))
        hi = int(rng.integers(lo + 1, 401))
        assert oracle.argminmax(y, lo, hi, nan) == np_argminmax(y, lo, hi, nan), (lo, hi)


def test_argminmax_all_nan_bin():
    y = np.array([np.nan] * 5, dtype=np.float32)
    assert oracle.argminmax(y, 1, 4, "ignore") == (1, 1)
    assert oracle.argminmax(y, 1, 4, "propagate") == (1, 1)


# ----------------------------------------------------------------------------- MinMax / M4

@pytest.mark.parametrize("dtype", INT_DTYPES + FLOAT_DTYPES)
@pytest.mark.parametrize("nan", ["propagate", "ignore"])
def test_minmax_m4_brute_force_tiny(dtype, nan):
    rng = np.random.default_rng(21)
    for trial in range(30):
        n = int(rng.integers(1, 30))
        y = inputs.ties_and_specials(n, dtype, seed=trial)
        for n_out in (2, 4, 6, 8, 12, 28, 32):
            got = oracle.minmax(None, y, n_out, nan)
            exp = np.arange(n) if n_out >= n else bf_binned(y, bf_edges_index(n, n_out // 2), 2, nan)
            np.testing.assert_array_equal(got, exp)
            if n_out % 4 == 0:
                got = oracle.m4(None, y, n_out, nan)
                exp = np.arange(n) if n_out >= n else bf_binned(y, bf_edges_index(n, n_out // 4), 4, nan)
                np.testing.assert_array_equal(got, exp)


@pytest.mark.parametrize("x_dtype", ["int64", "uint8", "int16"])
def test_minmax_m4_brute_force_int_x(x_dtype):
    rng = np.random.default_rng(22)
    info = np.iinfo(x_dtype)
    for trial in range(25):
        n = int(rng.integers(2, 40))
        x = np.sort(rng.integers(max(info.min, -100), min(info.max, 100), size=n, endpoint=True, dtype=x_dtype))
        y = rng.standard_normal(n).astype(np.float32)
        xs = [int(t) for t in x]
        for n_out in (4, 8, 12):
            if n_out >= n:
                continue
            np.testing.assert_array_equal(oracle.minmax(x, y, n_out), bf_binned(y, bf_edges_int_x(xs, n_out // 2), 2, "propagate"))
            np.testing.assert_array_equal(oracle.m4(x, y, n_out), bf_binned(y, bf_edges_int_x(xs, n_out // 4), 4, "propagate"))


@pytest.mark.parametrize("dtype", ["int8", "uint16", "float32", "float64"])
@pytest.mark.parametrize("nan", ["propagate", "ignore"])
def test_binned_range_brute_force_tiny(dtype, nan):
    """Bins [b0, b1) of the whole-series layout select exactly what brute force
    selects in those bins (edges by exhaustive scan, extrema by numpy)."""
    rng = np.random.default_rng(23)
    for trial in range(25):
        n = int(rng.integers(3, 40))
        y = inputs.ties_and_specials(n, dtype, seed=100 + trial)
        for algo, per in (("minmax", 2), ("m4", 4)):
            for nb in (1, 2, 3, 5, 9):
                n_out = nb * per
                if n_out >= n:
                    continue
                s = bf_edges_index(n, nb)
                b0 = int(rng.integers(0, nb + 1))
                b1 = int(rng.integers(b0, nb + 1))
                got = oracle.binned_range(algo, None, y, n_out, b0, b1, nan)
                np.testing.assert_array_equal(got, bf_binned(y, s[b0:b1 + 1], per, nan))


@pytest.mark.parametrize("x_dtype", ["int64", "int16", "float64"])
def test_binned_range_concatenation_is_the_whole_output(x_dtype):
    """Cutting the bins anywhere (also inside runs of equal x, where bins are
    empty) and concatenating the parts in bin order gives the whole output."""
    rng = np.random.default_rng(24)
    for trial in range(20):
        n = int(rng.integers(50, 3000))
        gaps = rng.choice([0, 0, 1, 2, 40], size=n - 1)
        x = np.concatenate([[0], np.cumsum(gaps)]).astype(x_dtype)
        y = inputs.random_walk(n, "float32", seed=200 + trial)
        y[rng.integers(0, n, 3)] = np.nan
        for algo, per in (("minmax", 2), ("m4", 4)):
            for nan in ("propagate", "ignore"):
                n_out = per * int(rng.integers(1, max(2, n // (2 * per))))
                whole = oracle.downsample(algo, x, y, n_out, nan)
                nb = n_out // per
                cuts = sorted({0, nb, *rng.integers(0, nb + 1, size=3).tolist()})
                parts = [oracle.binned_range(algo, x, y, n_out, a, b, nan) for a, b in zip(cuts, cuts[1:])]
                np.testing.assert_array_equal(np.concatenate(parts), whole)
                np.testing.assert_array_equal(oracle.binned_threads(algo, x, y, n_out, nan, threads=5), whole)


def test_binned_range_rejects_undefined_ranges():
    y = np.arange(100, dtype=np.float32)
    for args in (("minmax", None, y, 10, -1, 3), ("minmax", None, y, 10, 3, 2), ("minmax", None, y, 10, 0, 6),
                 ("m4", None, y, 10, 0, 1), ("minmax", None, y, 100, 0, 1)):
        with pytest.raises(oracle.OracleError):
            oracle.binned_range(*args)


def check_invariants(idx, n, n_out, algo):
    assert idx.dtype == np.int64
    assert np.all(np.diff(idx) > 0), "strictly increasing and unique"
    if n_out >= n:
        np.testing.assert_array_equal(idx, np.arange(n))
        return
    assert len(idx) <= n_out
    if n > 0 and algo in ("m4", "lttb", "minmaxlttb"):
        assert idx[0] == 0 and idx[-1] == n - 1
    if algo in ("lttb", "minmaxlttb"):
        assert len(idx) <= n_out


@pytest.mark.parametrize("algo", ["minmax", "m4"])
def test_picks_are_true_extrema_random_walk(algo):
    y = inputs.random_walk(50_000, "float32", seed=0)
    n_out = 1000
    idx = oracle.downsample(algo, None, y, n_out)
    check_invariants(idx, len(y), n_out, algo)
    per = 2 if algo == "minmax" else 4
    s = bf_edges_index(len(y), n_out // per) if len(y) < 100 else list(oracle.bin_edges(None, len(y), n_out // per))
    # every bin's true extrema (lowest index among ties) are in the output
    sel = set(idx.tolist())
    for b in range(len(s) - 1):
        mn, mx = np_argminmax(y, s[b], s[b + 1], "propagate")
        assert mn in sel and mx in sel


def test_index_edges_closed_form_large():
    n, nb = 10 ** 9 + 7, 1000
    s = oracle.bin_edges(None, n, nb)
    for i in range(nb):
        assert s[i] == -((-i * (n - 1)) // nb)


def test_cross_dtype_uint_vs_int_mapping():
    """Section 2.1.2: a uint compares like the int obtained by flipping its top bit."""
    rng = np.random.default_rng(5)
    for bits in (8, 16, 32, 64):
        u = np.dtype(f"uint{bits}")
        s = np.dtype(f"int{bits}")
        v = rng.integers(0, np.iinfo(u).max, size=3000, dtype=u, endpoint=True)
        v[::7] = v[3]                                     # ties
        flipped = (v ^ (u.type(1) << u.type(bits - 1))).view(s)
        for algo in ("minmax", "m4"):
            np.testing.assert_array_equal(oracle.downsample(algo, None, v, 200), oracle.downsample(algo, None, flipped, 200))


def test_cross_dtype_f16_vs_f32_and_int_widths():
    rng = np.random.default_rng(6)
    v = rng.integers(-100, 100, size=5000)
    ref = oracle.minmax(None, v.astype(np.int8), 300)
    for dt in ("int16", "int32", "int64", "float16", "float32", "float64"):
        np.testing.assert_array_equal(oracle.minmax(None, v.astype(dt), 300), ref)
        np.testing.assert_array_equal(oracle.m4(None, v.astype(dt), 300), oracle.m4(None, v.astype(np.int8), 300))
    h = inputs.random_walk(4000, "float16", seed=1)
    np.testing.assert_array_equal(oracle.minmax(None, h, 100, "ignore"), oracle.minmax(None, h.astype(np.float32), 100, "ignore"))


@pytest.mark.parametrize("algo", ["minmax", "m4"])
def test_equal_x_matches_no_x_outputs(algo):
    y = inputs.random_walk(20_000, "float64", seed=2)
    ref = oracle.downsample(algo, None, y, 400)
    for x_dtype in ("int64", "float64", "uint32"):
        np.testing.assert_array_equal(oracle.downsample(algo, np.arange(len(y)).astype(x_dtype), y, 400), ref)


def test_monotone_and_constant_closed_forms():
    n, n_out = 1000, 20
    s = bf_edges_index(n, n_out // 2)
    up = np.arange(n, dtype=np.float32)
    exp = sorted({v for b in range(len(s) - 1) for v in (s[b], s[b + 1] - 1)})
    np.testing.assert_array_equal(oracle.minmax(None, up, n_out), exp)
    const = np.full(n, 3, dtype=np.int32)
    np.testing.assert_array_equal(oracle.minmax(None, const, n_out), s[:-1])
    s4 = bf_edges_index(n, n_out // 4)
    np.testing.assert_array_equal(oracle.m4(None, const, n_out), sorted({v for b in range(len(s4) - 1) for v in (s4[b], s4[b + 1] - 1)}))


def test_invalid_arguments():
    y = np.zeros(10, dtype=np.float32)
    for algo, n_out in (("minmax", 3), ("minmax", 0), ("m4", 6), ("m4", 2), ("lttb", 2), ("minmaxlttb", 2)):
        with pytest.raises(oracle.OracleError):
            oracle.downsample(algo, None, y, n_out)
    with pytest.raises(oracle.OracleError):
        oracle.minmaxlttb(None, y, 4, minmax_ratio=0)


def test_empty_input():
    y = np.zeros(0, dtype=np.float32)
    for algo in ("minmax", "m4", "lttb", "minmaxlttb"):
        assert len(oracle.downsample(algo, None, y, 4)) == 0


# ----------------------------------------------------------------------------- LTTB

def test_lttb_exact_rational_brute_force():
    """Small-integer points: the binary64 chain must meet the exact-rational
    chain whenever every step's winner beats the runner-up by a clear margin."""
    rng = np.random.default_rng(31)
    checked = 0
    for trial in range(300):
        m = int(rng.integers(4, 40))
        n_out = int(rng.integers(3, m))
        py = rng.integers(-50, 50, size=m).astype(np.float64)
        px = None if trial % 2 else np.cumsum(rng.integers(1, 5, size=m)).astype(np.float64)
        exp, gap = bf_lttb_exact(frac_list(px if px is not None else np.arange(m)), frac_list(py), n_out)
        if gap < 1e-9:
            continue
        got = oracle.lttb_points(px, py, n_out)
        np.testing.assert_array_equal(got, exp, err_msg=f"trial {trial}")
        checked += 1
    assert checked > 150


def test_lttb_three_points_is_farthest_from_chord():
    """n_out = 3: one bucket, the third vertex is the last point, so the pick
    is the interior point farthest from the chord first->last."""
    rng = np.random.default_rng(32)
    for trial in range(50):
        m = int(rng.integers(4, 200))
        y = rng.standard_normal(m)
        got = oracle.lttb(None, y, 3)
        fy = frac_list(y)
        dist = [abs((m - 1) * (fy[b] - fy[0]) - (fy[m - 1] - fy[0]) * b) for b in range(1, m - 1)]
        best = max(dist)
        if sorted(dist)[-2] >= best * (1 - Fraction(1, 10 ** 9)) and len(dist) > 1:
            continue
        assert list(got) == [0, 1 + dist.index(best), m - 1]


def test_lttb_collinear_integer_data_picks_bucket_starts():
    """On a line with power-of-two buckets every mean is exact and every area
    is exactly 0, so each step keeps its bucket's first index."""
    for B, k, c, d in ((4, 4, 3, -7), (8, 2, -5, 11), (16, 8, 1, 0)):
        m = B * k + 2
        x = np.arange(m, dtype=np.float64) * 2
        y = c * x + d
        got = oracle.lttb(x, y, B + 2)
        np.testing.assert_array_equal(got, [0] + [1 + j * k for j in range(B)] + [m - 1])


@pytest.mark.parametrize("dtype", ["float32", "int16", "uint8", "float64"])
def test_lttb_invariants_and_length(dtype):
    rng = np.random.default_rng(33)
    for trial in range(20):
        n = int(rng.integers(3, 3000))
        y = inputs.random_walk(n, "float64", seed=trial)
        if dtype != "float64":
            y = np.clip(y, -100, 100).astype(dtype) if dtype.startswith("int") or dtype.startswith("uint") else y.astype(dtype)
        n_out = int(rng.integers(3, n + 5))
        idx = oracle.lttb(None, y, n_out)
        check_invariants(idx, n, n_out, "lttb")
        assert len(idx) == min(n_out, n)
        if n_out < n:
            B = n_out - 2
            for j in range(B):
                lo = 1 + (j * (n - 2)) // B
                hi = 1 + ((j + 1) * (n - 2)) // B
                assert lo <= idx[j + 1] < hi


def test_minmaxlttb_large_ratio_equals_lttb():
    """With n_out*ratio >= n-2 the preselection keeps every interior point."""
    for n, n_out in ((500, 20), (1001, 50), (64, 9)):
        y = inputs.random_walk(n, "float32", seed=n)
        ratio = (n // n_out) + 2
        np.testing.assert_array_equal(oracle.minmaxlttb(None, y, n_out, ratio), oracle.lttb(None, y, n_out))
        x = np.cumsum(np.random.default_rng(n).integers(1, 4, size=n))
        np.testing.assert_array_equal(oracle.minmaxlttb(x, y, n_out, ratio), oracle.lttb(x, y, n_out))


def test_minmaxlttb_brute_force():
    rng = np.random.default_rng(34)
    checked = 0
    for trial in range(200):
        n = int(rng.integers(6, 60))
        n_out = int(rng.integers(3, n))
        ratio = int(rng.integers(1, 4))
        y = rng.integers(-30, 30, size=n).astype(np.float64)
        n_sel = 2 * ((n_out * ratio) // 2)
        interior = y[1:n - 1]
        if n_sel >= n - 2:
            R = list(range(n))
        else:
            sel = bf_binned(interior, bf_edges_index(n - 2, n_sel // 2), 2, "propagate")
            R = [0] + [int(t) + 1 for t in sel] + [n - 1]
        picks, gap = bf_lttb_exact([Fraction(r) for r in R], frac_list(y[R]), n_out)
        if gap < 1e-9:
            continue
        np.testing.assert_array_equal(oracle.minmaxlttb(None, y, n_out, ratio), [R[p] for p in picks])
        checked += 1
    assert checked > 100


# ----------------------------------------------------------------------------- LTTB bucket averages

def lttb_bucket(j, n, n_out):
    """[lo, hi) of LTTB bucket j over points 1..n-2 (B = n_out - 2 equal-count buckets)."""
    B = n_out - 2
    return 1 + (j * (n - 2)) // B, 1 + ((j + 1) * (n - 2)) // B


@pytest.mark.parametrize("n,n_out", [(11, 5), (1000, 7), (4001, 50), (100_003, 1000)])
def test_lttb_means_closed_form_on_index_values(n, n_out):
    """y = index and no x: every average of bucket [lo, hi) is (lo + hi - 1) / 2
    in both coordinates, exactly (sums of integers below 2^53, one division)."""
    y = np.arange(n, dtype=np.int64)
    got = oracle.lttb_means(None, y, n_out)
    assert got.shape == (n_out - 3, 2)
    for j in range(1, n_out - 2):
        lo, hi = lttb_bucket(j, n, n_out)
        exp = float(Fraction(lo + hi - 1, 2))
        assert got[j - 1, 0] == exp and got[j - 1, 1] == exp, j


def test_lttb_means_sum_in_index_order_not_exactly():
    """The average is the binary64 sum taken in index order: 1e16 + 1 rounds
    back to 1e16 (a tie, to even), so [1e16, 1, -1e16] averages to 0, not 1/3."""
    n, n_out = 11, 5
    lo, hi = lttb_bucket(1, n, n_out)
    assert (lo, hi) == (4, 7)
    y = np.zeros(n)
    y[4:7] = [1e16, 1.0, -1e16]
    got = oracle.lttb_means(None, y, n_out)
    assert got[0, 1] == 0.0
    assert abs(float(Fraction(1, 3)) - got[0, 1]) > 0.3
    y[4:7] = [1.0, 1e16, -1e16]            # 1 + 1e16 rounds the same way
    assert oracle.lttb_means(None, y, n_out)[0, 1] == 0.0
    y[4:7] = [1e16, -1e16, 1.0]            # cancellation first: the 1 survives
    assert oracle.lttb_means(None, y, n_out)[0, 1] == float(Fraction(1, 3))


def test_lttb_means_nan_modes():
    """NaN-propagate: a NaN y makes the bucket's y average NaN (its x average
    stays finite); NaN-ignore leaves that point out of both sums and the count."""
    n, n_out = 11, 5
    y = np.arange(n, dtype=np.float64)
    y[5] = np.nan
    x = np.arange(n, dtype=np.float64) * 3.0
    prop = oracle.lttb_means(x, y, n_out, nan="propagate")
    assert np.isnan(prop[0, 1]) and prop[0, 0] == 15.0           # x = 12, 15, 18
    ign = oracle.lttb_means(x, y, n_out, nan="ignore")
    assert ign[0, 0] == 15.0 and ign[0, 1] == 5.0                # points 4 and 6
    y[4:7] = np.nan
    assert np.isnan(oracle.lttb_means(x, y, n_out, nan="ignore")[0]).all()   # 0 / 0


def test_lttb_means_rejects_undefined_shapes():
    y = np.arange(10, dtype=np.float64)
    for n_out in (2, 10, 11):
        with pytest.raises(oracle.OracleError):
            oracle.lttb_means(None, y, n_out)


# ----------------------------------------------------------------------------- EveryNth

@pytest.mark.parametrize("n,n_out", [(11, 3), (1000, 7), (1001, 1000), (100_003, 999), (10 ** 6, 4000)])
def test_everynth_closed_form_without_x(n, n_out):
    """No x: the first index of each of n_out equal index bins, ceil(i(n-1)/n_out):
    exactly n_out strictly increasing picks starting at 0 (exact integer arithmetic)."""
    y = np.zeros(n, dtype=np.float32)
    got = oracle.everynth(None, y, n_out)
    exp = [-((-i * (n - 1)) // n_out) for i in range(n_out)]
    np.testing.assert_array_equal(got, exp)
    assert got[0] == 0 and np.all(np.diff(got) >= 1)


def test_everynth_brute_force_integer_x():
    """Sorted integer x with gaps and repeats: bin i is {j : (x_j - x_0) n_out in
    [i span, (i+1) span)}; the pick is its first j, scanned exactly."""
    rng = np.random.default_rng(41)
    for trial in range(200):
        n = int(rng.integers(2, 60))
        n_out = int(rng.integers(1, n))
        xs = np.cumsum(rng.integers(0, 4, size=n)).astype(np.int64)
        xs[0] = 0
        exp = [s for s, e in zip(bf_edges_int_x(xs.tolist(), n_out)[:-1], bf_edges_int_x(xs.tolist(), n_out)[1:])
               if s < e]
        got = oracle.everynth(xs, np.zeros(n), n_out)
        np.testing.assert_array_equal(got, exp, err_msg=f"trial {trial}")


@pytest.mark.parametrize("x_dtype", ["int64", "float64", "uint32"])
def test_everynth_equal_x_matches_no_x(x_dtype):
    n = 50_001
    y = inputs.random_walk(n, "float32", 3)
    for n_out in (10, 999, 5000):
        np.testing.assert_array_equal(oracle.everynth(np.arange(n).astype(x_dtype), y, n_out),
                                      oracle.everynth(None, y, n_out))


def test_everynth_is_the_first_pick_of_each_m4_bin():
    """With the same bins (M4 with 4 n_out), EveryNth is the first M4 pick of each
    non-empty bin: a subset of M4 of one pick per bin."""
    n = 20_011
    y = inputs.random_walk(n, "float32", 4)
    x = inputs.geometric_x(n, 4)
    for xx in (None, x):
        for n_out in (7, 250, 3000):
            e = oracle.everynth(xx, y, n_out)
            m4 = oracle.m4(xx, y, 4 * n_out)
            assert set(e.tolist()) <= set(m4.tolist())
            s = oracle.bin_edges(xx, n, n_out)
            assert len(e) == int(np.sum(s[1:] > s[:-1]))


def test_everynth_degenerate_shapes():
    y = np.arange(5, dtype=np.float64)
    np.testing.assert_array_equal(oracle.everynth(None, y, 5), np.arange(5))
    np.testing.assert_array_equal(oracle.everynth(None, y, 9), np.arange(5))
    np.testing.assert_array_equal(oracle.everynth(None, y, 1), [0])
    assert len(oracle.everynth(None, y[:0], 3)) == 0
    with pytest.raises(oracle.OracleError):
        oracle.everynth(None, y, 0)
