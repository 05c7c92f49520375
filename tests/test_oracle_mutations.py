"""The pins are strong enough to catch plausible mistakes in the oracle: each
case below plants one mistake in a copy of tsds_oracle.c (a flipped
comparison, a floor for a ceiling, a swapped operand, a dropped term, an
off-by-one index), compiles it, and runs the pin suite against it, which must
fail.  The copies live in a temporary directory; the real oracle is never
touched."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "tsds_oracle.c")

MUTATIONS = [
    # tie rule: a later index wins ties for the minimum
    ("if (y_less(y, y_dtype, i, mn)) mn = i;", "if (!y_less(y, y_dtype, mn, i)) mn = i;"),
    # index bins: floor instead of ceil
    ("s[i] = (int64_t)((num + (u128)nb - 1) / (u128)nb);", "s[i] = (int64_t)(num / (u128)nb);"),
    # LTTB area: the second term's x difference with its sign flipped
    ("double t2 = (xa - px_at(px, b)) * (ym - ya);", "double t2 = (px_at(px, b) - xa) * (ym - ya);"),
    # M4: the wrong last point of a bin
    ("v[3] = hi - 1;", "v[3] = hi - 2 < lo ? lo : hi - 2;"),
    # LTTB: the last of equal areas wins
    ("if (best < 0 || area > best_area)", "if (best < 0 || area >= best_area)"),
    # float x: the edge of the next bin
    ("double e = x0 + (span * (double)i) / (double)nb;", "double e = x0 + (span * (double)(i+1)) / (double)nb;"),
    # LTTB: the last bucket's third vertex is the second-to-last point
    ("xm = px_at(px, m - 1);", "xm = px_at(px, m - 2);"),
    # NaN-ignore means keep NaN points
    ("if (nan_mode == ORC_NAN_IGNORE && isnan(py[k])) continue;", "if (0) continue;"),
    # MinMaxLTTB: the last preselected index not shifted to the whole series
    ("for (int64_t i = 1; i <= k; ++i) R[i] += 1;", "for (int64_t i = 1; i < k; ++i) R[i] += 1;"),
    # float16 decoding drops the sign
    ("return sign ? -v : v;", "return v;"),
    # EveryNth: the last point of each bin instead of the first
    ("if (s[b] < s[b + 1]) out[cnt++] = s[b];", "if (s[b] < s[b + 1]) out[cnt++] = s[b + 1] - 1;"),
    # bucket means: divided by one more than the count
    ("*mx = sx / (double)c;", "*mx = sx / (double)(c + 1);"),
    # LTTB buckets laid out over m-1 points instead of m-2
    ("return 1 + (int64_t)(((u128)j * (u128)(m - 2)) / (u128)B);",
     "return 1 + (int64_t)(((u128)j * (u128)(m - 1)) / (u128)B);"),
    # integer x edges: strict instead of reaching the edge
    ("if (int_offset(x, dt, mid) * (u128)nb >= rhs) hi = mid; else lo = mid + 1;",
     "if (int_offset(x, dt, mid) * (u128)nb > rhs) hi = mid; else lo = mid + 1;"),
    # float x edges: strict instead of reaching the edge
    ("if (get_f(x, dt, mid) >= e) hi = mid; else lo = mid + 1;", "if (get_f(x, dt, mid) > e) hi = mid; else lo = mid + 1;"),
    # NaN-propagate: the last NaN of a bin instead of the first
    ("if (y_isnan(y, y_dtype, i)) { *imin = i; *imax = i; return 0; }",
     "if (y_isnan(y, y_dtype, i)) { *imin = i; *imax = i; }"),
    # tie rule for the maximum
    ("if (y_less(y, y_dtype, mx, i)) mx = i;   /* strict: the earliest maximum stays */",
     "if (!y_less(y, y_dtype, i, mx)) mx = i;"),
    # an all-NaN bin (NaN-ignore) selects its last index
    ("if (mn < 0) { mn = lo; mx = lo; }", "if (mn < 0) { mn = hi - 1; mx = hi - 1; }"),
    # uint64 x offsets taken as signed differences
    ("return (u128)(get_u(x, dt, j) - get_u(x, dt, 0));",
     "return (u128)(__int128)((int64_t)get_u(x, dt, j) - (int64_t)get_u(x, dt, 0));"),
    # LTTB NaN-propagate: the last NaN area wins
    ("if (nan_mode == ORC_NAN_PROPAGATE && !best_is_nan) { best = b; best_is_nan = 1; }",
     "if (nan_mode == ORC_NAN_PROPAGATE) { best = b; best_is_nan = 1; }"),
    # MinMaxLTTB preselection size rounded up
    ("int64_t n_sel = 2 * ((n_out * minmax_ratio) / 2);", "int64_t n_sel = 2 * ((n_out * minmax_ratio + 1) / 2);"),
    # bin ranges: the range starts at bin 0 whatever b0 is
    ("return binned_range(x, x_dtype, y, y_dtype, n, n_out, nan_mode, out, per_bin, b0, b1);",
     "return binned_range(x, x_dtype, y, y_dtype, n, n_out, nan_mode, out, per_bin, 0, b1);"),
    # LTTB area: the wrong vertex in the first term
    ("double t1 = (xa - xm) * (py[b] - ya);", "double t1 = (xa - xm) * (py[b] - ym);"),
]


@pytest.mark.parametrize("old,new", MUTATIONS, ids=[f"m{i}" for i in range(len(MUTATIONS))])
def test_planted_mistake_fails_the_pins(old, new, tmp_path):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found once: {old}"
    mutated = tmp_path / "tsds_oracle.c"
    mutated.write_text(src.replace(old, new))
    (tmp_path / "tsds_oracle.h").write_text(open(os.path.join(ROOT, "oracle", "tsds_oracle.h")).read())
    lib = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared", "-o",
                    str(lib), str(mutated), "-lm"], check=True)
    env = dict(os.environ, TSDS_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-x", "-q",
                        "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin caught: {new}\n{r.stdout[-500:]}"
    assert "failed" in r.stdout.lower() or "error" in r.stdout.lower()
