/*
 * tsds_oracle.c -- CPU oracle for MinMax, M4, LTTB and MinMaxLTTB as used by
 * "tsdownsample" (arXiv 2307.05389).
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow, single-threaded restatement written
 * for obviousness, not speed.  Built with -O2 -ffp-contract=off so that no
 * multiply-add is fused; no SIMD intrinsics; no code shared with the CUDA
 * library.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg use it.
 *
 * The paper names the algorithms (Section 1) and gives the per-bin argmin /
 * argmax loop (Section 2.1, Listing 1) and the interface (Section 2.3); it
 * defines neither the bins nor LTTB's buckets.  Where it is silent this file
 * follows these readings:
 *   - MinMax uses n_out/2 bins, M4 n_out/4 bins.
 *   - Without x, bin i starts at ceil(i*(n-1)/nb); with x, bin i starts at the
 *     first point whose x reaches x_0 + i*(x_{n-1}-x_0)/nb (exact integer
 *     arithmetic for integer x, binary64 with each operation rounded for
 *     floating x).  The last bin ends at n.  Empty bins select nothing
 *     (Section 2.3 footnote on gaps).
 *   - Ties go to the lowest index (the strict comparisons of Listing 1);
 *     -0 and +0 are equal; float16 compares as the IEEE value it encodes.
 *   - NaN-propagate: a bin holding a NaN selects its first NaN as both argmin
 *     and argmax.  NaN-ignore: NaNs are skipped; an all-NaN bin selects its
 *     first index.
 *   - A bin's output is the sorted, de-duplicated set of its selections.
 *   - n_out >= n returns every index.
 *   - LTTB: B = n_out-2 buckets over points 1..m-2, bucket j covering
 *     [1 + floor(j(m-2)/B), 1 + floor((j+1)(m-2)/B)); the point after the last
 *     bucket is the last point.  Means are binary64 sums in index order
 *     divided by the count.  The doubled triangle area is
 *     |(xa-xm)(yb-ya) - (xa-xb)(ym-ya)| with every operation rounded; the
 *     largest area wins, ties to the lowest index.
 *   - MinMaxLTTB: MinMax over the interior points 1..n-2 with
 *     2*floor(n_out*ratio/2) selections, plus the first and last point, then
 *     LTTB over those points with their original x (or index).
 */
#include "tsds_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ---------------------------------------------------------------- element access */

static int valid_dtype(int dt) { return dt >= ORC_I8 && dt <= ORC_F64; }
static int is_float(int dt) { return dt == ORC_F16 || dt == ORC_F32 || dt == ORC_F64; }
static int is_signed_int(int dt) { return dt >= ORC_I8 && dt <= ORC_I64; }

static size_t dtype_size(int dt) {
  switch (dt) {
    case ORC_I8: case ORC_U8: return 1;
    case ORC_I16: case ORC_U16: case ORC_F16: return 2;
    case ORC_I32: case ORC_U32: case ORC_F32: return 4;
    default: return 8;
  }
}

/* IEEE 754 binary16: sign, 5-bit exponent (bias 15), 10-bit fraction. */
double orc_f16_to_f64(uint16_t h) {
  int sign = (h >> 15) & 1;
  int e = (h >> 10) & 0x1F;
  int f = h & 0x3FF;
  double v;
  if (e == 0) {
    v = ldexp((double)f, -24);               /* subnormal: f * 2^-24 */
  } else if (e == 31) {
    v = (f == 0) ? INFINITY : NAN;
  } else {
    v = ldexp((double)(1024 + f), e - 25);  /* (1 + f/1024) * 2^(e-15) */
  }
  return sign ? -v : v;
}

static int64_t get_i(const void* p, int dt, int64_t i) {
  switch (dt) {
    case ORC_I8: return ((const int8_t*)p)[i];
    case ORC_I16: return ((const int16_t*)p)[i];
    case ORC_I32: return ((const int32_t*)p)[i];
    default: return ((const int64_t*)p)[i];
  }
}

static uint64_t get_u(const void* p, int dt, int64_t i) {
  switch (dt) {
    case ORC_U8: return ((const uint8_t*)p)[i];
    case ORC_U16: return ((const uint16_t*)p)[i];
    case ORC_U32: return ((const uint32_t*)p)[i];
    default: return ((const uint64_t*)p)[i];
  }
}

static double get_f(const void* p, int dt, int64_t i) {
  switch (dt) {
    case ORC_F16: return orc_f16_to_f64(((const uint16_t*)p)[i]);
    case ORC_F32: return (double)((const float*)p)[i];
    default: return ((const double*)p)[i];
  }
}

/* Any element as binary64, rounded to nearest (exact except for 64-bit
 * integers beyond 2^53). */
static double get_as_double(const void* p, int dt, int64_t i) {
  if (is_float(dt)) return get_f(p, dt, i);
  if (is_signed_int(dt)) return (double)get_i(p, dt, i);
  return (double)get_u(p, dt, i);
}

static int y_isnan(const void* y, int dt, int64_t i) {
  return is_float(dt) && isnan(get_f(y, dt, i));
}

/* y[i] < y[j] as numbers (never true when either is NaN). */
static int y_less(const void* y, int dt, int64_t i, int64_t j) {
  if (is_float(dt)) return get_f(y, dt, i) < get_f(y, dt, j);
  if (is_signed_int(dt)) return get_i(y, dt, i) < get_i(y, dt, j);
  return get_u(y, dt, i) < get_u(y, dt, j);
}

/* ---------------------------------------------------------------- bins */

/* (x_j - x_0) for sorted integer x, as an unsigned 128-bit number. */
static u128 int_offset(const void* x, int dt, int64_t j) {
  if (is_signed_int(dt)) {
    __int128 d = (__int128)get_i(x, dt, j) - (__int128)get_i(x, dt, 0);
    return (u128)d;
  }
  return (u128)(get_u(x, dt, j) - get_u(x, dt, 0));
}

/* First j in [0, n) with predicate true, for a predicate that is false then
 * true along the sorted x (a plain lower bound). */
static int64_t first_int_edge(const void* x, int dt, int64_t n, int64_t nb, int64_t i, u128 span) {
  int64_t lo = 0, hi = n;             /* answer in [lo, hi] */
  u128 rhs = (u128)i * span;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (int_offset(x, dt, mid) * (u128)nb >= rhs) hi = mid; else lo = mid + 1;
  }
  return lo;
}

static int64_t first_float_edge(const void* x, int dt, int64_t n, double e) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (get_f(x, dt, mid) >= e) hi = mid; else lo = mid + 1;
  }
  return lo;
}

int64_t orc_bin_edges(const void* x, int x_dtype, int64_t n, int64_t nb, int64_t* s) {
  if (n < 1 || nb < 1 || !s) return ORC_EINVAL;
  if (x && !valid_dtype(x_dtype)) return ORC_EINVAL;
  s[0] = 0;
  s[nb] = n;
  if (!x) {
    /* equally spaced: bin i starts at ceil(i*(n-1)/nb) */
    for (int64_t i = 1; i < nb; ++i) {
      u128 num = (u128)i * (u128)(n - 1);
      s[i] = (int64_t)((num + (u128)nb - 1) / (u128)nb);
    }
  } else if (is_float(x_dtype)) {
    double x0 = get_f(x, x_dtype, 0);
    double xl = get_f(x, x_dtype, n - 1);
    double span = xl - x0;
    for (int64_t i = 1; i < nb; ++i) {
      double e = x0 + (span * (double)i) / (double)nb;
      s[i] = first_float_edge(x, x_dtype, n, e);
    }
  } else {
    u128 span = int_offset(x, x_dtype, n - 1);
    for (int64_t i = 1; i < nb; ++i) s[i] = first_int_edge(x, x_dtype, n, nb, i, span);
  }
  return nb + 1;
}

/* ---------------------------------------------------------------- argmin / argmax */

int orc_argminmax(const void* y, int y_dtype, int64_t lo, int64_t hi, int nan_mode,
                  int64_t* imin, int64_t* imax) {
  if (!y || !valid_dtype(y_dtype) || lo < 0 || hi <= lo) return ORC_EINVAL;
  if (nan_mode == ORC_NAN_PROPAGATE) {
    for (int64_t i = lo; i < hi; ++i) {
      if (y_isnan(y, y_dtype, i)) { *imin = i; *imax = i; return 0; }
    }
  }
  int64_t mn = -1, mx = -1;
  for (int64_t i = lo; i < hi; ++i) {
    if (y_isnan(y, y_dtype, i)) continue;
    if (mn < 0) { mn = i; mx = i; continue; }
    if (y_less(y, y_dtype, i, mn)) mn = i;   /* strict: the earliest minimum stays */
    if (y_less(y, y_dtype, mx, i)) mx = i;   /* strict: the earliest maximum stays */
  }
  if (mn < 0) { mn = lo; mx = lo; }          /* all NaN (NaN-ignore) */
  *imin = mn;
  *imax = mx;
  return 0;
}

/* ---------------------------------------------------------------- MinMax / M4 */

/* Append the sorted distinct values of v[0..k) to out. */
static void append_sorted_unique(int64_t* v, int k, int64_t* out, int64_t* cnt) {
  for (int a = 1; a < k; ++a) {           /* insertion sort, k <= 4 */
    int64_t t = v[a];
    int b = a - 1;
    while (b >= 0 && v[b] > t) { v[b + 1] = v[b]; --b; }
    v[b + 1] = t;
  }
  for (int a = 0; a < k; ++a) {
    if (a > 0 && v[a] == v[a - 1]) continue;
    out[(*cnt)++] = v[a];
  }
}

static int args_ok(const void* x, int x_dtype, const void* y, int y_dtype, int64_t n) {
  if (n < 0) return 0;
  if (n > 0 && !y) return 0;
  if (!valid_dtype(y_dtype)) return 0;
  if (x && !valid_dtype(x_dtype)) return 0;
  return 1;
}

static int64_t all_indices(int64_t n, int64_t* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = i;
  return n;
}

/* The output of bins [b0, b1) with per_bin = 2 (MinMax) or 4 (M4) selections
 * per bin, the bins laid out over the whole series.  Each bin's selections
 * depend on that bin alone (Section 2.2 runs bins on separate threads), so
 * the output of all nb bins is the concatenation of these pieces in bin
 * order. */
static int64_t binned_range(const void* x, int x_dtype, const void* y, int y_dtype, int64_t n,
                            int64_t n_out, int nan_mode, int64_t* out, int per_bin, int64_t b0, int64_t b1) {
  int64_t nb = n_out / per_bin;
  int64_t* s = (int64_t*)malloc((size_t)(nb + 1) * sizeof(int64_t));
  if (!s) return ORC_EINVAL;
  orc_bin_edges(x, x_dtype, n, nb, s);
  int64_t cnt = 0;
  for (int64_t b = b0; b < b1; ++b) {
    int64_t lo = s[b], hi = s[b + 1];
    if (lo >= hi) continue;                 /* empty bin: nothing selected */
    int64_t mn, mx;
    orc_argminmax(y, y_dtype, lo, hi, nan_mode, &mn, &mx);
    int64_t v[4];
    if (per_bin == 2) {
      v[0] = mn; v[1] = mx;
      append_sorted_unique(v, 2, out, &cnt);
    } else {
      v[0] = lo; v[1] = mn; v[2] = mx; v[3] = hi - 1;
      append_sorted_unique(v, 4, out, &cnt);
    }
  }
  free(s);
  return cnt;
}

static int64_t binned(const void* x, int x_dtype, const void* y, int y_dtype, int64_t n,
                      int64_t n_out, int nan_mode, int64_t* out, int per_bin) {
  return binned_range(x, x_dtype, y, y_dtype, n, n_out, nan_mode, out, per_bin, 0, n_out / per_bin);
}

int64_t orc_minmax(const void* x, int x_dtype, const void* y, int y_dtype, int64_t n,
                   int64_t n_out, int nan_mode, int64_t* out) {
  if (!args_ok(x, x_dtype, y, y_dtype, n) || n_out < 2 || n_out % 2 != 0) return ORC_EINVAL;
  if (n_out >= n) return all_indices(n, out);
  return binned(x, x_dtype, y, y_dtype, n, n_out, nan_mode, out, 2);
}

int64_t orc_m4(const void* x, int x_dtype, const void* y, int y_dtype, int64_t n,
               int64_t n_out, int nan_mode, int64_t* out) {
  if (!args_ok(x, x_dtype, y, y_dtype, n) || n_out < 4 || n_out % 4 != 0) return ORC_EINVAL;
  if (n_out >= n) return all_indices(n, out);
  return binned(x, x_dtype, y, y_dtype, n, n_out, nan_mode, out, 4);
}

int64_t orc_binned_range(int per_bin, const void* x, int x_dtype, const void* y, int y_dtype, int64_t n,
                         int64_t n_out, int nan_mode, int64_t b0, int64_t b1, int64_t* out) {
  if (per_bin != 2 && per_bin != 4) return ORC_EINVAL;
  if (!args_ok(x, x_dtype, y, y_dtype, n) || n_out < per_bin || n_out % per_bin != 0 || n_out >= n) return ORC_EINVAL;
  if (b0 < 0 || b1 < b0 || b1 > n_out / per_bin) return ORC_EINVAL;
  return binned_range(x, x_dtype, y, y_dtype, n, n_out, nan_mode, out, per_bin, b0, b1);
}

/* EveryNth (Section 1 names it; the reading here): n_out bins laid out as
 * MinMax/M4 lay them out (index space without x, equal-width x ranges with
 * x), and the first point of every non-empty bin. */
int64_t orc_everynth(const void* x, int x_dtype, const void* y, int y_dtype, int64_t n,
                     int64_t n_out, int nan_mode, int64_t* out) {
  (void)nan_mode;
  if (!args_ok(x, x_dtype, y, y_dtype, n) || n_out < 1) return ORC_EINVAL;
  if (n_out >= n) return all_indices(n, out);
  int64_t* s = (int64_t*)malloc((size_t)(n_out + 1) * sizeof(int64_t));
  if (!s) return ORC_EINVAL;
  orc_bin_edges(x, x_dtype, n, n_out, s);
  int64_t cnt = 0;
  for (int64_t b = 0; b < n_out; ++b)
    if (s[b] < s[b + 1]) out[cnt++] = s[b];
  free(s);
  return cnt;
}

/* ---------------------------------------------------------------- LTTB */

/* Bucket j of B over points 1..m-2 starts at 1 + floor(j*(m-2)/B). */
static int64_t bucket_start(int64_t j, int64_t m, int64_t B) {
  return 1 + (int64_t)(((u128)j * (u128)(m - 2)) / (u128)B);
}

static double px_at(const double* px, int64_t k) { return px ? px[k] : (double)k; }

/* Mean of the points [lo, hi): binary64 sums in index order, then one division
 * by the count.  NaN-ignore leaves out points whose y is NaN. */
static void bucket_mean(const double* px, const double* py, int64_t lo, int64_t hi,
                        int nan_mode, double* mx, double* my) {
  double sx = 0.0, sy = 0.0;
  int64_t c = 0;
  for (int64_t k = lo; k < hi; ++k) {
    if (nan_mode == ORC_NAN_IGNORE && isnan(py[k])) continue;
    sx += px_at(px, k);
    sy += py[k];
    ++c;
  }
  *mx = sx / (double)c;   /* c == 0 gives NaN */
  *my = sy / (double)c;
}

int64_t orc_lttb_points(const double* px, const double* py, int64_t m, int64_t n_out,
                        int nan_mode, int64_t* out) {
  if (m < 0 || n_out < 3 || (m > 0 && !py)) return ORC_EINVAL;
  if (n_out >= m) return all_indices(m, out);
  int64_t B = n_out - 2;
  int64_t a = 0;                           /* previous selection */
  out[0] = 0;
  for (int64_t j = 0; j < B; ++j) {
    int64_t lo = bucket_start(j, m, B);
    int64_t hi = bucket_start(j + 1, m, B);
    double xm, ym;
    if (j == B - 1) {
      xm = px_at(px, m - 1);
      ym = py[m - 1];
    } else {
      bucket_mean(px, py, hi, bucket_start(j + 2, m, B), nan_mode, &xm, &ym);
    }
    double xa = px_at(px, a), ya = py[a];
    int64_t best = -1;
    double best_area = 0.0;
    int best_is_nan = 0;
    for (int64_t b = lo; b < hi; ++b) {
      double t1 = (xa - xm) * (py[b] - ya);
      double t2 = (xa - px_at(px, b)) * (ym - ya);
      double area = fabs(t1 - t2);
      if (isnan(area)) {
        /* NaN-propagate: a NaN area beats every number; the first one stays. */
        if (nan_mode == ORC_NAN_PROPAGATE && !best_is_nan) { best = b; best_is_nan = 1; }
        continue;
      }
      if (best_is_nan) continue;
      if (best < 0 || area > best_area) { best = b; best_area = area; }
    }
    if (best < 0) best = lo;                 /* no candidate (NaN-ignore) */
    out[j + 1] = best;
    a = best;
  }
  out[B + 1] = m - 1;
  return n_out;
}

int64_t orc_lttb(const void* x, int x_dtype, const void* y, int y_dtype, int64_t n,
                 int64_t n_out, int nan_mode, int64_t* out) {
  if (!args_ok(x, x_dtype, y, y_dtype, n) || n_out < 3) return ORC_EINVAL;
  if (n_out >= n) return all_indices(n, out);
  double* px = NULL;
  double* py = (double*)malloc((size_t)n * sizeof(double));
  if (!py) return ORC_EINVAL;
  if (x) {
    px = (double*)malloc((size_t)n * sizeof(double));
    if (!px) { free(py); return ORC_EINVAL; }
    for (int64_t i = 0; i < n; ++i) px[i] = get_as_double(x, x_dtype, i);
  }
  for (int64_t i = 0; i < n; ++i) py[i] = get_as_double(y, y_dtype, i);
  int64_t r = orc_lttb_points(px, py, n, n_out, nan_mode, out);
  free(px);
  free(py);
  return r;
}

/* The averages step j = 0 .. B-2 of orc_lttb_points uses: buckets 1 .. B-1,
 * (x, y) pairs, from the same binary64 conversion as orc_lttb. */
int64_t orc_lttb_means(const void* x, int x_dtype, const void* y, int y_dtype, int64_t n,
                       int64_t n_out, int nan_mode, double* out) {
  if (!args_ok(x, x_dtype, y, y_dtype, n) || n_out < 3 || n_out >= n) return ORC_EINVAL;
  double* px = NULL;
  double* py = (double*)malloc((size_t)n * sizeof(double));
  if (!py) return ORC_EINVAL;
  if (x) {
    px = (double*)malloc((size_t)n * sizeof(double));
    if (!px) { free(py); return ORC_EINVAL; }
    for (int64_t i = 0; i < n; ++i) px[i] = get_as_double(x, x_dtype, i);
  }
  for (int64_t i = 0; i < n; ++i) py[i] = get_as_double(y, y_dtype, i);
  int64_t B = n_out - 2;
  for (int64_t j = 1; j < B; ++j)
    bucket_mean(px, py, bucket_start(j, n, B), bucket_start(j + 1, n, B), nan_mode, &out[2 * (j - 1)],
                &out[2 * (j - 1) + 1]);
  free(px);
  free(py);
  return B - 1;
}

/* ---------------------------------------------------------------- MinMaxLTTB */

int64_t orc_minmaxlttb(const void* x, int x_dtype, const void* y, int y_dtype, int64_t n,
                       int64_t n_out, int64_t minmax_ratio, int nan_mode, int64_t* out) {
  if (!args_ok(x, x_dtype, y, y_dtype, n) || n_out < 3 || minmax_ratio < 1) return ORC_EINVAL;
  if (minmax_ratio > (INT64_MAX / 4) / n_out) return ORC_EINVAL;
  if (n_out >= n) return all_indices(n, out);
  /* n > n_out >= 3, so the interior 1..n-2 holds at least two points. */
  int64_t n_sel = 2 * ((n_out * minmax_ratio) / 2);
  int64_t n_in = n - 2;
  int64_t cap = (n_sel < n_in ? n_sel : n_in) + 2;
  int64_t* R = (int64_t*)malloc((size_t)cap * sizeof(int64_t));
  if (!R) return ORC_EINVAL;
  const void* x_in = x ? (const void*)((const char*)x + dtype_size(x_dtype)) : NULL;
  const void* y_in = (const void*)((const char*)y + dtype_size(y_dtype));
  int64_t k = orc_minmax(x_in, x_dtype, y_in, y_dtype, n_in, n_sel, nan_mode, R + 1);
  if (k < 0) { free(R); return k; }
  R[0] = 0;
  for (int64_t i = 1; i <= k; ++i) R[i] += 1;   /* interior index -> series index */
  R[k + 1] = n - 1;
  int64_t m = k + 2;

  double* px = x ? (double*)malloc((size_t)m * sizeof(double)) : NULL;
  double* py = (double*)malloc((size_t)m * sizeof(double));
  int64_t* pick = (int64_t*)malloc((size_t)m * sizeof(int64_t));
  if ((x && !px) || !py || !pick) { free(R); free(px); free(py); free(pick); return ORC_EINVAL; }
  for (int64_t i = 0; i < m; ++i) {
    if (px) px[i] = get_as_double(x, x_dtype, R[i]);
    py[i] = get_as_double(y, y_dtype, R[i]);
  }
  int64_t cnt;
  if (px) {
    cnt = orc_lttb_points(px, py, m, n_out, nan_mode, pick);
  } else {
    /* x is the original index of each selected point */
    double* pxi = (double*)malloc((size_t)m * sizeof(double));
    if (!pxi) { free(R); free(py); free(pick); return ORC_EINVAL; }
    for (int64_t i = 0; i < m; ++i) pxi[i] = (double)R[i];
    cnt = orc_lttb_points(pxi, py, m, n_out, nan_mode, pick);
    free(pxi);
  }
  for (int64_t i = 0; i < cnt; ++i) out[i] = R[pick[i]];
  free(R); free(px); free(py); free(pick);
  return cnt;
}
