/*
 * tsds_oracle.h -- CPU oracle for the downsampling algorithms of
 * "tsdownsample: high-performance time series downsampling for scalable
 * visualization" (arXiv 2307.05389).
 *
 * TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, single-threaded C
 * restatement of what the algorithms compute.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg load it; the library's product
 * path never links, includes or calls anything here, and this file shares no
 * code, header, constant or table with the CUDA library.
 *
 * Every function returns the number of indices written (>= 0) or ORC_EINVAL
 * for an argument the algorithms do not define.  Indices are int64 and
 * strictly increasing.  All buffers are host memory owned by the caller.
 */
#ifndef TSDS_ORACLE_H
#define TSDS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Element types: the eleven dtypes the paper's ArgMinMax supports (Section 2.1). */
enum {
  ORC_I8 = 0, ORC_I16, ORC_I32, ORC_I64,
  ORC_U8, ORC_U16, ORC_U32, ORC_U64,
  ORC_F16, ORC_F32, ORC_F64
};
enum { ORC_NAN_PROPAGATE = 0, ORC_NAN_IGNORE = 1 };
#define ORC_EINVAL (-1)

/* binary16 -> binary64, exact (IEEE 754-2008 binary16, Section 2.1.2 footnote). */
double orc_f16_to_f64(uint16_t h);

/* Bin edges s[0..nb] (nb+1 values) for n points, as the MinMax/M4 bin planner
 * defines them (Section 2.2: a search-sorted bin index generator).  x may be
 * NULL (equally spaced points). */
int64_t orc_bin_edges(const void* x, int x_dtype, int64_t n, int64_t nb, int64_t* s);

/* Per-bin argmin/argmax over y[lo, hi) (Section 2.1, Listing 1). */
int orc_argminmax(const void* y, int y_dtype, int64_t lo, int64_t hi, int nan_mode,
                  int64_t* imin, int64_t* imax);

/* downsample([x], y, n_out) for each algorithm (Section 2.3).  out must hold
 * n_out indices (n when n_out >= n). */
int64_t orc_minmax(const void* x, int x_dtype, const void* y, int y_dtype, int64_t n,
                   int64_t n_out, int nan_mode, int64_t* out);
int64_t orc_m4(const void* x, int x_dtype, const void* y, int y_dtype, int64_t n,
               int64_t n_out, int nan_mode, int64_t* out);
int64_t orc_lttb(const void* x, int x_dtype, const void* y, int y_dtype, int64_t n,
                 int64_t n_out, int nan_mode, int64_t* out);
int64_t orc_minmaxlttb(const void* x, int x_dtype, const void* y, int y_dtype, int64_t n,
                       int64_t n_out, int64_t minmax_ratio, int nan_mode, int64_t* out);

/* The part of the MinMax (per_bin 2) or M4 (per_bin 4) output that bins
 * [b0, b1) select, with the bins laid out over the whole series (n_out < n).
 * Bins are independent, so the full output is the concatenation of these
 * parts over consecutive bin ranges.  out must hold per_bin*(b1-b0) indices. */
int64_t orc_binned_range(int per_bin, const void* x, int x_dtype, const void* y, int y_dtype, int64_t n,
                         int64_t n_out, int nan_mode, int64_t b0, int64_t b1, int64_t* out);

/* EveryNth (reading): the first point of each non-empty bin of the MinMax/M4
 * bin layout with n_out bins; n_out >= 1. */
int64_t orc_everynth(const void* x, int x_dtype, const void* y, int y_dtype, int64_t n,
                     int64_t n_out, int nan_mode, int64_t* out);

/* The LTTB bucket chain on points already converted to binary64 (px may be
 * NULL: x = index).  Exposed so the tests can pin the chain on hand-built
 * point sets. */
int64_t orc_lttb_points(const double* px, const double* py, int64_t m, int64_t n_out,
                        int nan_mode, int64_t* out);

/* The bucket averages of orc_lttb (buckets 1 .. n_out-3, (x, y) pairs into
 * out[2*(n_out-3)]): binary64 sums in index order divided by the count.
 * Needs 3 <= n_out < n.  Returns n_out - 3. */
int64_t orc_lttb_means(const void* x, int x_dtype, const void* y, int y_dtype, int64_t n,
                       int64_t n_out, int nan_mode, double* out);

#ifdef __cplusplus
}
#endif
#endif
