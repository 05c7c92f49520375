/*
 * tsds.h -- C ABI of the GB300 time-series downsampling library.
 *
 * The library computes, on one NVIDIA GB300 GPU, the index selections of the
 * downsampling algorithms offered by "tsdownsample: high-performance time
 * series downsampling for scalable visualization" (arXiv 2307.05389):
 * MinMax, M4, LTTB and MinMaxLTTB.  Each call mirrors the paper's interface
 * downsample([x], y, n_out) -> indices (Section 2.3), returning int64 indices
 * of the selected points in increasing order.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers named x, y, out and out_count are CUDA device pointers owned by
 *    the caller.  The library never frees them, never keeps them past the
 *    call's completion on the stream and never copies y or x.
 *  - y holds n elements of y_dtype; x is NULL (equally spaced points, Section
 *    2.3) or holds n elements of x_dtype sorted non-decreasing, with no NaN.
 *    That order is checked only in checked mode (tsds_checked), which
 *    rejects an x out of order; without it such an x is outside the contract
 *    and the call's behaviour is undefined.  Both must be aligned to their
 *    element size.
 *  - out must have room for n_out indices (for MinMaxLTTB also n_out); when
 *    n_out >= n it receives 0..n-1 and needs room for n.  *out_count (a device
 *    int64) receives the number of indices written.  With x, empty bins select
 *    nothing, so MinMax and M4 may return fewer than n_out indices (Section
 *    2.3 footnote).
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL selects the legacy default stream).  Scratch memory is taken from a
 *    library-owned, stream-ordered pool on the current device and returned to
 *    it in stream order; tsds_shutdown releases the pool.
 *  - Status codes are returned, never exceptions.  TSDS_EINVAL leaves out and
 *    out_count untouched.  tsds_last_error() describes the last failure of
 *    the calling thread.
 *
 * Semantics (the paper states the interface and the argmin/argmax loop,
 * Section 2.1 Listing 1; it does not define bins or LTTB buckets, so the
 * library fixes these readings):
 *  - MinMax uses n_out/2 bins, M4 n_out/4 bins.  Without x, bin i starts at
 *    ceil(i*(n-1)/nb); with x, bin i starts at the first point whose x
 *    reaches x_0 + i*(x_{n-1}-x_0)/nb (exact integer arithmetic for integer x,
 *    binary64 with each operation rounded to nearest for floating x).  The
 *    last bin ends at n.
 *  - Per bin MinMax selects {argmin, argmax}, M4 {first, argmin, argmax,
 *    last}; each bin's selections are emitted once each, in increasing order.
 *    Ties go to the lowest index; -0 equals +0; float16 compares as the value
 *    it encodes.
 *  - TSDS_NAN_PROPAGATE: a bin holding a NaN selects its first NaN as argmin
 *    and argmax.  TSDS_NAN_IGNORE: NaNs are skipped; an all-NaN bin selects
 *    its first index.
 *  - LTTB keeps the first and last point and picks one point in each of
 *    n_out-2 buckets over the interior (bucket j covers points
 *    [1+floor(j(m-2)/B), 1+floor((j+1)(m-2)/B))), maximising the doubled
 *    triangle area |(xa-xm)(yb-ya) - (xa-xb)(ym-ya)| in binary64 with every
 *    operation rounded and no fused multiply-add, where a is the previous
 *    pick and (xm, ym) the next bucket's mean (index-order binary64 sums
 *    divided by the count) or, after the last bucket, the last point.  x is
 *    the point's x converted to binary64, or its index.
 */
#ifndef TSDS_H
#define TSDS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The eleven element types of the paper's ArgMinMax (Section 2.1). */
typedef enum {
  TSDS_I8 = 0, TSDS_I16 = 1, TSDS_I32 = 2, TSDS_I64 = 3,
  TSDS_U8 = 4, TSDS_U16 = 5, TSDS_U32 = 6, TSDS_U64 = 7,
  TSDS_F16 = 8, TSDS_F32 = 9, TSDS_F64 = 10
} tsds_dtype;

typedef enum { TSDS_NAN_PROPAGATE = 0, TSDS_NAN_IGNORE = 1 } tsds_nan_mode;

typedef enum {
  TSDS_OK = 0,
  TSDS_EINVAL = 1,    /* an argument outside what the algorithm defines */
  TSDS_ENOMEM = 2,    /* device memory could not be allocated (scratch pool, plan) */
  TSDS_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
  TSDS_ETIMEOUT = 4,  /* a bounded device-side wait ran out */
  TSDS_EINTERNAL = 5  /* a device-side consistency check failed */
} tsds_status;

/* MinMax (Section 1; per-bin argmin/argmax of Section 2.1).
 * n >= 0; n_out even and >= 2.  Selects at most n_out indices. */
tsds_status tsds_minmax(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                        int64_t n, int64_t n_out, tsds_nan_mode nan, int64_t* out,
                        int64_t* out_count, void* stream);

/* M4 (Section 1): first, argmin, argmax and last of each bin.
 * n >= 0; n_out a positive multiple of 4. */
tsds_status tsds_m4(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                    int64_t n, int64_t n_out, tsds_nan_mode nan, int64_t* out,
                    int64_t* out_count, void* stream);

/* LTTB (Section 1; sequential over buckets, Table 1 caption).
 * n >= 0; n_out >= 3.  Selects exactly min(n, n_out) indices. */
tsds_status tsds_lttb(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                      int64_t n, int64_t n_out, tsds_nan_mode nan, int64_t* out,
                      int64_t* out_count, void* stream);

/* MinMaxLTTB (Section 1): MinMax over the interior points 1..n-2 with
 * 2*floor(n_out*minmax_ratio/2) selections, plus the first and last point,
 * then LTTB over those points (with their original x or index).
 * n >= 0; n_out >= 3; minmax_ratio >= 1.  Selects min(n, n_out) indices
 * unless the preselection itself returns fewer than n_out points. */
tsds_status tsds_minmaxlttb(const void* x, tsds_dtype x_dtype, const void* y,
                            tsds_dtype y_dtype, int64_t n, int64_t n_out,
                            int64_t minmax_ratio, tsds_nan_mode nan, int64_t* out,
                            int64_t* out_count, void* stream);

/* Part of MinMax / M4 by bin range (Section 2.2: bins are independent, which
 * is what lets the paper run them on separate threads).  With the bins laid
 * out over the whole series exactly as tsds_minmax / tsds_m4 lay them out
 * (nb = n_out/2 or n_out/4), writes what bins [bin_lo, bin_hi) select, in
 * order, to out (capacity 2*(bin_hi-bin_lo) or 4*(bin_hi-bin_lo) indices, global
 * into the whole series) and the count to *out_count.  Concatenating the
 * outputs of consecutive ranges that cover [0, nb) gives the whole output, so
 * ranks that each hold the series can split its bins and gather the lists
 * (the Python helper paper_2307_05389_gb300.shard does this).  Only the y of
 * the range's bins is read.  TSDS_EINVAL when n_out is not a valid MinMax/M4
 * n_out, when n_out >= n (the output is every index, with no bins), or when
 * the range is not inside [0, nb); bin_lo == bin_hi writes a count of 0. */
tsds_status tsds_minmax_bins(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                             int64_t n, int64_t n_out, int64_t bin_lo, int64_t bin_hi, tsds_nan_mode nan,
                             int64_t* out, int64_t* out_count, void* stream);
tsds_status tsds_m4_bins(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                         int64_t n, int64_t n_out, int64_t bin_lo, int64_t bin_hi, tsds_nan_mode nan,
                         int64_t* out, int64_t* out_count, void* stream);

/* Host-buffer form of MinMax and M4 (the paper's downsample([x], y, n_out),
 * Section 2.3, on a series in host memory), for one or more of them over the
 * same series, returning the indices in host memory.
 *   count                 number of algorithms, 1..16;
 *   algos[i], n_outs[i]   TSDS_ALGO_MINMAX or TSDS_ALGO_M4 and its n_out (a
 *                         positive multiple of 2 or 4; n_out >= n returns
 *                         every index, as tsds_minmax/tsds_m4 do);
 *   x, x_dtype            optional sorted x (NULL: index bins), either device
 *                         memory or page-locked host memory; it is read in
 *                         place by the bin search, which probes about log2(n)
 *                         values per bin, so it is never copied;
 *   y_host, y_dtype, n    y in host memory (page-locked memory lets the copies
 *                         overlap the reduction; pageable memory works too);
 *   y_dev                 optional device buffer of n * size(y_dtype) bytes,
 *                         aligned to the element size, that receives y (it
 *                         holds y on return); NULL: the library takes one from
 *                         its pool for the call;
 *   outs_host[i]          host buffer for min(n_outs[i], n) int64 indices;
 *   counts_host[i]        receives how many were written.
 * y goes to the device in chunks (an eighth of it, between 16 and 256 MB) on
 * a private stream that first waits for the work already queued on `stream`;
 * after each chunk, the bins whose points have all arrived are reduced on
 * `stream` (bin ranges, as in tsds_minmax_bins), so the copy and the
 * reduction overlap; the ranges' outputs are joined on the host in bin order.
 * The result equals tsds_minmax / tsds_m4 on the same series.  Synchronous:
 * returns when every output is in host memory (`stream` is synchronised).
 * Errors: TSDS_EINVAL for the argument errors of tsds_minmax/tsds_m4, for a
 * count, algorithm, NULL output or misaligned y_dev, and for an x that is
 * pageable host memory (checked before any device work); CUDA failures as in
 * the other calls; a device-side failure of the streaming pass is returned as
 * its status. */
tsds_status tsds_downsample_host(int count, const int* algos, const int64_t* n_outs, const void* x,
                                 tsds_dtype x_dtype, const void* y_host, tsds_dtype y_dtype, int64_t n,
                                 tsds_nan_mode nan, void* y_dev, int64_t* const* outs_host, int64_t* counts_host,
                                 void* stream);

/* EveryNth (Section 1 names it among the algorithms; reading): the n_out bins
 * MinMax/M4 lay out (index space without x: bin i starts at
 * ceil(i(n-1)/n_out); equal-width x ranges with x) and the first point of
 * every non-empty bin, so exactly n_out points without x.  No y value is
 * read (y is still required, for a uniform interface, and nan is accepted
 * and unused).  n >= 0; n_out >= 1. */
tsds_status tsds_everynth(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                          int64_t n, int64_t n_out, tsds_nan_mode nan, int64_t* out,
                          int64_t* out_count, void* stream);

/* The same algorithms with the selected points' values gathered in the
 * kernel that writes the indices, so that a plot gets (x, y) pairs without a
 * further pass (Section 3, Listing 2: the selected indices are used to fetch
 * the subset of the series that is drawn).  Besides out[i]: y_out[i] = y[out[i]] (raw
 * elements of y_dtype) and x_out[i] = x[out[i]] (raw elements of x_dtype),
 * for i < *out_count.  Either pointer may be NULL (no copy); x_out needs x
 * (without x the index is the x value).  y_out / x_out are device buffers of
 * the capacity out has, aligned to their element size; TSDS_EINVAL
 * otherwise.  Other arguments, results and errors as in the plain calls. */
tsds_status tsds_minmax_values(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                               int64_t n, int64_t n_out, tsds_nan_mode nan, int64_t* out,
                               int64_t* out_count, void* x_out, void* y_out, void* stream);
tsds_status tsds_m4_values(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                           int64_t n, int64_t n_out, tsds_nan_mode nan, int64_t* out,
                           int64_t* out_count, void* x_out, void* y_out, void* stream);
tsds_status tsds_lttb_values(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                             int64_t n, int64_t n_out, tsds_nan_mode nan, int64_t* out,
                             int64_t* out_count, void* x_out, void* y_out, void* stream);
tsds_status tsds_minmaxlttb_values(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                                   int64_t n, int64_t n_out, int64_t minmax_ratio, tsds_nan_mode nan,
                                   int64_t* out, int64_t* out_count, void* x_out, void* y_out,
                                   void* stream);
tsds_status tsds_everynth_values(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                                 int64_t n, int64_t n_out, tsds_nan_mode nan, int64_t* out,
                                 int64_t* out_count, void* x_out, void* y_out, void* stream);

/* ---- Batched form: many series of one dtype in one launch sequence.
 *
 * The paper parallelises one series over CPU threads (Section 2.2, the
 * `parallel` option of Section 2.3).  Here a batch of series shares one
 * streaming launch: every series' y is cut into windows that the GPU's warps
 * claim from one counter, whatever series they belong to, so thousands of
 * small and large series cost one launch sequence instead of one each. */

typedef enum { TSDS_ALGO_MINMAX = 0, TSDS_ALGO_M4 = 1 } tsds_algo;

/* One series of a batch.  x, y, out and out_count are device pointers owned
 * by the caller, with the same meaning as in tsds_minmax; either every series
 * of a batch has x or none has.  n_out follows the algorithm's rule. */
typedef struct {
  const void* x;
  const void* y;
  int64_t n;
  int64_t n_out;
  int64_t* out;
  int64_t* out_count;
} tsds_series;

/* MinMax or M4 of every series in `series` (a host array of `count`
 * descriptors), asynchronously on `stream`; each series' indices and count
 * are exactly those of the single-series call.  1 <= count <= 65535.
 * Scratch comes from the library's stream-ordered pool.  TSDS_EINVAL names
 * the offending series. */
tsds_status tsds_batched(tsds_algo algo, const tsds_series* series, int64_t count,
                         tsds_dtype x_dtype, tsds_dtype y_dtype, tsds_nan_mode nan, void* stream);

/* MinMaxLTTB of every series in `series` (a host array of `count`
 * descriptors; n_out >= 3 each, minmax_ratio and nan shared) in one launch
 * sequence, asynchronously on `stream`: the MinMax preselection of every
 * series' interior shares the binned launches, and the LTTB pass of every
 * series runs as one job of each LTTB kernel (Section 1: the preselection
 * keeps LTTB's cost low; Section 2.2: many series at once instead of one at
 * a time).  Each series' indices and count are exactly those of
 * tsds_minmaxlttb on that series, and each out needs the room that call's
 * out needs (n_out indices, or n when n_out >= n).  1 <= count <= 65535.  The descriptors are
 * staged from pageable memory, so the call may wait for earlier work on
 * `stream` before it returns.  TSDS_EINVAL names the offending series. */
tsds_status tsds_batched_minmaxlttb(const tsds_series* series, int64_t count, tsds_dtype x_dtype,
                                    tsds_dtype y_dtype, int64_t minmax_ratio, tsds_nan_mode nan, void* stream);

/* A plan keeps a batch's descriptors and scratch resident so the same batch
 * (same buffers; their contents may change between executions) can be
 * downsampled again with one call.  Flags: */
#define TSDS_PLAN_GRAPH 1    /* replay the launch sequence as one CUDA graph */
#define TSDS_PLAN_AUTOTUNE 2 /* time the candidate window sizes / CTAs per SM on
                                this batch and keep the fastest; results are
                                cached per workload class for the process and,
                                when TSDS_TUNE_CACHE names a file, in that file */
typedef struct tsds_plan_s* tsds_plan;

/* Creates a plan (allocates its device scratch with cudaMalloc, uploads the
 * descriptors, autotunes and captures the graph if asked; synchronises
 * `stream`).  *plan is NULL on failure. */
tsds_status tsds_plan_create(tsds_plan* plan, tsds_algo algo, const tsds_series* series, int64_t count,
                             tsds_dtype x_dtype, tsds_dtype y_dtype, tsds_nan_mode nan, int flags,
                             void* stream);

/* Enqueues one execution of the plan on `stream`.  Executions of one plan
 * share its scratch: do not let two of them overlap on the GPU. */
tsds_status tsds_plan_execute(tsds_plan plan, void* stream);

/* The launch shape the plan uses and its sizes (any pointer may be NULL):
 * window bytes, CTAs per SM (0: as many as fit), windows, scratch bytes, and
 * the kernel variant of the streaming pass it runs (1, 2 or 3 as in
 * tsds_stream_variant). */
tsds_status tsds_plan_info(tsds_plan plan, int64_t* window_bytes, int* ctas_per_sm, int64_t* windows,
                           int64_t* scratch_bytes, int* variant);

/* Waits for the device to finish queued work, then frees the plan. */
tsds_status tsds_plan_destroy(tsds_plan plan);

/* ---- Served form: viewport queries over resident series.
 *
 * Interactive exploration re-downsamples the visible range on every zoom or
 * pan (Section 1).  A server keeps series resident (caller-owned device
 * memory), accepts queries at any time from any thread, and runs them in
 * batches on `streams` CUDA streams: whenever a batch finishes, queued
 * queries join the next batch as far as `max_batch` and the device-memory
 * budget allow (continuous batching), so a query's result is the same alone
 * or in a mix.  Results are the indices (into the whole series) that the
 * single-series call returns on the selected range, copied to host memory. */

#define TSDS_ALGO_MINMAXLTTB 2   /* third algorithm code accepted by the server */

typedef struct {
  int32_t streams;        /* batches in flight at once, 1..16 (default 2) */
  int32_t max_batch;      /* queries per batch, 1..4096 (default 256) */
  int64_t memory_budget;  /* device scratch bytes the in-flight batches may hold (default 1 GiB);
                             a query larger than the budget runs alone */
} tsds_server_config;

typedef struct {
  int64_t series;         /* id from tsds_server_add_series */
  int32_t algo;           /* TSDS_ALGO_MINMAX, TSDS_ALGO_M4 or TSDS_ALGO_MINMAXLTTB */
  int32_t nan;            /* tsds_nan_mode */
  int32_t by_x;           /* 1: points with x_lo <= x <= x (compared as binary64); 0: indices [lo, hi) */
  int32_t reserved;
  double x_lo, x_hi;
  int64_t lo, hi;
  int64_t n_out;          /* the algorithm's n_out rule applies */
  int64_t minmax_ratio;   /* MinMaxLTTB only, >= 1 */
} tsds_query;

typedef struct {
  int64_t submitted, completed, batches;
  int64_t points, bytes;  /* points (and bytes of y) inside the completed queries' ranges */
  double span_s;          /* first submission to last completion */
  double p50_us, p99_us, mean_us, max_us;  /* submission-to-completion latency */
} tsds_server_stats;

typedef struct tsds_server_s* tsds_server;

/* Starts a server on the current device (cfg may be NULL for the defaults).
 * All series of a server share y_dtype and x_dtype (x_dtype is ignored when
 * the series have no x). */
tsds_status tsds_server_create(tsds_server* server, const tsds_server_config* cfg, tsds_dtype x_dtype,
                               tsds_dtype y_dtype);

/* Registers a resident series (device pointers kept until tsds_server_destroy;
 * x sorted non-decreasing or NULL; every series of a server has x or none). */
tsds_status tsds_server_add_series(tsds_server server, const void* x, const void* y, int64_t n, int64_t* id);

/* Queues a query; returns at once with a ticket.  Thread-safe. */
tsds_status tsds_server_submit(tsds_server server, const tsds_query* query, int64_t* ticket);

/* Result of a ticket.  timeout_us: 0 = do not wait, < 0 = wait until done,
 * > 0 = wait at most that long.  *done = 1 when finished, then the indices
 * (at most the query's n_out) are copied to `out` (host memory, capacity
 * `cap`), *count and *latency_us (submission to completion) are set and the
 * ticket is released. */
tsds_status tsds_server_result(tsds_server server, int64_t ticket, int64_t timeout_us, int64_t* out, int64_t cap,
                               int64_t* count, int* done, double* latency_us);

tsds_status tsds_server_stats_get(tsds_server server, tsds_server_stats* stats);
tsds_status tsds_server_reset_stats(tsds_server server);

/* Finishes queued and running queries, then stops the server. */
tsds_status tsds_server_destroy(tsds_server server);

/* MinMax without allocating (the paper has no counterpart: it exists for
 * callers of this library that cannot allocate device memory during a call,
 * e.g. code whose device memory is wholly owned by another allocator, or a
 * latency-bound redraw loop where cudaMalloc/cudaFree may synchronise the
 * device).  Same arguments, semantics and results as tsds_minmax, but the
 * scratch memory is a fixed 8 MiB array compiled into the library (held by
 * every device that loads the library until the process exits) and the call
 * makes no allocation of any kind.
 *  - Size limit: the scratch needs about (n_out/2)*28 + 64*ceil(n*sizeof(y)/65536)
 *    bytes; a call that needs more than 8 MiB returns TSDS_EINVAL with the
 *    sizes in tsds_last_error() before touching the device (at n_out = 2000
 *    about 8 GB of y fit).
 *  - The first call on a device, with that device current, looks up the
 *    array's device address (cudaGetSymbolAddress); make that first call
 *    before any stream capture.  The address is kept until tsds_shutdown:
 *    after a reset of the device (cudaDeviceReset) call tsds_shutdown
 *    before the next call, so that the address is looked up again.
 *  - Every call shares the one array and clears the parts that must start at
 *    zero; calls whose work overlaps on the GPU (other streams, other
 *    threads) race on it and give wrong results.  Serialise them. */
tsds_status tsds_minmax_noalloc(const void* x, tsds_dtype x_dtype, const void* y,
                                tsds_dtype y_dtype, int64_t n, int64_t n_out, tsds_nan_mode nan,
                                int64_t* out, int64_t* out_count, void* stream);

/* Message for the calling thread's last failed call ("" if none). */
const char* tsds_last_error(void);

/* Releases the scratch pools of every device the library touched and forgets
 * the per-device state (the static scratch address of tsds_minmax_noalloc,
 * launch-shape caches).  Work still queued on streams must have completed.
 * Later calls re-create them.  Call it after a device reset before using the
 * library on that device again. */
void tsds_shutdown(void);

/* Library version, "major.minor.patch". */
const char* tsds_version(void);

/* ---- tracing (the paper reports median wall times, Section 4; these give
 * the device-side view of the same work). */

/* Number of CUDA kernels this library has launched in the process so far. */
int64_t tsds_kernel_launches(void);

/* on != 0: every later MinMax/M4 streaming argmin/argmax launch (also the
 * MinMaxLTTB preselection) is bracketed by two CUDA events recorded on the
 * call's stream.  Recording adds no synchronisation. */
void tsds_timing_enable(int on);

/* Failure-detection check: runs one kernel whose shared-memory barrier wait
 * is never satisfied and gives up after `rounds` bounded wait rounds, the same
 * way the streaming pass gives up on a copy that never lands; returns the
 * status the kernel recorded (TSDS_ETIMEOUT when the bound works).  Nothing is
 * copied and the context stays usable.  Synchronises `stream`.  When the
 * streaming pass itself records a timeout, the affected call reports
 * *out_count = -TSDS_ETIMEOUT. */
tsds_status tsds_check_wait_timeout(unsigned rounds, void* stream);

/* Kernel variant of the streaming argmin/argmax pass for every later call in
 * the process (no counterpart in the paper, whose CPU kernel has one form):
 *   0  automatic (the default).  Single-series calls of at most 256 MB: a
 *      warp per bin in one launch with bins of at least 8 KB (or at most 4096
 *      bins of at most 64 KB), else variant 4 below 8 KB mean bins and
 *      variant 2 above; larger calls: variant 4 below 64 KB mean bins,
 *      variant 2 above.
 *      Batches and served queries: series or queries are grouped by bin size
 *      (variant 4 below 64 KB for batches without x and below 32 KB for
 *      queries, a warp per bin from there up to 64 KB, variant 2 above;
 *      batches with x take variant 3 below 768 bytes (8-byte y), 1.5 KB
 *      (4-byte), 1 KB (2-byte) or 512 bytes (1-byte), a warp per bin up to
 *      64 KB);
 *   1  shared-memory ring (bulk async copies into shared memory, one warp
 *      per bin);
 *   2  register streaming, one warp per bin;
 *   3  segmented: y staged through shared memory by per-lane async copies,
 *      bins split across lanes;
 *   4  lane groups: each bin reduced whole by a group of 1 to 32 lanes
 *      (single-series calls; bins above 64 KB are handed to variant 2).
 * The environment variable TSDS_STREAM_VARIANT=ring|ldg|seg|grp sets 1 to 4
 * when the library loads.  Results are identical; only speed differs.
 * Batched plans that were tuned keep the variant they chose.  Returns the
 * previous setting, or -1 (and sets nothing) when `variant` is not 0..4. */
int tsds_stream_variant(int variant);

/* Waits for the launches recorded since the previous read, writes the sum of
 * their device durations in milliseconds to *total_ms (may be NULL) and their
 * number to *launches (may be NULL), and forgets them.  TSDS_ECUDA if an
 * event query fails. */
tsds_status tsds_timing_read(double* total_ms, int64_t* launches);

/* Failure injection for tests: the next `count` device allocations the
 * library makes (its stream-ordered scratch and the memory of a new plan)
 * fail as if the device were out of memory, without allocating, and the
 * calls that needed them return TSDS_ENOMEM.  Work a call had already
 * enqueued before the failed allocation still runs; its outputs are then
 * unspecified.  count <= 0 clears the injection. */
void tsds_inject_alloc_failures(int count);

/* Checked mode.  When on, every entry point that takes x (the single-series
 * calls and their *_values forms, tsds_lttb_means, tsds_batched,
 * tsds_plan_create, tsds_server_add_series) first verifies on the device that
 * x is sorted non-decreasing with no NaN (one extra read of x), waits for the
 * answer on the call's stream (the legacy default stream for
 * tsds_server_add_series) and returns TSDS_EINVAL, naming the first position
 * i where x[i] is NaN or x[i] > x[i+1], before launching anything else.
 * tsds_minmax_noalloc is never checked (it takes no scratch).  The mode starts
 * on when the environment variable TSDS_CHECKED is set to anything but "0"
 * when the library loads.  on = 0 or 1 sets the mode, on < 0 leaves it;
 * returns the mode before the call. */
int tsds_checked(int on);

/* Measurement aid: the read-only streaming ceiling.  The per-bin pass reads
 * each y element once and writes next to nothing (Section 2.1: one pass over
 * the data, bound by memory), so besides the copy bandwidth its speed is set
 * against this kernel, which does only that: it reads the `bytes` bytes at
 * `buf` (device memory, 16-byte aligned, bytes a multiple of 16) once with
 * 16-byte loads over a grid of a few CTAs per SM and XORs the XOR of all its
 * 8-byte little-endian words into *sink (one device uint64, not cleared
 * first).  The XOR makes every load observable.  Enqueued on `stream`;
 * bytes == 0 launches nothing.  TSDS_EINVAL (nothing launched) when bytes is
 * negative or not a multiple of 16, buf is null or misaligned with bytes > 0,
 * or sink is null. */
tsds_status tsds_read_stream(const void* buf, int64_t bytes, uint64_t* sink, void* stream);

/* Diagnostic: the bucket averages an LTTB call with the same arguments uses
 * (Section 1: the third point of each step's triangle is the average of the
 * next bucket).  Bucket j of B = n_out - 2 covers points
 * [1 + floor(j(n-2)/B), 1 + floor((j+1)(n-2)/B)); its average is the binary64
 * sum of its x (or index) and y values in index order, each divided by the
 * count (NaN-ignore leaves out points whose y is NaN).  Writes the averages of
 * buckets 1 .. B-1 to `means` (device memory, 2*(n_out-3) doubles: x then y of
 * each bucket), enqueued on `stream`.  Needs 3 <= n_out < n; TSDS_EINVAL
 * otherwise (nothing written). */
tsds_status tsds_lttb_means(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                            int64_t n, int64_t n_out, tsds_nan_mode nan, double* means, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TSDS_H */
