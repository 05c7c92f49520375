// internal.h -- structures shared by the host runtime and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tsds.h"

namespace tsds {

// Bytes of y one warp claims at a time in the streaming argmin/argmax pass.
constexpr int64_t kWindowBytes = 64 * 1024;
constexpr int kStreamThreads = 256;   // 8 warps per CTA

// EVERYNTH: the first point of each non-empty bin (no argmin/argmax pass).
enum Algo : int { ALGO_MINMAX = 0, ALGO_M4 = 1, ALGO_EVERYNTH = 2 };

// Optional fused value gather: beside each index the kernel that writes
// out[i] also copies the selected point's raw y element to y_out[i] and its
// raw x element to x_out[i] (either pointer may be null).
struct Gather {
  void* y_out;
  void* x_out;
  int y_size;
  int x_size;
};

// One series as the binned kernels see it.  For a single call there is one;
// the batched launch passes an array.
struct SeriesDev {
  const void* y;
  const void* x;
  int64_t n;          // points
  int64_t nb;         // bins (0: the series returns every index)
  int64_t* edges;     // nb+1 bin starts, edges[nb] = n
  int64_t* res;       // 2*nb: per-bin argmin, argmax (global indices of this series)
  uint32_t* cnt;      // nb: pieces of the bin finished so far (zero between calls)
  int64_t win_base;   // first window of this series in the launch's window numbering
  int64_t* out;       // output indices
  int64_t* out_count; // device count
  int64_t idx_bias;   // added to every index written (1 for the MinMaxLTTB interior)
  const unsigned long long* status;  // device status word of the streaming pass (null: none);
                                     // non-zero makes emit report -status as the count
  Gather g;           // values written beside the indices (y[v], x[v] for index v + idx_bias)
  int32_t mode;       // batched: 0 the series is cut into windows; 1 a warp per bin, and
                      // win_base is its first CTA in that launch (kBinsPerCta bins each);
                      // 2 lane groups (no windows); 3 lane groups, with windows for the
                      // bins above the lane-group size limit
  int32_t grp;        // modes 2 and 3: the lane-group shape, g_log2 | tile_rounds << 8
  int64_t tile_base;  // modes 2 and 3: first tile of the series in the lane-group launch
};

// Partial argmin/argmax of one bin piece: ordered 64-bit keys plus indices.
struct Piece {
  uint64_t kmin;
  int64_t imin;
  uint64_t kmax;
  int64_t imax;
};

struct WorkCounters {
  unsigned long long next_window;
  unsigned long long status;   // tsds_status of a device-side failure (TSDS_ETIMEOUT), 0 when fine
  unsigned long long large;    // lane-group pass: bins it left to the windowed pass (too large)
  unsigned long long pad[5];
};

inline int64_t dtype_size(tsds_dtype d) {
  switch (d) {
    case TSDS_I8: case TSDS_U8: return 1;
    case TSDS_I16: case TSDS_U16: case TSDS_F16: return 2;
    case TSDS_I32: case TSDS_U32: case TSDS_F32: return 4;
    default: return 8;
  }
}
inline bool dtype_valid(int d) { return d >= TSDS_I8 && d <= TSDS_F64; }
inline bool dtype_is_float(tsds_dtype d) { return d == TSDS_F16 || d == TSDS_F32 || d == TSDS_F64; }

inline int64_t window_elems(tsds_dtype y_dtype) { return kWindowBytes / dtype_size(y_dtype); }

// Variants of the streaming pass: RING stages y through a shared-memory ring
// filled by bulk async copies, LDG streams it through registers with one warp
// per bin (cheapest per byte: large bins), SEG stages it through per-lane
// async copies and splits bins across lanes (cheapest per bin: small bins).  AUTO picks SEG when the bytes-weighted mean bin size is below
// seg_max_bin_bytes(element size), LDG otherwise (crossovers measured on
// GB300 over 1 GB and 40 MB inputs).
enum StreamVariant : int { STREAM_AUTO = 0, STREAM_RING = 1, STREAM_LDG = 2, STREAM_SEG = 3, STREAM_GRP = 4 };
inline int64_t seg_max_bin_bytes(int64_t elem_bytes) {
  return elem_bytes == 8 ? 768 : elem_bytes == 4 ? 1536 : elem_bytes == 2 ? 1024 : 512;
}

// Launch shape of the streaming pass (the batched plans autotune it).
struct StreamConfig {
  int64_t window_bytes = kWindowBytes;  // bytes of y per warp claim: a multiple of 4096
  int ctas_per_sm = 0;                  // 0: as many as fit
  // When set, the number of windows is read from device memory here (the
  // server resolves query ranges on the device) and the full persistent grid
  // is launched.
  const int64_t* total_windows_dev = nullptr;
  int variant = STREAM_AUTO;
  int64_t mean_bin_bytes = 0;           // bytes-weighted mean bin size of the launch
  int64_t window_first = 0;             // the launch takes windows [window_first, total_windows)
  const int64_t* window_first_dev = nullptr;   // when set, window_first is read here on the device
  // Register streaming after the lane-group pass: only bins of more than
  // min_bin points, and nothing at all when *large_dev is zero.
  int64_t min_bin = 0;
  const unsigned long long* large_dev = nullptr;
  // Batched plans: lanes per bin of the lane-group series, 2^grp_scale times
  // the default choice, and bins per lane-group tile, 2^grp_tile_scale times
  // the default (autotuner dimensions).
  int grp_scale = 0;
  int grp_tile_scale = 0;
};
// A mean_bin_bytes at which the register-streaming pass never prefetches.
constexpr int64_t kPrefetchOffBinBytes = 1ll << 40;

// The lane-group pass (stream_grp.cuh): groups of 2^g_log2 lanes, tiles of
// (32 >> g_log2) * tile_rounds consecutive bins claimed through
// work->next_window.  Bins of more than max_bin points are left out and
// counted in work->large (max_bin 0: none is left out).  Single series: s_dev
// null; batched: tile_series maps tiles to series (win_base = first tile).
constexpr int kGrpTileMaxBins = 128;   // bins per lane-group tile at most
// vectors a lane loads before it uses any of them: 16 for elements of up to
// 4 bytes, 8 for 8-byte elements (whose 64-bit keys take twice the registers)
constexpr int kGrpU = 16;
constexpr int kGrpU64 = 8;
__host__ __device__ constexpr int grp_unroll(int64_t elem_bytes) { return elem_bytes == 8 ? kGrpU64 : kGrpU; }
// Bins above this size are left to the windowed register-streaming pass (a
// group reads a bin at a few GB/s, so one huge x-space bin would otherwise
// hold up the launch).
constexpr int64_t kGrpMaxBinBytes = 64 * 1024;
struct GrpShape {
  int g_log2 = 0;
  int tile_rounds = 1;
  int64_t max_bin = 0;
};
// Lane-group shape for a launch whose bins average mean_bin_bytes: groups of
// G lanes whose 4*G*U vectors (U = grp_unroll) cover a bin's interior (a bin's first and
// last vector are taken apart; on GB300 four rounds of loads per lane
// measured 10-20 % faster than two from 1 KB bins on, and two lanes per bin
// 11 % faster than one at 512-byte bins; the per-bin work then weighs less
// against the streaming), tiles of
// about 16 KB (a tile of bins below 4 KB has its bytes requested into L2 when
// it starts: with 32 KB tiles the requests in flight outgrew L2 and 31 % of
// the lines were fetched twice; 16 KB tiles measured 1.008x the bytes of y).
__host__ __device__ inline GrpShape grp_shape(int64_t mean_bin_bytes, int64_t elem_bytes) {
  GrpShape g;
  const int64_t inner = mean_bin_bytes / 16 - 1;
  int lg = 0;
  while (lg < 5 && ((int64_t)grp_unroll(elem_bytes) << (lg + 2)) < inner) ++lg;
  if (lg == 0 && inner > 16) lg = 1;   // bins of 384 bytes and more: at least two lanes
  g.g_log2 = lg;
  const int64_t groups = 32 >> lg;
  int64_t rounds = (16 * 1024) / (groups * (mean_bin_bytes > 0 ? mean_bin_bytes : 1));
  const int64_t max_rounds = kGrpTileMaxBins / groups;
  g.tile_rounds = (int)(rounds < 1 ? 1 : rounds > max_rounds ? max_rounds : rounds);
  g.max_bin = kGrpMaxBinBytes / elem_bytes;
  return g;
}
// SeriesDev::grp of a shape.
__host__ __device__ inline int32_t grp_pack(int g_log2, int tile_rounds) { return g_log2 | (tile_rounds << 8); }
// Whether a single-series windowed call with this mean bin size takes the
// lane-group pass (automatic choice below kGrpAutoMaxBinBytes, or forced by
// tsds_stream_variant(STREAM_GRP)).
constexpr int64_t kGrpAutoMaxBinBytes = 8 * 1024;
// (bytes: y of the call; beyond 256 MB the limit is kGrpAutoMaxBinBytesLarge)
constexpr int64_t kGrpAutoMaxBinBytesLarge = 64 * 1024;
// Batches without x: series whose bins average below this run in the
// lane-group pass (the 4096-series batch measured 2.68 ms for MinMax on GB300
// with this limit, 2.91 ms with 8 KB and a warp per bin above).
constexpr int64_t kGrpBatchedMaxBinBytes = 64 * 1024;
// Served queries: bins below this run in the lane-group pass (x-space bins;
// larger bins of such a query go to the windowed pass).
constexpr int64_t kGrpServedMaxBinBytes = 32 * 1024;
bool grp_call(int64_t mean_bin_bytes, int64_t bytes, bool has_x);
cudaError_t launch_argminmax_grp(const SeriesDev* s_dev, const SeriesDev& single, const int32_t* tile_series,
                                 int64_t total_tiles, WorkCounters* work, tsds_dtype y_dtype, tsds_nan_mode nan,
                                 const GrpShape& shape, cudaStream_t st, const int64_t* total_dev = nullptr,
                                 int sm_count = 0);

// The variant a launch with this shape runs for elements of elem_bytes.
int stream_variant_for(const StreamConfig& cfg, int64_t elem_bytes);

// ---- launchers (each returns the launch's cudaError_t)

// Bin starts for every series in `s` (count series, array in device memory
// or, for count == 1, also usable by value).
cudaError_t launch_edges(const SeriesDev* s_dev, int count, const SeriesDev* s_host_single,
                         bool has_x, tsds_dtype x_dtype, int64_t max_nb, cudaStream_t st);

// Window -> series map for a batched launch (window_bytes as in StreamConfig).
cudaError_t launch_window_map(const SeriesDev* s_dev, int count, int32_t* win_series,
                              tsds_dtype y_dtype, cudaStream_t st, int64_t window_bytes = kWindowBytes);

// The streaming per-bin argmin/argmax pass.
cudaError_t launch_argminmax(const SeriesDev* s_dev, int count, const SeriesDev& single,
                             const int32_t* win_series, int64_t total_windows,
                             Piece* first_piece, Piece* last_piece, WorkCounters* work,
                             tsds_dtype y_dtype, tsds_nan_mode nan, cudaStream_t st,
                             const StreamConfig& cfg = StreamConfig());

// The same pass for one series with the SM count given by the caller instead
// of the library's per-device state (for the entry point that must not create
// the library's memory pool).
cudaError_t launch_argminmax_sm(const SeriesDev& single, int64_t total_windows, Piece* first_piece,
                                Piece* last_piece, WorkCounters* work, tsds_dtype y_dtype, tsds_nan_mode nan,
                                const StreamConfig& cfg, int sm_count, cudaStream_t st);

// Single-series calls with bins of at most 64 KB on average, no explicit
// streaming variant, and either at most 256 MB of y (at most 4096 bins, or
// bins of at least 8 KB) or bins of at least 8 KB (with x; 32 KB without): a
// warp per bin in one
// launch (index-bin starts in the kernel,
// x-space starts from launch_edges first).  With emit (at most
// kSmallEmitMaxBins bins) the last CTA also emits, with `done` a zeroed
// counter; otherwise launch_emit / launch_emit_tiled follow.
constexpr int64_t kSmallMaxBinBytes = 64 * 1024;
constexpr int64_t kSmallMaxBytes = 256ll << 20;
constexpr int64_t kSmallEmitMaxBins = 1024;
bool small_call(int64_t n, int64_t nb, tsds_dtype y_dtype, bool has_x);
cudaError_t launch_small(const SeriesDev& S, tsds_dtype y_dtype, tsds_nan_mode nan, Algo algo, bool has_x,
                         unsigned* done, bool emit, cudaStream_t st);

// A kernel whose barrier wait nothing satisfies, bounded by `rounds`; writes
// the status it ends with (TSDS_ETIMEOUT) to *status.
cudaError_t launch_wait_probe(unsigned long long* status, unsigned rounds, cudaStream_t st);

// Batched series in mode 1: a warp per bin over CTAs of kBinsPerCta bins
// (cta_series maps each CTA to its series; launch_cta_map fills it).
constexpr int kBinsPerCta = 8;
cudaError_t launch_cta_map(const SeriesDev* s_dev, int count, int32_t* cta_series, cudaStream_t st);
// Batched series in modes 2 and 3 (lane groups): tile_series[tile_base + t] = the
// series, for each of its tiles (shape in SeriesDev::grp).
cudaError_t launch_tile_map(const SeriesDev* s_dev, int count, int32_t* tile_series, cudaStream_t st);
// ctas_dev (optional): the actual number of CTAs, read on the device (ctas is then a bound)
cudaError_t launch_bins_multi(const SeriesDev* s_dev, const int32_t* cta_series, int64_t ctas, tsds_dtype y_dtype,
                              tsds_nan_mode nan, cudaStream_t st, const int64_t* ctas_dev = nullptr);

// Every series with nb == 0 gets 0..n-1 (its n_out >= n) and *out_count = n.
cudaError_t launch_iota_batched(const SeriesDev* s_dev, int count, cudaStream_t st);

// Per-bin selections -> compacted, sorted output and count.
cudaError_t launch_emit(const SeriesDev* s_dev, int count, const SeriesDev& single, Algo algo,
                        cudaStream_t st);

// The same for one series with many bins, over tiles of bins on many CTAs
// (tile_count: emit_tiles(nb) int64 of scratch).
constexpr int64_t kEmitTiledMinBins = 4096;
int64_t emit_tiles(int64_t nb);
cudaError_t launch_emit_tiled(const SeriesDev& single, Algo algo, int64_t* tile_count, cudaStream_t st);

// out[i] = i for i < n, *count = n; with a gather, y_out[i] = y[i] and x_out[i] = x[i].
cudaError_t launch_iota(int64_t* out, int64_t n, int64_t* count, cudaStream_t st, const void* y = nullptr,
                        const void* x = nullptr, const Gather* g = nullptr);

int device_sm_count();

// tsds_shutdown: drop the per-device state kept outside the scratch pools
// (the static scratch address of tsds_minmax_noalloc, the occupancy caches).
void noalloc_forget_devices();
void forget_stream_occupancy();

// Checked mode (tsds_checked, TSDS_CHECKED=1): every entry point that takes x
// first verifies on the device that it is sorted non-decreasing with no NaN,
// waits for the answer and returns TSDS_EINVAL before launching anything else.
bool checked_mode();
// The smallest out-of-order position of x goes to *first_bad (left as is when
// x is in order).
cudaError_t launch_check_sorted(const void* x, tsds_dtype xd, int64_t n, unsigned long long* first_bad,
                                cudaStream_t st);
// TSDS_OK when checked mode is off, x is null, or x[0..n) is in order;
// otherwise TSDS_EINVAL naming `who` and the first bad index.  Synchronises st
// when it checks.
tsds_status check_sorted_x(const char* who, const void* x, tsds_dtype xd, int64_t n, cudaStream_t st);
tsds_status fail(tsds_status s, const char* fmt, ...);
// Checked mode over a batch: every series' x in order (one wait for all);
// TSDS_EINVAL names the series and the position.
tsds_status check_batch_sorted(const tsds_series* s, int64_t count, tsds_dtype x_dtype, cudaStream_t st);

// Reads bytes (a multiple of 16) at buf (16-byte aligned) once, 16 bytes per
// load, and XORs the XOR of its 8-byte words into *sink.
cudaError_t launch_read_stream(const void* buf, int64_t bytes, uint64_t* sink, cudaStream_t st);

// Counts every kernel this library launches (reported by tsds_kernel_launches).
void note_launch(int kernels = 1);

// Kernel timing (tsds_timing_enable): when on, the streaming argmin/argmax
// launches are bracketed by CUDA events on their stream.
bool timing_on();
void timing_begin(cudaStream_t st, void** token);
void timing_end(cudaStream_t st, void* token);

// Scratch memory taken from the library's per-device pool in stream order and
// handed back in stream order when the owning call has queued its launches.
struct Scratch {
  void* p = nullptr;
  cudaStream_t st = nullptr;
  ~Scratch() {
    if (p) cudaFreeAsync(p, st);
  }
};
cudaError_t scratch_alloc(Scratch& s, size_t bytes, cudaStream_t st);

}  // namespace tsds
