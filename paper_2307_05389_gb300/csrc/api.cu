// api.cu -- the C ABI (include/tsds.h): argument checks, the per-device
// stream-ordered scratch pool, and the launch sequence of each algorithm.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"
#include "lttb.h"

namespace tsds {

// ---------------------------------------------------------------- errors

static thread_local char g_err[512] = "";

tsds_status fail(tsds_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return s;
}

#define TSDS_CK(call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      if (e_ == cudaErrorMemoryAllocation)                                               \
        return fail(TSDS_ENOMEM, "%s: %s", #call, cudaGetErrorString(e_));               \
      return fail(TSDS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));                  \
    }                                                                                    \
  } while (0)

// ---------------------------------------------------------------- per-device state

struct DevState {
  cudaMemPool_t pool = nullptr;
  int sm_count = 0;
};
static std::mutex g_mu;
static std::map<int, DevState> g_dev;

static DevState* dev_state(cudaError_t* err) {
  int d = 0;
  *err = cudaGetDevice(&d);
  if (*err != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  DevState& s = g_dev[d];
  if (!s.pool) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = d;
    *err = cudaMemPoolCreate(&s.pool, &props);
    if (*err != cudaSuccess) { s.pool = nullptr; return nullptr; }
    uint64_t keep = ~0ull;   // keep freed blocks cached for the next call
    cudaMemPoolSetAttribute(s.pool, cudaMemPoolAttrReleaseThreshold, &keep);
    *err = cudaDeviceGetAttribute(&s.sm_count, cudaDevAttrMultiProcessorCount, d);
    if (*err != cudaSuccess) return nullptr;
  }
  return &s;
}

int device_sm_count() {
  cudaError_t e;
  DevState* s = dev_state(&e);
  return s ? s->sm_count : 148;
}

// Failure injection (tsds_inject_alloc_failures): the next g_fail_allocs
// device allocations report cudaErrorMemoryAllocation without allocating.
static std::atomic<int> g_fail_allocs{0};

bool take_injected_alloc_failure() {
  int v = g_fail_allocs.load();
  while (v > 0)
    if (g_fail_allocs.compare_exchange_weak(v, v - 1)) return true;
  return false;
}

cudaError_t scratch_alloc(Scratch& s, size_t bytes, cudaStream_t st) {
  cudaError_t e;
  DevState* d = dev_state(&e);
  if (!d) return e;
  if (take_injected_alloc_failure()) return cudaErrorMemoryAllocation;
  s.st = st;
  if (bytes == 0) bytes = 256;
  return cudaMallocFromPoolAsync(&s.p, bytes, d->pool, st);
}

// ---------------------------------------------------------------- tracing

static std::atomic<long long> g_launches{0};
static std::atomic<int> g_timing{0};
struct TimedLaunch {
  cudaEvent_t a, b;
};
static std::mutex g_tmu;
static std::vector<TimedLaunch> g_timed;
static std::vector<cudaEvent_t> g_free_events;

void note_launch(int kernels) { g_launches.fetch_add(kernels, std::memory_order_relaxed); }
bool timing_on() { return g_timing.load(std::memory_order_relaxed) != 0; }

static cudaEvent_t take_event() {
  std::lock_guard<std::mutex> lk(g_tmu);
  if (!g_free_events.empty()) {
    cudaEvent_t e = g_free_events.back();
    g_free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void timing_begin(cudaStream_t st, void** token) {
  *token = nullptr;
  if (!timing_on()) return;
  cudaEvent_t a = take_event();
  if (a && cudaEventRecord(a, st) == cudaSuccess) *token = a;
}

void timing_end(cudaStream_t st, void* token) {
  if (!token) return;
  cudaEvent_t b = take_event();
  if (!b) return;
  cudaEventRecord(b, st);
  std::lock_guard<std::mutex> lk(g_tmu);
  g_timed.push_back(TimedLaunch{static_cast<cudaEvent_t>(token), b});
}

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ---------------------------------------------------------------- argument checks

static tsds_status check_common(const void* x, int x_dtype, const void* y, int y_dtype, int64_t n,
                                int nan, const int64_t* out, const int64_t* out_count) {
  if (n < 0) return fail(TSDS_EINVAL, "n must be >= 0 (got %lld)", (long long)n);
  if (!dtype_valid(y_dtype)) return fail(TSDS_EINVAL, "unknown y dtype %d", y_dtype);
  if (x && !dtype_valid(x_dtype)) return fail(TSDS_EINVAL, "unknown x dtype %d", x_dtype);
  if (nan != TSDS_NAN_PROPAGATE && nan != TSDS_NAN_IGNORE) return fail(TSDS_EINVAL, "unknown NaN mode %d", nan);
  if (n > 0 && !y) return fail(TSDS_EINVAL, "y is NULL");
  if (!out_count) return fail(TSDS_EINVAL, "out_count is NULL");
  if (n > 0 && !out) return fail(TSDS_EINVAL, "out is NULL");
  if (y && (reinterpret_cast<uintptr_t>(y) % dtype_size((tsds_dtype)y_dtype)) != 0)
    return fail(TSDS_EINVAL, "y is not aligned to its element size");
  if (x && (reinterpret_cast<uintptr_t>(x) % dtype_size((tsds_dtype)x_dtype)) != 0)
    return fail(TSDS_EINVAL, "x is not aligned to its element size");
  return TSDS_OK;
}

// ---------------------------------------------------------------- NVTX

// A named NVTX range around each public call (visible in Nsight tools; a
// no-op when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

// ---------------------------------------------------------------- checked mode

static int checked_from_env() {
  const char* e = getenv("TSDS_CHECKED");
  return (e && e[0] && strcmp(e, "0") != 0) ? 1 : 0;
}
static std::atomic<int> g_checked{checked_from_env()};

bool checked_mode() { return g_checked.load() != 0; }

tsds_status check_sorted_x(const char* who, const void* x, tsds_dtype xd, int64_t n, cudaStream_t st) {
  if (!checked_mode() || !x || n <= 0) return TSDS_OK;
  Scratch sc;
  TSDS_CK(scratch_alloc(sc, 256, st));
  unsigned long long* word = static_cast<unsigned long long*>(sc.p);
  TSDS_CK(cudaMemsetAsync(word, 0xff, sizeof *word, st));
  TSDS_CK(launch_check_sorted(x, xd, n, word, st));
  unsigned long long bad = 0;
  TSDS_CK(cudaMemcpyAsync(&bad, word, sizeof bad, cudaMemcpyDeviceToHost, st));
  TSDS_CK(cudaStreamSynchronize(st));
  if (bad != ~0ull)
    return fail(TSDS_EINVAL, "%s: x is not sorted non-decreasing (NaN or x[i] > x[i+1] at i = %llu; checked mode)",
                who, bad);
  return TSDS_OK;
}

// ---------------------------------------------------------------- MinMax / M4

// Scratch layout of one binned call.
struct BinnedLayout {
  size_t edges, res, cnt, work, work2, first, last, tiles, total, zero_begin, zero_bytes;
};

static BinnedLayout binned_layout(int64_t nb, int64_t windows) {
  BinnedLayout L;
  size_t o = 0;
  L.tiles = o; o = align_up(o + (size_t)(nb >= kEmitTiledMinBins ? emit_tiles(nb) : 0) * 8, 256);
  L.edges = o; o = align_up(o + (size_t)(nb + 1) * 8, 256);
  L.res = o;   o = align_up(o + (size_t)nb * 16, 256);
  L.cnt = o;   o = align_up(o + (size_t)nb * 4, 256);
  L.work = o;  o = align_up(o + sizeof(WorkCounters), 256);
  L.work2 = o; o = align_up(o + sizeof(WorkCounters), 256);
  L.first = o; o = align_up(o + (size_t)windows * sizeof(Piece), 256);
  L.last = o;  o = align_up(o + (size_t)windows * sizeof(Piece), 256);
  L.total = o;
  L.zero_begin = L.cnt;
  L.zero_bytes = L.first - L.cnt;
  return L;
}

// The MinMax/M4 pipeline on one series with nb bins, writing to out/out_count
// with idx_bias added to every index.
tsds_status run_binned_series(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                              int64_t n, int64_t nb, tsds_nan_mode nan, Algo algo, int64_t* out,
                              int64_t* out_count, int64_t idx_bias, cudaStream_t st, const Gather* g) {
  if (small_call(n, nb, y_dtype, x != nullptr)) {
    // a warp per bin: one launch (after the edge search when x is given), then
    // the emit kernels when there are too many bins for the last CTA to emit
    const bool emit = nb <= kSmallEmitMaxBins;
    const size_t o_res = align_up((size_t)(nb + 1) * 8, 256);
    const size_t o_done = o_res + align_up((size_t)nb * 16, 256);
    const size_t o_tiles = o_done + 256;
    Scratch s;
    TSDS_CK(scratch_alloc(s, o_tiles + align_up((size_t)emit_tiles(nb) * 8, 256), st));
    char* base = static_cast<char*>(s.p);
    TSDS_CK(cudaMemsetAsync(base + o_done, 0, sizeof(unsigned), st));
    SeriesDev S;
    memset(&S, 0, sizeof S);
    S.y = y;
    S.x = x;
    S.n = n;
    S.nb = nb;
    S.edges = reinterpret_cast<int64_t*>(base);
    S.res = reinterpret_cast<int64_t*>(base + o_res);
    S.out = out;
    S.out_count = out_count;
    S.idx_bias = idx_bias;
    if (g) S.g = *g;
    if (x) TSDS_CK(launch_edges(nullptr, 1, &S, true, x_dtype, nb, st));
    void* tok;
    timing_begin(st, &tok);
    TSDS_CK(launch_small(S, y_dtype, nan, algo, x != nullptr, reinterpret_cast<unsigned*>(base + o_done), emit, st));
    timing_end(st, tok);
    if (!emit) {
      if (nb >= kEmitTiledMinBins) TSDS_CK(launch_emit_tiled(S, algo, reinterpret_cast<int64_t*>(base + o_tiles), st));
      else TSDS_CK(launch_emit(nullptr, 1, S, algo, st));
    }
    return TSDS_OK;
  }
  // Window size: 64 KB for large inputs; smaller (down to 4 KB, a multiple of
  // the 4 KB ring chunk) when fewer windows than about twice the resident
  // warps would leave SMs idle.
  StreamConfig cfg;
  cfg.mean_bin_bytes = nb > 0 ? n / nb * dtype_size(y_dtype) : 0;
  const bool grp = grp_call(cfg.mean_bin_bytes, n * dtype_size(y_dtype), x != nullptr);
  {
    const int64_t bytes = n * dtype_size(y_dtype);
    const int64_t warps = (int64_t)device_sm_count() * 3 * 4;
    int64_t wb = (bytes / (2 * warps) + 4095) / 4096 * 4096;
    cfg.window_bytes = wb < 4096 ? 4096 : (wb > kWindowBytes ? kWindowBytes : wb);
  }
  const int64_t welems = cfg.window_bytes / dtype_size(y_dtype);
  const int64_t windows = (n + welems - 1) / welems;
  const BinnedLayout L = binned_layout(nb, windows);
  Scratch s;
  TSDS_CK(scratch_alloc(s, L.total, st));
  char* base = static_cast<char*>(s.p);
  TSDS_CK(cudaMemsetAsync(base + L.zero_begin, 0, L.zero_bytes, st));
  SeriesDev S;
  memset(&S, 0, sizeof S);
  S.status = &reinterpret_cast<WorkCounters*>(base + L.work)->status;
  S.y = y;
  S.x = x;
  S.n = n;
  S.nb = nb;
  S.edges = reinterpret_cast<int64_t*>(base + L.edges);
  S.res = reinterpret_cast<int64_t*>(base + L.res);
  S.cnt = reinterpret_cast<uint32_t*>(base + L.cnt);
  S.win_base = 0;
  S.out = out;
  S.out_count = out_count;
  S.idx_bias = idx_bias;
  if (g) S.g = *g;
  TSDS_CK(launch_edges(nullptr, 1, &S, x != nullptr, x_dtype, nb, st));
  void* tok;
  timing_begin(st, &tok);
  if (grp) {
    // lanes-per-bin pass; bins far above the mean (possible with x) go to a
    // register-streaming pass over the windows, which skips every other bin
    // and exits at once when there is none
    GrpShape shape = grp_shape(cfg.mean_bin_bytes, dtype_size(y_dtype));
    const int64_t max_points = x ? n : (n - 1) / nb + 2;   // no x: bins differ by at most one point
    const bool large_pass = max_points > shape.max_bin;
    if (!large_pass) shape.max_bin = 0;
    const int64_t tile_bins = (int64_t)(32 >> shape.g_log2) * shape.tile_rounds;
    WorkCounters* w1 = reinterpret_cast<WorkCounters*>(base + L.work);
    TSDS_CK(launch_argminmax_grp(nullptr, S, nullptr, (nb + tile_bins - 1) / tile_bins, w1, y_dtype, nan, shape, st));
    if (large_pass) {
      cfg.variant = STREAM_LDG;
      cfg.mean_bin_bytes = kPrefetchOffBinBytes;   // the bins it reads are large: no L2 prefetch
      cfg.min_bin = shape.max_bin;
      cfg.large_dev = &w1->large;
      TSDS_CK(launch_argminmax(nullptr, 1, S, nullptr, windows, reinterpret_cast<Piece*>(base + L.first),
                               reinterpret_cast<Piece*>(base + L.last),
                               reinterpret_cast<WorkCounters*>(base + L.work2), y_dtype, nan, st, cfg));
    }
  } else {
    TSDS_CK(launch_argminmax(nullptr, 1, S, nullptr, windows, reinterpret_cast<Piece*>(base + L.first),
                             reinterpret_cast<Piece*>(base + L.last), reinterpret_cast<WorkCounters*>(base + L.work),
                             y_dtype, nan, st, cfg));
  }
  timing_end(st, tok);
  if (nb >= kEmitTiledMinBins) TSDS_CK(launch_emit_tiled(S, algo, reinterpret_cast<int64_t*>(base + L.tiles), st));
  else TSDS_CK(launch_emit(nullptr, 1, S, algo, st));
  return TSDS_OK;
}

// Bins [b0, b1) of the whole-series layout of nb bins: the bin starts of the
// whole series, then the lane-group pass over those bins only (bins above its
// size limit go to a register-streaming pass over the windows that skips
// every other bin and exits at once when there is none), then the emit of
// those bins.  Output: what those bins select, in order.
// edges: the whole series' bin starts already on the device, or null to
// compute them here.
static tsds_status run_binned_range(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                                    int64_t n, int64_t nb, int64_t b0, int64_t b1, tsds_nan_mode nan, Algo algo,
                                    int64_t* out, int64_t* out_count, cudaStream_t st, int64_t* edges = nullptr) {
  const int64_t k = b1 - b0;
  const int64_t elem = dtype_size(y_dtype);
  const int64_t welems = kWindowBytes / elem;
  const int64_t windows = (n + welems - 1) / welems;
  size_t o = 0;
  const size_t o_edges = o; o = align_up(o + (size_t)(edges ? 0 : nb + 1) * 8, 256);
  const size_t o_res = o;   o = align_up(o + (size_t)k * 16, 256);
  const size_t o_cnt = o;   o = align_up(o + (size_t)k * 4, 256);
  const size_t o_work = o;  o = align_up(o + 2 * sizeof(WorkCounters), 256);
  const size_t o_first = o; o = align_up(o + (size_t)windows * sizeof(Piece), 256);
  const size_t o_last = o;  o = align_up(o + (size_t)windows * sizeof(Piece), 256);
  const size_t o_tiles = o; o = align_up(o + (size_t)(k >= kEmitTiledMinBins ? emit_tiles(k) : 0) * 8, 256);
  Scratch s;
  TSDS_CK(scratch_alloc(s, o, st));
  char* base = static_cast<char*>(s.p);
  TSDS_CK(cudaMemsetAsync(base + o_cnt, 0, o_first - o_cnt, st));
  SeriesDev S;
  memset(&S, 0, sizeof S);
  S.y = y;
  S.x = x;
  S.n = n;
  S.nb = nb;
  S.edges = edges ? edges : reinterpret_cast<int64_t*>(base + o_edges);
  if (!edges) TSDS_CK(launch_edges(nullptr, 1, &S, x != nullptr, x_dtype, nb, st));
  // the range as a series of its own: its bins' starts are the whole series' starts b0..b1
  WorkCounters* w = reinterpret_cast<WorkCounters*>(base + o_work);
  S.nb = k;
  S.edges += b0;
  S.res = reinterpret_cast<int64_t*>(base + o_res);
  S.cnt = reinterpret_cast<uint32_t*>(base + o_cnt);
  S.out = out;
  S.out_count = out_count;
  S.status = &w->status;
  StreamConfig cfg;
  cfg.mean_bin_bytes = n / nb * elem;
  GrpShape shape = grp_shape(cfg.mean_bin_bytes, elem);
  const int64_t tile_bins = (int64_t)(32 >> shape.g_log2) * shape.tile_rounds;
  void* tok;
  timing_begin(st, &tok);
  TSDS_CK(launch_argminmax_grp(nullptr, S, nullptr, (k + tile_bins - 1) / tile_bins, w, y_dtype, nan, shape, st));
  cfg.variant = STREAM_LDG;
  cfg.mean_bin_bytes = kPrefetchOffBinBytes;
  cfg.min_bin = shape.max_bin;
  cfg.large_dev = &w->large;
  TSDS_CK(launch_argminmax(nullptr, 1, S, nullptr, windows, reinterpret_cast<Piece*>(base + o_first),
                           reinterpret_cast<Piece*>(base + o_last), w + 1, y_dtype, nan, st, cfg));
  timing_end(st, tok);
  if (k >= kEmitTiledMinBins) TSDS_CK(launch_emit_tiled(S, algo, reinterpret_cast<int64_t*>(base + o_tiles), st));
  else TSDS_CK(launch_emit(nullptr, 1, S, algo, st));
  return TSDS_OK;
}

static tsds_status binned_range_entry(Algo algo, const void* x, tsds_dtype x_dtype, const void* y,
                                      tsds_dtype y_dtype, int64_t n, int64_t n_out, int64_t bin_lo, int64_t bin_hi,
                                      tsds_nan_mode nan, int64_t* out, int64_t* out_count, void* stream) {
  g_err[0] = 0;
  const char* who = algo == ALGO_MINMAX ? "tsds_minmax_bins" : "tsds_m4_bins";
  tsds_status s = check_common(x, x_dtype, y, y_dtype, n, nan, out, out_count);
  if (s != TSDS_OK) return s;
  const int per_bin = algo == ALGO_MINMAX ? 2 : 4;
  if (n_out < per_bin || n_out % per_bin != 0)
    return fail(TSDS_EINVAL, "%s: n_out must be a positive multiple of %d (got %lld)", who, per_bin, (long long)n_out);
  if (n_out >= n)
    return fail(TSDS_EINVAL, "%s: n_out >= n selects every index and has no bins (n = %lld, n_out = %lld)", who,
                (long long)n, (long long)n_out);
  const int64_t nb = n_out / per_bin;
  if (bin_lo < 0 || bin_hi < bin_lo || bin_hi > nb)
    return fail(TSDS_EINVAL, "%s: bins [%lld, %lld) are not inside [0, %lld)", who, (long long)bin_lo,
                (long long)bin_hi, (long long)nb);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s = check_sorted_x(who, x, x_dtype, n, st);
  if (s != TSDS_OK) return s;
  if (bin_hi == bin_lo) {
    TSDS_CK(cudaMemsetAsync(out_count, 0, sizeof(int64_t), st));
    return TSDS_OK;
  }
  return run_binned_range(x, x_dtype, y, y_dtype, n, nb, bin_lo, bin_hi, nan, algo, out, out_count, st);
}

// Host-buffer form: y is copied to the device in chunks on a private stream;
// after each chunk the bins whose points have all arrived are reduced on the
// caller's stream (bin ranges over the whole series' bin starts, Section 2.2's
// independent bins), so the copy and the reduction overlap; the range outputs
// are compacted on the host in bin order.
static int64_t host_chunk_bytes(int64_t total) {
  int64_t c = total / 8;
  const int64_t lo = 16ll << 20, hi = 256ll << 20;
  c = c < lo ? lo : c > hi ? hi : c;
  return c / 64 * 64;
}

struct HostJob {
  Algo algo = ALGO_MINMAX;
  int per = 2;
  int64_t nb = 0;
  int64_t* edges_dev = nullptr;
  int64_t* out_dev = nullptr;
  int64_t* cnt_dev = nullptr;
  std::vector<int64_t> edges;
  std::vector<int64_t> range_lo;   // first bin of each range (ranges in bin order)
};

static tsds_status host_entry(int count, const int* algos, const int64_t* n_outs, const void* x, tsds_dtype x_dtype,
                              const void* y_host, tsds_dtype y_dtype, int64_t n, tsds_nan_mode nan, void* y_dev,
                              int64_t* const* outs_host, int64_t* counts_host, void* stream) {
  g_err[0] = 0;
  const char* who = "tsds_downsample_host";
  if (count < 1 || count > 16) return fail(TSDS_EINVAL, "%s: count must be in [1, 16] (got %d)", who, count);
  if (!algos || !n_outs || !outs_host || !counts_host)
    return fail(TSDS_EINVAL, "%s: algos, n_outs, outs_host and counts_host must not be NULL", who);
  tsds_status s = check_common(x, x_dtype, y_host, y_dtype, n, nan, outs_host[0], counts_host);
  if (s != TSDS_OK) return s;
  for (int i = 0; i < count; ++i) {
    if (algos[i] != TSDS_ALGO_MINMAX && algos[i] != TSDS_ALGO_M4)
      return fail(TSDS_EINVAL, "%s: algos[%d] = %d is neither TSDS_ALGO_MINMAX nor TSDS_ALGO_M4", who, i, algos[i]);
    const int per = algos[i] == TSDS_ALGO_MINMAX ? 2 : 4;
    if (n_outs[i] < per || n_outs[i] % per != 0)
      return fail(TSDS_EINVAL, "%s: n_outs[%d] must be a positive multiple of %d (got %lld)", who, i, per,
                  (long long)n_outs[i]);
    if (n > 0 && !outs_host[i]) return fail(TSDS_EINVAL, "%s: outs_host[%d] is NULL", who, i);
  }
  if (y_dev && reinterpret_cast<uintptr_t>(y_dev) % dtype_size(y_dtype) != 0)
    return fail(TSDS_EINVAL, "%s: y_dev is not aligned to its element size", who);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // x: device memory, or page-locked host memory read in place through its
  // device address
  const void* xd = x;
  if (x) {
    cudaPointerAttributes pa;
    const cudaError_t e = cudaPointerGetAttributes(&pa, x);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(TSDS_EINVAL, "%s: x is not an address CUDA knows (%s)", who, cudaGetErrorString(e));
    }
    if (pa.type == cudaMemoryTypeUnregistered || (pa.type == cudaMemoryTypeHost && !pa.devicePointer))
      return fail(TSDS_EINVAL, "%s: x must be device memory or page-locked host memory", who);
    if (pa.type == cudaMemoryTypeHost) xd = pa.devicePointer;
  }
  s = check_sorted_x(who, xd, x_dtype, n, st);
  if (s != TSDS_OK) return s;
  if (n == 0) {
    for (int i = 0; i < count; ++i) counts_host[i] = 0;
    return TSDS_OK;
  }
  const int64_t es = dtype_size(y_dtype);
  const int64_t total = n * es;
  const int64_t chunk = host_chunk_bytes(total);
  const int64_t chunks = (total + chunk - 1) / chunk;
  // scratch: y (unless the caller gives a buffer), then per binned job its
  // bin starts, its range outputs at their largest and one count per chunk
  std::vector<HostJob> jobs;
  size_t o = align_up(y_dev ? 0 : (size_t)total, 256);
  for (int i = 0; i < count; ++i) {
    HostJob j;
    j.algo = algos[i] == TSDS_ALGO_MINMAX ? ALGO_MINMAX : ALGO_M4;
    j.per = algos[i] == TSDS_ALGO_MINMAX ? 2 : 4;
    j.nb = n_outs[i] >= n ? 0 : n_outs[i] / j.per;
    jobs.push_back(std::move(j));
  }
  std::vector<size_t> off(count * 3);
  for (int i = 0; i < count; ++i) {
    const int64_t nb = jobs[i].nb;
    off[3 * i] = o;     o = align_up(o + (size_t)(nb > 0 ? nb + 1 : 0) * 8, 256);
    off[3 * i + 1] = o; o = align_up(o + (size_t)(nb * jobs[i].per) * 8, 256);
    off[3 * i + 2] = o; o = align_up(o + (size_t)chunks * 8, 256);
  }
  Scratch sc;
  TSDS_CK(scratch_alloc(sc, o, st));
  char* base = static_cast<char*>(sc.p);
  char* yd = y_dev ? static_cast<char*>(y_dev) : base;
  // bin starts of every binned job (x read in place), copied to the host to
  // cut the bins into per-chunk ranges
  for (int i = 0; i < count; ++i) {
    HostJob& j = jobs[i];
    if (j.nb == 0) continue;
    j.edges_dev = reinterpret_cast<int64_t*>(base + off[3 * i]);
    j.out_dev = reinterpret_cast<int64_t*>(base + off[3 * i + 1]);
    j.cnt_dev = reinterpret_cast<int64_t*>(base + off[3 * i + 2]);
    SeriesDev S;
    memset(&S, 0, sizeof S);
    S.x = xd;
    S.n = n;
    S.nb = j.nb;
    S.edges = j.edges_dev;
    TSDS_CK(launch_edges(nullptr, 1, &S, xd != nullptr, x_dtype, j.nb, st));
    j.edges.resize((size_t)j.nb + 1);
    TSDS_CK(cudaMemcpyAsync(j.edges.data(), j.edges_dev, (size_t)(j.nb + 1) * 8, cudaMemcpyDeviceToHost, st));
  }
  TSDS_CK(cudaStreamSynchronize(st));
  // the copy stream starts after the caller's earlier work on `stream` (y_dev
  // may still be read by it); one event per chunk.  On every way out the
  // caller's stream waits for the last copy, so that nothing later on it (the
  // scratch's release among them) overtakes a copy still in flight.
  struct Events {
    cudaStream_t cs = nullptr, st = nullptr;
    std::vector<cudaEvent_t> ev;
    int64_t last = -1;
    ~Events() {
      if (last >= 0) cudaStreamWaitEvent(st, ev[(size_t)last], 0);
      for (cudaEvent_t e : ev) cudaEventDestroy(e);
      if (cs) cudaStreamDestroy(cs);
    }
  } E;
  E.st = st;
  TSDS_CK(cudaStreamCreateWithFlags(&E.cs, cudaStreamNonBlocking));
  E.ev.assign((size_t)chunks + 1, nullptr);
  for (auto& e : E.ev) TSDS_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  TSDS_CK(cudaEventRecord(E.ev[chunks], st));
  TSDS_CK(cudaStreamWaitEvent(E.cs, E.ev[chunks], 0));
  const char* yh = static_cast<const char*>(y_host);
  for (int64_t c = 0; c < chunks; ++c) {
    const int64_t b = c * chunk, len = (c + 1 == chunks ? total : b + chunk) - b;
    TSDS_CK(cudaMemcpyAsync(yd + b, yh + b, (size_t)len, cudaMemcpyHostToDevice, E.cs));
    TSDS_CK(cudaEventRecord(E.ev[c], E.cs));
    E.last = c;
  }
  std::vector<int64_t> done((size_t)count, 0);
  for (int64_t c = 0; c < chunks; ++c) {
    TSDS_CK(cudaStreamWaitEvent(st, E.ev[c], 0));
    const int64_t have = c + 1 == chunks ? n : (c + 1) * chunk / es;   // points on the device
    for (int i = 0; i < count; ++i) {
      HostJob& j = jobs[i];
      if (j.nb == 0) continue;
      // bins whose last point has arrived: edges[b + 1] <= have
      const int64_t b1 = (int64_t)(std::upper_bound(j.edges.begin() + 1, j.edges.end(), have) - (j.edges.begin() + 1));
      if (b1 <= done[i]) continue;
      int64_t* cnt = j.cnt_dev + j.range_lo.size();
      s = run_binned_range(xd, x_dtype, yd, y_dtype, n, j.nb, done[i], b1, nan, j.algo, j.out_dev + j.per * done[i],
                           cnt, st, j.edges_dev);
      if (s != TSDS_OK) return s;
      j.range_lo.push_back(done[i]);
      done[i] = b1;
    }
  }
  // outputs: each job's ranges back to the host, compacted in bin order
  std::vector<std::vector<int64_t>> stage((size_t)count), counts((size_t)count);
  for (int i = 0; i < count; ++i) {
    HostJob& j = jobs[i];
    if (j.nb == 0) continue;
    stage[i].resize((size_t)(j.nb * j.per));
    counts[i].resize(j.range_lo.size());
    TSDS_CK(cudaMemcpyAsync(stage[i].data(), j.out_dev, stage[i].size() * 8, cudaMemcpyDeviceToHost, st));
    TSDS_CK(cudaMemcpyAsync(counts[i].data(), j.cnt_dev, counts[i].size() * 8, cudaMemcpyDeviceToHost, st));
  }
  TSDS_CK(cudaStreamSynchronize(st));
  for (int i = 0; i < count; ++i) {
    HostJob& j = jobs[i];
    if (j.nb == 0) {
      for (int64_t v = 0; v < n; ++v) outs_host[i][v] = v;   // n_out >= n: every index
      counts_host[i] = n;
      continue;
    }
    int64_t pos = 0;
    for (size_t r = 0; r < j.range_lo.size(); ++r) {
      const int64_t k = counts[i][r];
      if (k < 0) return fail((tsds_status)(-k), "%s: the streaming pass reported a device-side failure", who);
      memcpy(outs_host[i] + pos, stage[i].data() + j.per * j.range_lo[r], (size_t)k * 8);
      pos += k;
    }
    counts_host[i] = pos;
  }
  return TSDS_OK;
}

// EveryNth: the bin starts (index space or x space, as for MinMax/M4) with
// n_out bins, then the emit of the first point of every non-empty bin.
static tsds_status run_everynth(const void* x, tsds_dtype x_dtype, int64_t n, int64_t nb, int64_t* out,
                                int64_t* out_count, cudaStream_t st, const void* y, const Gather* g) {
  const bool tiled = nb >= kEmitTiledMinBins;
  const size_t o_tiles = align_up((size_t)(nb + 1) * 8, 256);
  Scratch s;
  TSDS_CK(scratch_alloc(s, o_tiles + (tiled ? align_up((size_t)emit_tiles(nb) * 8, 256) : 0), st));
  char* base = static_cast<char*>(s.p);
  SeriesDev S;
  memset(&S, 0, sizeof S);
  S.y = y;
  S.x = x;
  S.n = n;
  S.nb = nb;
  S.edges = reinterpret_cast<int64_t*>(base);
  S.out = out;
  S.out_count = out_count;
  if (g) S.g = *g;
  TSDS_CK(launch_edges(nullptr, 1, &S, x != nullptr, x_dtype, nb, st));
  if (tiled) TSDS_CK(launch_emit_tiled(S, ALGO_EVERYNTH, reinterpret_cast<int64_t*>(base + o_tiles), st));
  else TSDS_CK(launch_emit(nullptr, 1, S, ALGO_EVERYNTH, st));
  return TSDS_OK;
}

// Checks the optional value outputs and fills g (null g when there are none).
static tsds_status gather_args(const void* x, tsds_dtype x_dtype, tsds_dtype y_dtype, void* x_out, void* y_out,
                               Gather& g, const Gather*& gp) {
  gp = nullptr;
  if (!x_out && !y_out) return TSDS_OK;
  if (x_out && !x) return fail(TSDS_EINVAL, "x_out needs x (without x the index is the x value)");
  g.y_size = (int)dtype_size(y_dtype);
  g.x_size = x ? (int)dtype_size(x_dtype) : 0;
  if (y_out && reinterpret_cast<uintptr_t>(y_out) % (uintptr_t)g.y_size != 0)
    return fail(TSDS_EINVAL, "y_out is not aligned to its %d-byte elements", g.y_size);
  if (x_out && reinterpret_cast<uintptr_t>(x_out) % (uintptr_t)g.x_size != 0)
    return fail(TSDS_EINVAL, "x_out is not aligned to its %d-byte elements", g.x_size);
  g.y_out = y_out;
  g.x_out = x_out;
  gp = &g;
  return TSDS_OK;
}

static tsds_status run_binned(Algo algo, const void* x, tsds_dtype x_dtype, const void* y,
                              tsds_dtype y_dtype, int64_t n, int64_t n_out, tsds_nan_mode nan,
                              int64_t* out, int64_t* out_count, void* stream, void* x_out = nullptr,
                              void* y_out = nullptr) {
  g_err[0] = 0;
  tsds_status s = check_common(x, x_dtype, y, y_dtype, n, nan, out, out_count);
  if (s != TSDS_OK) return s;
  Gather g;
  const Gather* gp;
  s = gather_args(x, x_dtype, y_dtype, x_out, y_out, g, gp);
  if (s != TSDS_OK) return s;
  const int per_bin = algo == ALGO_MINMAX ? 2 : algo == ALGO_M4 ? 4 : 1;
  if (n_out < per_bin || n_out % per_bin != 0)
    return fail(TSDS_EINVAL, "%s needs n_out to be a positive multiple of %d (got %lld)",
                algo == ALGO_MINMAX ? "MinMax" : algo == ALGO_M4 ? "M4" : "EveryNth", per_bin, (long long)n_out);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s = check_sorted_x(algo == ALGO_MINMAX ? "MinMax" : algo == ALGO_M4 ? "M4" : "EveryNth", x, x_dtype, n, st);
  if (s != TSDS_OK) return s;
  if (n == 0) {
    TSDS_CK(cudaMemsetAsync(out_count, 0, sizeof(int64_t), st));
    return TSDS_OK;
  }
  if (n_out >= n) {
    TSDS_CK(launch_iota(out, n, out_count, st, y, x, gp));
    return TSDS_OK;
  }
  if (algo == ALGO_EVERYNTH) return run_everynth(x, x_dtype, n, n_out, out, out_count, st, y, gp);
  return run_binned_series(x, x_dtype, y, y_dtype, n, n_out / per_bin, nan, algo, out, out_count, 0, st, gp);
}

}  // namespace tsds

using namespace tsds;

extern "C" {

tsds_status tsds_minmax(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                        int64_t n, int64_t n_out, tsds_nan_mode nan, int64_t* out,
                        int64_t* out_count, void* stream) {
  NvtxRange nvtx_("tsds_minmax");
  return run_binned(ALGO_MINMAX, x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, stream);
}

tsds_status tsds_m4(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                    int64_t n, int64_t n_out, tsds_nan_mode nan, int64_t* out,
                    int64_t* out_count, void* stream) {
  NvtxRange nvtx_("tsds_m4");
  return run_binned(ALGO_M4, x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, stream);
}

static tsds_status lttb_entry(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype, int64_t n,
                              int64_t n_out, tsds_nan_mode nan, int64_t* out, int64_t* out_count, void* stream,
                              void* x_out, void* y_out) {
  g_err[0] = 0;
  tsds_status s = check_common(x, x_dtype, y, y_dtype, n, nan, out, out_count);
  if (s != TSDS_OK) return s;
  if (n_out < 3) return fail(TSDS_EINVAL, "LTTB needs n_out >= 3 (got %lld)", (long long)n_out);
  Gather g;
  const Gather* gp;
  s = gather_args(x, x_dtype, y_dtype, x_out, y_out, g, gp);
  if (s != TSDS_OK) return s;
  s = check_sorted_x("LTTB", x, x_dtype, n, static_cast<cudaStream_t>(stream));
  if (s != TSDS_OK) return s;
  return run_lttb(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, static_cast<cudaStream_t>(stream),
                  nullptr, gp);
}

static tsds_status minmaxlttb_entry(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                                    int64_t n, int64_t n_out, int64_t minmax_ratio, tsds_nan_mode nan, int64_t* out,
                                    int64_t* out_count, void* stream, void* x_out, void* y_out) {
  g_err[0] = 0;
  tsds_status s = check_common(x, x_dtype, y, y_dtype, n, nan, out, out_count);
  if (s != TSDS_OK) return s;
  if (n_out < 3) return fail(TSDS_EINVAL, "MinMaxLTTB needs n_out >= 3 (got %lld)", (long long)n_out);
  if (minmax_ratio < 1) return fail(TSDS_EINVAL, "minmax_ratio must be >= 1 (got %lld)", (long long)minmax_ratio);
  if (minmax_ratio > (INT64_MAX / 4) / n_out) return fail(TSDS_EINVAL, "n_out * minmax_ratio overflows");
  Gather g;
  const Gather* gp;
  s = gather_args(x, x_dtype, y_dtype, x_out, y_out, g, gp);
  if (s != TSDS_OK) return s;
  s = check_sorted_x("MinMaxLTTB", x, x_dtype, n, static_cast<cudaStream_t>(stream));
  if (s != TSDS_OK) return s;
  return run_minmaxlttb(x, x_dtype, y, y_dtype, n, n_out, minmax_ratio, nan, out, out_count,
                        static_cast<cudaStream_t>(stream), gp);
}

tsds_status tsds_lttb(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                      int64_t n, int64_t n_out, tsds_nan_mode nan, int64_t* out,
                      int64_t* out_count, void* stream) {
  NvtxRange nvtx_("tsds_lttb");
  return lttb_entry(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, stream, nullptr, nullptr);
}

tsds_status tsds_minmaxlttb(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                            int64_t n, int64_t n_out, int64_t minmax_ratio, tsds_nan_mode nan,
                            int64_t* out, int64_t* out_count, void* stream) {
  NvtxRange nvtx_("tsds_minmaxlttb");
  return minmaxlttb_entry(x, x_dtype, y, y_dtype, n, n_out, minmax_ratio, nan, out, out_count, stream, nullptr,
                          nullptr);
}

tsds_status tsds_minmax_bins(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype, int64_t n,
                             int64_t n_out, int64_t bin_lo, int64_t bin_hi, tsds_nan_mode nan, int64_t* out,
                             int64_t* out_count, void* stream) {
  NvtxRange nvtx_("tsds_minmax_bins");
  return binned_range_entry(ALGO_MINMAX, x, x_dtype, y, y_dtype, n, n_out, bin_lo, bin_hi, nan, out, out_count,
                            stream);
}

tsds_status tsds_m4_bins(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype, int64_t n,
                         int64_t n_out, int64_t bin_lo, int64_t bin_hi, tsds_nan_mode nan, int64_t* out,
                         int64_t* out_count, void* stream) {
  NvtxRange nvtx_("tsds_m4_bins");
  return binned_range_entry(ALGO_M4, x, x_dtype, y, y_dtype, n, n_out, bin_lo, bin_hi, nan, out, out_count, stream);
}

tsds_status tsds_downsample_host(int count, const int* algos, const int64_t* n_outs, const void* x,
                                 tsds_dtype x_dtype, const void* y_host, tsds_dtype y_dtype, int64_t n,
                                 tsds_nan_mode nan, void* y_dev, int64_t* const* outs_host, int64_t* counts_host,
                                 void* stream) {
  NvtxRange nvtx_("tsds_downsample_host");
  return host_entry(count, algos, n_outs, x, x_dtype, y_host, y_dtype, n, nan, y_dev, outs_host, counts_host,
                    stream);
}

tsds_status tsds_everynth(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype, int64_t n,
                          int64_t n_out, tsds_nan_mode nan, int64_t* out, int64_t* out_count, void* stream) {
  NvtxRange nvtx_("tsds_everynth");
  return run_binned(ALGO_EVERYNTH, x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, stream);
}

tsds_status tsds_everynth_values(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype, int64_t n,
                                 int64_t n_out, tsds_nan_mode nan, int64_t* out, int64_t* out_count, void* x_out,
                                 void* y_out, void* stream) {
  NvtxRange nvtx_("tsds_everynth_values");
  return run_binned(ALGO_EVERYNTH, x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, stream, x_out, y_out);
}

tsds_status tsds_minmax_values(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype, int64_t n,
                               int64_t n_out, tsds_nan_mode nan, int64_t* out, int64_t* out_count, void* x_out,
                               void* y_out, void* stream) {
  NvtxRange nvtx_("tsds_minmax_values");
  return run_binned(ALGO_MINMAX, x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, stream, x_out, y_out);
}

tsds_status tsds_m4_values(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype, int64_t n,
                           int64_t n_out, tsds_nan_mode nan, int64_t* out, int64_t* out_count, void* x_out,
                           void* y_out, void* stream) {
  NvtxRange nvtx_("tsds_m4_values");
  return run_binned(ALGO_M4, x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, stream, x_out, y_out);
}

tsds_status tsds_lttb_values(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype, int64_t n,
                             int64_t n_out, tsds_nan_mode nan, int64_t* out, int64_t* out_count, void* x_out,
                             void* y_out, void* stream) {
  NvtxRange nvtx_("tsds_lttb_values");
  return lttb_entry(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, stream, x_out, y_out);
}

tsds_status tsds_minmaxlttb_values(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype, int64_t n,
                                   int64_t n_out, int64_t minmax_ratio, tsds_nan_mode nan, int64_t* out,
                                   int64_t* out_count, void* x_out, void* y_out, void* stream) {
  NvtxRange nvtx_("tsds_minmaxlttb_values");
  return minmaxlttb_entry(x, x_dtype, y, y_dtype, n, n_out, minmax_ratio, nan, out, out_count, stream, x_out,
                          y_out);
}

tsds_status tsds_lttb_means(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                            int64_t n, int64_t n_out, tsds_nan_mode nan, double* means, void* stream) {
  NvtxRange nvtx_("tsds_lttb_means");
  g_err[0] = 0;
  if (!means) return fail(TSDS_EINVAL, "tsds_lttb_means: means is NULL");
  if (n_out < 3 || n_out >= n)
    return fail(TSDS_EINVAL, "tsds_lttb_means needs 3 <= n_out < n (got n_out %lld, n %lld)", (long long)n_out,
                (long long)n);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch sc;
  TSDS_CK(scratch_alloc(sc, align_up((size_t)(n_out + 1) * sizeof(int64_t), 256), st));
  int64_t* out = static_cast<int64_t*>(sc.p);
  tsds_status s = check_common(x, x_dtype, y, y_dtype, n, nan, out, out + n_out);
  if (s != TSDS_OK) return s;
  s = check_sorted_x("tsds_lttb_means", x, x_dtype, n, st);
  if (s != TSDS_OK) return s;
  return run_lttb(x, x_dtype, y, y_dtype, n, n_out, nan, out, out + n_out, st, means);
}

const char* tsds_last_error(void) { return g_err; }

void tsds_shutdown(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  int cur = 0;
  cudaGetDevice(&cur);
  for (auto& kv : g_dev) {
    if (kv.second.pool) {
      cudaSetDevice(kv.first);
      cudaMemPoolDestroy(kv.second.pool);
    }
  }
  g_dev.clear();
  cudaSetDevice(cur);
  noalloc_forget_devices();
  forget_stream_occupancy();
}

const char* tsds_version(void) { return "0.1.0"; }

int64_t tsds_kernel_launches(void) { return g_launches.load(); }

tsds_status tsds_check_wait_timeout(unsigned rounds, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch s;
  TSDS_CK(scratch_alloc(s, 256, st));
  unsigned long long* word = static_cast<unsigned long long*>(s.p);
  TSDS_CK(launch_wait_probe(word, rounds, st));
  unsigned long long v = 0;
  TSDS_CK(cudaMemcpyAsync(&v, word, sizeof v, cudaMemcpyDeviceToHost, st));
  TSDS_CK(cudaStreamSynchronize(st));
  return (tsds_status)v;
}

void tsds_timing_enable(int on) { g_timing.store(on ? 1 : 0); }

void tsds_inject_alloc_failures(int count) { g_fail_allocs.store(count > 0 ? count : 0); }

int tsds_checked(int on) {
  if (on < 0) return g_checked.load();
  return g_checked.exchange(on ? 1 : 0);
}

tsds_status tsds_read_stream(const void* buf, int64_t bytes, uint64_t* sink, void* stream) {
  NvtxRange nvtx_("tsds_read_stream");
  if (bytes < 0 || bytes % 16 != 0)
    return fail(TSDS_EINVAL, "tsds_read_stream: bytes must be a non-negative multiple of 16 (got %lld)",
                (long long)bytes);
  if (!sink) return fail(TSDS_EINVAL, "tsds_read_stream: sink is null");
  if (bytes > 0 && (!buf || (reinterpret_cast<uintptr_t>(buf) & 15) != 0))
    return fail(TSDS_EINVAL, "tsds_read_stream: buf must be a non-null 16-byte aligned pointer");
  TSDS_CK(launch_read_stream(buf, bytes, sink, static_cast<cudaStream_t>(stream)));
  return TSDS_OK;
}

tsds_status tsds_timing_read(double* total_ms, int64_t* launches) {
  std::vector<TimedLaunch> done;
  {
    std::lock_guard<std::mutex> lk(g_tmu);
    done.swap(g_timed);
  }
  double ms = 0.0;
  tsds_status st = TSDS_OK;
  for (auto& t : done) {
    float f = 0.f;
    if (cudaEventSynchronize(t.b) != cudaSuccess || cudaEventElapsedTime(&f, t.a, t.b) != cudaSuccess)
      st = fail(TSDS_ECUDA, "tsds_timing_read: event query failed");
    ms += f;
  }
  {
    std::lock_guard<std::mutex> lk(g_tmu);
    for (auto& t : done) { g_free_events.push_back(t.a); g_free_events.push_back(t.b); }
  }
  if (total_ms) *total_ms = ms;
  if (launches) *launches = (int64_t)done.size();
  return st;
}

}  // extern "C"
