// batched.cu -- MinMax / M4 over many series in one persistent launch.
//
// The paper's parallel mode splits one series' bins over CPU threads
// (Section 2.2, the `parallel` option of Section 2.3).  On the GPU the cost of
// a small series is the launch itself, so the batched form puts every series
// of a batch into one window numbering: one edge kernel (a grid row per
// series), one streaming argmin/argmax launch whose warps claim windows of
// any series from one counter (the window -> series map tells them which),
// one emit kernel (a CTA per series) and one kernel for series whose n_out
// covers them.  A plan keeps the descriptors and scratch resident, can pick
// its launch shape by timing candidates (autotune), and can replay its whole
// kernel sequence as one CUDA graph.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace tsds {

tsds_status fail(tsds_status s, const char* fmt, ...);
bool take_injected_alloc_failure();   // failure injection of the library's allocations (api.cu)

#define BT_CK(call)                                                                      \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(e_ == cudaErrorMemoryAllocation ? TSDS_ENOMEM : TSDS_ECUDA, "%s: %s",  \
                  #call, cudaGetErrorString(e_));                                        \
  } while (0)

static size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// Everything one batch needs, laid out in one scratch block.
struct BatchLayout {
  int64_t count = 0;
  int64_t total_nb = 0, max_nb = 0, total_windows = 0, y_bytes = 0;
  int64_t mean_bin_bytes = 0;  // bytes-weighted mean bin size of the binned series
  int64_t mean_bin_bytes0 = 0, mean_bin_bytes1 = 0;   // the same over groups 0 and 1
  // Series groups of the automatic variant: 0 large bins (register streaming
  // over windows), 1 small bins below seg_max_bin_bytes (segmented, windows
  // numbered after group 0's, from split_windows on), 2 bins from there up to
  // kSmallMaxBinBytes (a warp per bin, mid_ctas CTAs, no windows).  With an
  // explicit variant every series is cut into windows.
  // Group 3 (automatic variant, batches without x): bins below
  // kGrpBatchedMaxBinBytes run in the lane-group pass, grp_tiles tiles.
  std::vector<uint8_t> group;
  int64_t split_windows = 0, mid_ctas = 0, grp_tiles = 0;
  int64_t elem = 1;
  bool auto_groups = true;     // how the current numbering was made
  bool any_full = false;       // some series returns every index
  size_t off_desc = 0, off_edges = 0, off_res = 0, off_cnt = 0, off_work = 0, off_map = 0, off_first = 0,
         off_last = 0, off_ctas = 0, off_tiles = 0, total = 0;
  std::vector<SeriesDev> host; // descriptors (scratch pointers set by bind_layout)
  std::vector<int64_t> nb_before;  // bins of the series before each one
};

static bool batch_has_x(const tsds_series* s, int64_t count) {
  for (int64_t i = 0; i < count; ++i)
    if (s[i].n > 0) return s[i].x != nullptr;
  return false;
}

static tsds_status check_series(tsds_algo algo, const tsds_series* s, int64_t count, tsds_dtype x_dtype,
                                tsds_dtype y_dtype, tsds_nan_mode nan) {
  if (count < 1 || count > 65535) return fail(TSDS_EINVAL, "batched: count must be in [1, 65535] (got %lld)", (long long)count);
  if (!s) return fail(TSDS_EINVAL, "batched: series is NULL");
  if (algo != TSDS_ALGO_MINMAX && algo != TSDS_ALGO_M4) return fail(TSDS_EINVAL, "batched: unknown algorithm %d", (int)algo);
  if (!dtype_valid(y_dtype)) return fail(TSDS_EINVAL, "batched: unknown y dtype %d", (int)y_dtype);
  if (nan != TSDS_NAN_PROPAGATE && nan != TSDS_NAN_IGNORE) return fail(TSDS_EINVAL, "batched: unknown NaN mode");
  // x presence is decided by the non-empty series (an empty series' x may be NULL)
  bool has_x = false;
  for (int64_t i = 0; i < count; ++i)
    if (s[i].n > 0) { has_x = s[i].x != nullptr; break; }
  if (has_x && !dtype_valid(x_dtype)) return fail(TSDS_EINVAL, "batched: unknown x dtype %d", (int)x_dtype);
  const int per = algo == TSDS_ALGO_MINMAX ? 2 : 4;
  for (int64_t i = 0; i < count; ++i) {
    const tsds_series& q = s[i];
    if (q.n > 0 && (q.x != nullptr) != has_x)
      return fail(TSDS_EINVAL, "batched: series %lld: either every non-empty series has x or none", (long long)i);
    if (q.n < 0) return fail(TSDS_EINVAL, "batched: series %lld: n < 0", (long long)i);
    if (q.n_out < per || q.n_out % per) return fail(TSDS_EINVAL, "batched: series %lld: n_out must be a positive multiple of %d", (long long)i, per);
    if ((q.n > 0 && (!q.y || !q.out)) || !q.out_count) return fail(TSDS_EINVAL, "batched: series %lld: NULL buffer", (long long)i);
    if (reinterpret_cast<uintptr_t>(q.y) % dtype_size(y_dtype) ||
        (has_x && reinterpret_cast<uintptr_t>(q.x) % dtype_size(x_dtype)))
      return fail(TSDS_EINVAL, "batched: series %lld: x or y not aligned to its element size", (long long)i);
  }
  return TSDS_OK;
}

// Checked mode: every series' x in order, one check launch per series and a
// single wait for all of them.
tsds_status check_batch_sorted(const tsds_series* s, int64_t count, tsds_dtype x_dtype, cudaStream_t st) {
  if (!checked_mode() || !batch_has_x(s, count)) return TSDS_OK;
  Scratch sc;
  BT_CK(scratch_alloc(sc, (size_t)count * sizeof(unsigned long long), st));
  unsigned long long* words = static_cast<unsigned long long*>(sc.p);
  BT_CK(cudaMemsetAsync(words, 0xff, (size_t)count * sizeof(unsigned long long), st));
  for (int64_t i = 0; i < count; ++i)
    if (s[i].n > 0) BT_CK(launch_check_sorted(s[i].x, x_dtype, s[i].n, words + i, st));
  std::vector<unsigned long long> bad((size_t)count);
  BT_CK(cudaMemcpyAsync(bad.data(), words, (size_t)count * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  BT_CK(cudaStreamSynchronize(st));
  for (int64_t i = 0; i < count; ++i)
    if (bad[(size_t)i] != ~0ull)
      return fail(TSDS_EINVAL, "batched: series %lld: x is not sorted non-decreasing (NaN or x[i] > x[i+1] at i = %llu; "
                  "checked mode)", (long long)i, bad[(size_t)i]);
  return TSDS_OK;
}

// Window bases for windows of welems elements: group 0 first, then group 1
// (from split_windows on); with auto_groups, group 2 gets CTA bases and group
// 3 tile bases (its lane-group shape from the series' bin size, with G scaled
// by 2^grp_scale and the bins per tile by 2^tile_scale) instead.
static void number_windows(BatchLayout& L, int64_t welems, bool auto_groups, int grp_scale = 0,
                           int tile_scale = 0) {
  int64_t win = 0, cta = 0, tile = 0;
  L.auto_groups = auto_groups;
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) L.split_windows = win;
    for (size_t i = 0; i < L.host.size(); ++i) {
      SeriesDev& d = L.host[i];
      const int g = auto_groups ? L.group[i] : 0;
      if (g == 3) {
        if (pass == 0) {
          GrpShape sh = grp_shape(d.n * L.elem / d.nb, L.elem);
          int lg = sh.g_log2 + grp_scale;
          lg = lg < 0 ? 0 : lg > 5 ? 5 : lg;
          const int groups = 32 >> lg;
          int rounds = (int)(sh.tile_rounds * (int64_t)(32 >> sh.g_log2) / groups);
          rounds = tile_scale >= 0 ? rounds << tile_scale : rounds >> -tile_scale;
          if (rounds < 1) rounds = 1;
          if (rounds * groups > kGrpTileMaxBins) rounds = kGrpTileMaxBins / groups;
          d.mode = 2;
          d.grp = grp_pack(lg, rounds);
          d.tile_base = tile;
          tile += (d.nb + (int64_t)groups * rounds - 1) / ((int64_t)groups * rounds);
        }
        continue;
      }
      if (g == 2) {
        if (pass == 0) {
          d.mode = 1;
          d.win_base = cta;
          cta += (d.nb + kBinsPerCta - 1) / kBinsPerCta;
        }
        continue;
      }
      if (g != pass) continue;
      d.mode = 0;
      d.win_base = win;
      if (d.nb > 0) win += (d.n + welems - 1) / welems;
    }
  }
  L.total_windows = win;
  L.mid_ctas = cta;
  L.grp_tiles = tile;
}

// Layout for the smallest window size a plan may try (most windows).
static BatchLayout make_layout(tsds_algo algo, const tsds_series* s, int64_t count, tsds_dtype y_dtype,
                               int64_t window_bytes) {
  BatchLayout L;
  L.count = count;
  L.elem = dtype_size(y_dtype);
  // lane groups only without x: index bins never exceed the mean by more than a point
  const bool grp_ok = !batch_has_x(s, count);
  const int per = algo == TSDS_ALGO_MINMAX ? 2 : 4;
  const int64_t welems = window_bytes / dtype_size(y_dtype);
  L.host.resize((size_t)count);
  L.nb_before.resize((size_t)count);
  int64_t nb_sum = 0;
  double wsum = 0.0, wbin = 0.0, gsum[3] = {0.0, 0.0, 0.0}, gbin[3] = {0.0, 0.0, 0.0};
  L.group.assign((size_t)count, 0);
  for (int64_t i = 0; i < count; ++i) {
    const tsds_series& q = s[i];
    SeriesDev& d = L.host[(size_t)i];
    memset(&d, 0, sizeof d);
    d.y = q.y;
    d.x = q.x;
    d.n = q.n;
    d.nb = (q.n > 0 && q.n_out < q.n) ? q.n_out / per : 0;
    if (d.nb == 0) L.any_full = true;
    L.nb_before[(size_t)i] = nb_sum;
    d.out = q.out;
    d.out_count = q.out_count;
    d.idx_bias = 0;
    nb_sum += d.nb;
    L.max_nb = std::max(L.max_nb, d.nb);
    if (d.nb > 0) {
      const double bytes = (double)q.n * (double)dtype_size(y_dtype);
      wsum += bytes;
      wbin += bytes * (bytes / (double)d.nb);
      const double bin = bytes / (double)d.nb;
      int g = bin < (double)seg_max_bin_bytes(dtype_size(y_dtype)) ? 1 : bin <= (double)kSmallMaxBinBytes ? 2 : 0;
      if (grp_ok && bin < (double)kGrpBatchedMaxBinBytes) g = 3;
      L.group[(size_t)i] = (uint8_t)g;
      if (g < 3) {
        gsum[g] += bytes;
        gbin[g] += bytes * bin;
      }
    }
    L.y_bytes += q.n * dtype_size(y_dtype);
  }
  L.mean_bin_bytes = wsum > 0.0 ? (int64_t)(wbin / wsum) : 0;
  L.mean_bin_bytes0 = gsum[0] > 0.0 ? (int64_t)(gbin[0] / gsum[0]) : 0;
  L.mean_bin_bytes1 = gsum[1] > 0.0 ? (int64_t)(gbin[1] / gsum[1]) : 0;
  number_windows(L, welems, false);                 // every series windowed: the most windows
  const int64_t win_sum = L.total_windows;
  number_windows(L, welems, true);
  const int64_t ctas = L.mid_ctas;
  L.total_nb = nb_sum;
  size_t o = 0;
  L.off_desc = o;  o = up256(o + (size_t)count * sizeof(SeriesDev));
  L.off_edges = o; o = up256(o + (size_t)(nb_sum + count) * 8);
  L.off_res = o;   o = up256(o + (size_t)nb_sum * 16);
  L.off_cnt = o;   o = up256(o + (size_t)nb_sum * 4);
  L.off_work = o;  o = up256(o + 3 * sizeof(WorkCounters));   // one counter per launch of a split pass
  L.off_map = o;   o = up256(o + (size_t)win_sum * 4);
  L.off_first = o; o = up256(o + (size_t)win_sum * sizeof(Piece));
  L.off_last = o;  o = up256(o + (size_t)win_sum * sizeof(Piece));
  L.off_ctas = o;  o = up256(o + (size_t)ctas * 4);
  L.off_tiles = o; o = up256(o + (size_t)(L.grp_tiles > 0 ? nb_sum : 0) * 4);   // at least one bin per tile
  L.total = o;
  return L;
}

// Points the descriptors' scratch pointers into `base` and recomputes the
// window bases for `window_bytes` (which must be >= the layout's) and the
// launch shape's variant.
static void bind_layout(BatchLayout& L, char* base, tsds_dtype y_dtype, int64_t window_bytes, int variant,
                        int grp_scale = 0) {
  for (size_t i = 0; i < L.host.size(); ++i) {
    SeriesDev& d = L.host[i];
    const int64_t before = L.nb_before[i];
    // series i owns edges [before + i, before + i + nb + 1), res [2*before, +2nb), cnt [before, +nb)
    d.edges = reinterpret_cast<int64_t*>(base + L.off_edges) + before + (int64_t)i;
    d.res = reinterpret_cast<int64_t*>(base + L.off_res) + 2 * before;
    d.cnt = reinterpret_cast<uint32_t*>(base + L.off_cnt) + before;
    d.status = &reinterpret_cast<WorkCounters*>(base + L.off_work)->status;
  }
  number_windows(L, window_bytes / dtype_size(y_dtype), variant == STREAM_AUTO, grp_scale);
}

static void rebase_windows(BatchLayout& L, tsds_dtype y_dtype, int64_t window_bytes, int variant, int grp_scale,
                           int tile_scale) {
  number_windows(L, window_bytes / dtype_size(y_dtype), variant == STREAM_AUTO, grp_scale, tile_scale);
}

// The window map and (automatic variant) the CTA map of the current numbering.
static tsds_status launch_maps(const BatchLayout& L, char* base, tsds_dtype y_dtype, int64_t window_bytes,
                               cudaStream_t st) {
  const SeriesDev* sd = reinterpret_cast<const SeriesDev*>(base + L.off_desc);
  if (L.total_windows > 0)
    BT_CK(launch_window_map(sd, (int)L.count, reinterpret_cast<int32_t*>(base + L.off_map), y_dtype, st,
                            window_bytes));
  if (L.auto_groups && L.mid_ctas > 0)
    BT_CK(launch_cta_map(sd, (int)L.count, reinterpret_cast<int32_t*>(base + L.off_ctas), st));
  if (L.auto_groups && L.grp_tiles > 0)
    BT_CK(launch_tile_map(sd, (int)L.count, reinterpret_cast<int32_t*>(base + L.off_tiles), st));
  return TSDS_OK;
}

// Side stream and events a plan uses to run the two launches of a split pass
// side by side (null: one after the other on the caller's stream).
struct Fork {
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};

// The kernel sequence of one execution (descriptors, window and CTA maps in
// place).  With the automatic variant the pass is a launch per series group:
// a warp per bin for mid-size bins, register streaming over the large-bin
// series' windows and the segmented kernel over the small-bin ones (each
// windowed launch with its own work counter).
static tsds_status enqueue(const BatchLayout& L, char* base, tsds_algo algo, bool has_x, tsds_dtype x_dtype,
                           tsds_dtype y_dtype, tsds_nan_mode nan, const StreamConfig& shape, cudaStream_t st,
                           const Fork& fk = Fork()) {
  StreamConfig cfg = shape;
  cfg.mean_bin_bytes = L.mean_bin_bytes;
  const SeriesDev* sd = reinterpret_cast<const SeriesDev*>(base + L.off_desc);
  SeriesDev none;
  memset(&none, 0, sizeof none);
  BT_CK(cudaMemsetAsync(base + L.off_cnt, 0, L.off_map - L.off_cnt, st));
  if (L.max_nb > 0) {
    BT_CK(launch_edges(sd, (int)L.count, nullptr, has_x, x_dtype, L.max_nb, st));
    const int32_t* map = reinterpret_cast<const int32_t*>(base + L.off_map);
    Piece* fp = reinterpret_cast<Piece*>(base + L.off_first);
    Piece* lp = reinterpret_cast<Piece*>(base + L.off_last);
    WorkCounters* work = reinterpret_cast<WorkCounters*>(base + L.off_work);
    void* tok;
    timing_begin(st, &tok);
    if (cfg.variant == STREAM_AUTO && L.auto_groups) {
      // group 1 (segmented windows [split_windows, total)) on the plan's side
      // stream, beside group 2 (a warp per bin) and then group 0 (register
      // streaming over [0, split_windows)) on the caller's stream
      StreamConfig big = cfg, small = cfg;
      big.variant = STREAM_LDG;
      big.mean_bin_bytes = L.mean_bin_bytes0;
      small.variant = STREAM_SEG;
      small.mean_bin_bytes = L.mean_bin_bytes1;
      small.window_first = L.split_windows;
      const bool g0 = L.split_windows > 0, g1 = L.total_windows > L.split_windows, g2 = L.mid_ctas > 0,
                 g3 = L.grp_tiles > 0;
      cudaStream_t st2 = st;
      if ((g1 || g3) && (g0 || g2) && fk.side) {
        BT_CK(cudaEventRecord(fk.fork, st));
        BT_CK(cudaStreamWaitEvent(fk.side, fk.fork, 0));
        st2 = fk.side;
      }
      if (g3)   // lane groups (small bins, no x): shape per series, no bin above the size limit
        BT_CK(launch_argminmax_grp(sd, none, reinterpret_cast<const int32_t*>(base + L.off_tiles), L.grp_tiles,
                                   work + 2, y_dtype, nan, GrpShape(), st2));
      if (g1)
        BT_CK(launch_argminmax(sd, (int)L.count, none, map, L.total_windows, fp, lp, work + 1, y_dtype, nan, st2,
                               small));
      if (g2)
        BT_CK(launch_bins_multi(sd, reinterpret_cast<const int32_t*>(base + L.off_ctas), L.mid_ctas, y_dtype, nan,
                                st));
      if (g0)
        BT_CK(launch_argminmax(sd, (int)L.count, none, map, L.split_windows, fp, lp, work, y_dtype, nan, st, big));
      if (st2 != st) {
        BT_CK(cudaEventRecord(fk.join, fk.side));
        BT_CK(cudaStreamWaitEvent(st, fk.join, 0));
      }
    } else if (L.total_windows > 0) {
      BT_CK(launch_argminmax(sd, (int)L.count, none, map, L.total_windows, fp, lp, work, y_dtype, nan, st, cfg));
    }
    timing_end(st, tok);
    BT_CK(launch_emit(sd, (int)L.count, none, algo == TSDS_ALGO_MINMAX ? ALGO_MINMAX : ALGO_M4, st));
  }
  if (L.any_full) BT_CK(launch_iota_batched(sd, (int)L.count, st));
  return TSDS_OK;
}

static tsds_status upload(BatchLayout& L, char* base, tsds_dtype y_dtype, const StreamConfig& cfg, cudaStream_t st) {
  rebase_windows(L, y_dtype, cfg.window_bytes, cfg.variant, cfg.grp_scale, cfg.grp_tile_scale);
  BT_CK(cudaMemcpyAsync(base + L.off_desc, L.host.data(), L.host.size() * sizeof(SeriesDev),
                        cudaMemcpyHostToDevice, st));
  const tsds_status s = launch_maps(L, base, y_dtype, cfg.window_bytes, st);
  if (s != TSDS_OK) return s;
  // the host copy may be freed or reused once the upload has been consumed
  BT_CK(cudaStreamSynchronize(st));
  return TSDS_OK;
}

// ---------------------------------------------------------------- autotuner

static StreamConfig grp_candidate(int scale, int tile_scale = 0) {
  StreamConfig c;
  c.grp_scale = scale;
  c.grp_tile_scale = tile_scale;
  return c;
}

// Candidate launch shapes: window bytes, CTAs per SM, -, kernel variant
// (automatic: split by series bin size), lanes per bin and bins per tile of
// the lane-group series (power-of-two scales of the default).  The smallest
// window must come first: the scratch is laid out for it (the most windows).
// Without a tuned choice a plan runs the default shape (64 KB windows,
// automatic variant).  The vector width is not a dimension: every streaming
// kernel loads 16 bytes per lane, which reaches the copy bandwidth on large
// bins; below that the per-bin work, not the load width, sets the rate.
static const StreamConfig kCandidates[] = {
    {16 * 1024, 0, nullptr, STREAM_RING},  {32 * 1024, 0, nullptr, STREAM_RING}, {64 * 1024, 0, nullptr, STREAM_RING},
    {128 * 1024, 0, nullptr, STREAM_RING}, {64 * 1024, 2, nullptr, STREAM_RING}, {256 * 1024, 0, nullptr, STREAM_RING},
    {32 * 1024, 0, nullptr, STREAM_LDG},   {64 * 1024, 0, nullptr, STREAM_LDG},  {256 * 1024, 0, nullptr, STREAM_LDG},
    {32 * 1024, 0, nullptr, STREAM_SEG},   {64 * 1024, 0, nullptr, STREAM_SEG},  {256 * 1024, 0, nullptr, STREAM_SEG},
    {64 * 1024, 0, nullptr, STREAM_AUTO},  {256 * 1024, 0, nullptr, STREAM_AUTO},
    // automatic split with half and twice the lanes per bin in the lane-group series,
    // then with half and twice the bins per lane-group tile
    grp_candidate(-1), grp_candidate(1), grp_candidate(0, -1), grp_candidate(0, 1)};
constexpr int kNumCandidates = sizeof(kCandidates) / sizeof(kCandidates[0]);

static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune;   // workload class -> candidate index
static bool g_tune_loaded = false;

static std::string tune_key(tsds_algo algo, tsds_dtype y_dtype, bool has_x, const BatchLayout& L) {
  int bytes_class = 0, count_class = 0;
  for (int64_t b = std::max<int64_t>(L.y_bytes, 1); b > 1; b >>= 1) ++bytes_class;
  for (int64_t c = L.count; c > 1; c >>= 1) ++count_class;
  char k[128];
  int bin_class = 0;
  for (int64_t b = std::max<int64_t>(L.mean_bin_bytes, 1); b > 1; b >>= 1) ++bin_class;
  snprintf(k, sizeof k, "s4_a%d_y%d_x%d_b%d_c%d_m%d", (int)algo, (int)y_dtype, has_x ? 1 : 0, bytes_class,
           count_class, bin_class);
  return k;
}

static const char* tune_file() { return getenv("TSDS_TUNE_CACHE"); }

static void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* f = tune_file();
  if (!f) return;
  FILE* fp = fopen(f, "r");
  if (!fp) return;
  char key[128];
  int idx;
  while (fscanf(fp, "%127s %d", key, &idx) == 2)
    if (idx >= 0 && idx < kNumCandidates) g_tune[key] = idx;
  fclose(fp);
}

static void tune_store_locked() {
  const char* f = tune_file();
  if (!f) return;
  FILE* fp = fopen(f, "w");
  if (!fp) return;
  for (auto& kv : g_tune) fprintf(fp, "%s %d\n", kv.first.c_str(), kv.second);
  fclose(fp);
}

// ---------------------------------------------------------------- plans

struct PlanImpl {
  tsds_algo algo;
  tsds_dtype x_dtype, y_dtype;
  tsds_nan_mode nan;
  bool has_x = false;
  BatchLayout L;
  char* base = nullptr;
  StreamConfig cfg;
  int tuned_index = -1;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  Fork fork;
  int graph_kernels = 0;   // kernels one graph launch runs
  float tune_ms[kNumCandidates] = {0};
};

static tsds_status time_candidate(PlanImpl* P, const StreamConfig& c, cudaStream_t st, float* ms) {
  tsds_status s = upload(P->L, P->base, P->y_dtype, c, st);
  if (s != TSDS_OK) return s;
  cudaEvent_t a, b;
  BT_CK(cudaEventCreate(&a));
  BT_CK(cudaEventCreate(&b));
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(a, st);
    s = enqueue(P->L, P->base, P->algo, P->has_x, P->x_dtype, P->y_dtype, P->nan, c, st, P->fork);
    cudaEventRecord(b, st);
    if (s != TSDS_OK) break;
    cudaEventSynchronize(b);
    float t = 0.f;
    cudaEventElapsedTime(&t, a, b);
    if (rep > 0 && t < best) best = t;   // first run warms up
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = best;
  return s;
}

}  // namespace tsds

using namespace tsds;

struct tsds_plan_s {
  PlanImpl impl;
};

extern "C" {

tsds_status tsds_batched(tsds_algo algo, const tsds_series* series, int64_t count, tsds_dtype x_dtype,
                         tsds_dtype y_dtype, tsds_nan_mode nan, void* stream) {
  tsds_status s = check_series(algo, series, count, x_dtype, y_dtype, nan);
  if (s != TSDS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s = check_batch_sorted(series, count, x_dtype, st);
  if (s != TSDS_OK) return s;
  const StreamConfig cfg;
  BatchLayout L = make_layout(algo, series, count, y_dtype, cfg.window_bytes);
  Scratch sc;
  BT_CK(scratch_alloc(sc, L.total, st));
  char* base = static_cast<char*>(sc.p);
  bind_layout(L, base, y_dtype, cfg.window_bytes, cfg.variant);
  BT_CK(cudaMemcpyAsync(base + L.off_desc, L.host.data(), L.host.size() * sizeof(SeriesDev),
                        cudaMemcpyHostToDevice, st));
  s = launch_maps(L, base, y_dtype, cfg.window_bytes, st);
  if (s != TSDS_OK) return s;
  s = enqueue(L, base, algo, batch_has_x(series, count), x_dtype, y_dtype, nan, cfg, st);
  if (s != TSDS_OK) return s;
  // the pageable descriptor copy was staged by the runtime before cudaMemcpyAsync returned
  return TSDS_OK;
}

tsds_status tsds_plan_create(tsds_plan* plan, tsds_algo algo, const tsds_series* series, int64_t count,
                             tsds_dtype x_dtype, tsds_dtype y_dtype, tsds_nan_mode nan, int flags, void* stream) {
  if (!plan) return fail(TSDS_EINVAL, "tsds_plan_create: plan is NULL");
  *plan = nullptr;
  tsds_status s = check_series(algo, series, count, x_dtype, y_dtype, nan);
  if (s != TSDS_OK) return s;
  if (flags & ~(TSDS_PLAN_GRAPH | TSDS_PLAN_AUTOTUNE)) return fail(TSDS_EINVAL, "tsds_plan_create: unknown flags");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s = check_batch_sorted(series, count, x_dtype, st);
  if (s != TSDS_OK) return s;
  tsds_plan_s* p = new tsds_plan_s();
  PlanImpl* P = &p->impl;
  P->algo = algo;
  P->x_dtype = x_dtype;
  P->y_dtype = y_dtype;
  P->nan = nan;
  P->has_x = batch_has_x(series, count);
  P->L = make_layout(algo, series, count, y_dtype, kCandidates[0].window_bytes);
  cudaError_t e = take_injected_alloc_failure() ? cudaErrorMemoryAllocation : cudaMalloc(&P->base, P->L.total);
  if (e != cudaSuccess) {
    delete p;
    return fail(TSDS_ENOMEM, "tsds_plan_create: cudaMalloc(%zu): %s", P->L.total, cudaGetErrorString(e));
  }
  bind_layout(P->L, P->base, y_dtype, kCandidates[0].window_bytes, kCandidates[0].variant);
  if (cudaStreamCreateWithFlags(&P->fork.side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->fork.fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->fork.join, cudaEventDisableTiming) != cudaSuccess) {
    tsds_plan_destroy(p);
    return fail(TSDS_ECUDA, "tsds_plan_create: side stream or events could not be created");
  }

  int choice = -1;   // the default shape
  const std::string key = tune_key(algo, y_dtype, P->has_x, P->L);
  bool have = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) { choice = it->second; have = true; }
  }
  if ((flags & TSDS_PLAN_AUTOTUNE) && !have && P->L.total_windows > 0) {
    float best = 1e30f;
    for (int c = 0; c < kNumCandidates; ++c) {
      float ms = 0.f;
      s = time_candidate(P, kCandidates[c], st, &ms);
      if (s != TSDS_OK) { tsds_plan_destroy(p); return s; }
      P->tune_ms[c] = ms;
      if (ms < best) { best = ms; choice = c; }
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = choice;
    tune_store_locked();
  }
  P->tuned_index = choice;
  P->cfg = choice >= 0 ? kCandidates[choice] : StreamConfig();
  s = upload(P->L, P->base, y_dtype, P->cfg, st);
  if (s != TSDS_OK) { tsds_plan_destroy(p); return s; }

  if (flags & TSDS_PLAN_GRAPH) {
    // one run outside the capture first: every kernel of the sequence is
    // loaded and its launch shape looked up before capturing, since a module
    // load inside a capture invalidates it
    s = enqueue(P->L, P->base, algo, P->has_x, x_dtype, y_dtype, nan, P->cfg, st, P->fork);
    if (s != TSDS_OK) { tsds_plan_destroy(p); return s; }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { tsds_plan_destroy(p); return fail(TSDS_ECUDA, "plan warm-up: %s", cudaGetErrorString(e)); }
    cudaStream_t cap;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) { tsds_plan_destroy(p); return fail(TSDS_ECUDA, "graph capture stream: %s", cudaGetErrorString(e)); }
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      // kernels recorded into the graph count when the graph is launched
      const long long before = tsds_kernel_launches();
      s = enqueue(P->L, P->base, algo, P->has_x, x_dtype, y_dtype, nan, P->cfg, cap, P->fork);
      P->graph_kernels = (int)(tsds_kernel_launches() - before);
      note_launch(-P->graph_kernels);
      cudaError_t e2 = cudaStreamEndCapture(cap, &P->graph);
      if (s == TSDS_OK && e2 == cudaSuccess) e = cudaGraphInstantiate(&P->exec, P->graph, 0);
      else if (e2 != cudaSuccess) e = e2;
    }
    cudaStreamDestroy(cap);
    if (s != TSDS_OK) { tsds_plan_destroy(p); return s; }
    if (e != cudaSuccess) { tsds_plan_destroy(p); return fail(TSDS_ECUDA, "graph capture: %s", cudaGetErrorString(e)); }
  }
  *plan = p;
  return TSDS_OK;
}

tsds_status tsds_plan_execute(tsds_plan plan, void* stream) {
  if (!plan) return fail(TSDS_EINVAL, "tsds_plan_execute: plan is NULL");
  PlanImpl* P = &plan->impl;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (P->exec) {
    note_launch(P->graph_kernels);
    BT_CK(cudaGraphLaunch(P->exec, st));
    return TSDS_OK;
  }
  return enqueue(P->L, P->base, P->algo, P->has_x, P->x_dtype, P->y_dtype, P->nan, P->cfg, st, P->fork);
}

tsds_status tsds_plan_info(tsds_plan plan, int64_t* window_bytes, int* ctas_per_sm, int64_t* windows,
                           int64_t* scratch_bytes, int* variant) {
  if (!plan) return fail(TSDS_EINVAL, "tsds_plan_info: plan is NULL");
  PlanImpl* P = &plan->impl;
  if (window_bytes) *window_bytes = P->cfg.window_bytes;
  if (ctas_per_sm) *ctas_per_sm = P->cfg.ctas_per_sm;
  if (windows) *windows = P->L.total_windows;
  if (scratch_bytes) *scratch_bytes = (int64_t)P->L.total;
  if (variant) {
    StreamConfig c = P->cfg;
    c.mean_bin_bytes = P->L.mean_bin_bytes;
    // the automatic variant runs a launch per group
    *variant = c.variant == STREAM_AUTO ? STREAM_AUTO : stream_variant_for(c, dtype_size(P->y_dtype));
  }
  return TSDS_OK;
}

tsds_status tsds_plan_destroy(tsds_plan plan) {
  if (!plan) return TSDS_OK;
  PlanImpl* P = &plan->impl;
  cudaError_t e = cudaSuccess;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  if (P->fork.fork) cudaEventDestroy(P->fork.fork);
  if (P->fork.join) cudaEventDestroy(P->fork.join);
  if (P->base) {
    // plans own plain device memory: make sure no queued work still uses it
    e = cudaDeviceSynchronize();
    cudaFree(P->base);
  }
  if (P->fork.side) cudaStreamDestroy(P->fork.side);
  delete plan;
  if (e != cudaSuccess) return fail(TSDS_ECUDA, "tsds_plan_destroy: %s", cudaGetErrorString(e));
  return TSDS_OK;
}

}  // extern "C"
