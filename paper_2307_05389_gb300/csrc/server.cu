// server.cu -- the served form: viewport queries over resident series with
// continuous batching.
//
// The paper's setting is interactive exploration, where every zoom or pan
// re-downsamples the visible range (Section 1) and the downsampling itself
// becomes the bottleneck at scale.  Here a host thread owns a queue of
// queries (series, x range or index range, n_out = pixel width, algorithm)
// and keeps up to `streams` batches in flight on the GPU.  Whenever a batch
// finishes, queued queries are admitted into the next batch while its slot
// count and the device-memory budget allow, so requests that arrive while
// others run join the next launch instead of waiting for a drain.
//
// One batch is one launch sequence on its stream: the ranges are resolved on
// the device (a warp search of x per query), each query becomes a binned
// sub-series with an index offset, the window numbering is scanned on the
// device, the shared binned kernels run with the window count read from
// device memory, MinMaxLTTB queries continue through the LTTB job kernels,
// and one device-to-host copy returns every result.  A host callback on the
// stream marks the batch done.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "lttb.h"

namespace tsds {

// One admitted query as the batch kernels see it.
struct QueryDev {
  const void* y;
  const void* x;
  int64_t n;          // series length
  int32_t algo;
  int32_t nan;
  int32_t by_x;
  int32_t pad;
  double x_lo, x_hi;
  int64_t lo, hi;     // index range (by_x == 0)
  int64_t n_out;
  int64_t n_sel;      // MinMaxLTTB preselection size
  int64_t* out;       // n_out entries
  int64_t* info;      // [count, L, lo, k, m] (count = selected indices)
  int64_t* R;         // MinMaxLTTB points (global indices)
  int64_t* user_count;  // device-output batches: the caller's count word (null for the server)
};

constexpr int kInfoSlots = 8;

template <class X>
__device__ __forceinline__ double xval(const void* x, int64_t j) {
  return (double)static_cast<const X*>(x)[j];
}
__device__ __forceinline__ double x_as_double(const void* x, int dt, int64_t j) {
  switch (dt) {
    case TSDS_I8: return xval<int8_t>(x, j);
    case TSDS_I16: return xval<int16_t>(x, j);
    case TSDS_I32: return xval<int32_t>(x, j);
    case TSDS_I64: return (double)static_cast<const long long*>(x)[j];
    case TSDS_U8: return xval<uint8_t>(x, j);
    case TSDS_U16: return xval<uint16_t>(x, j);
    case TSDS_U32: return xval<uint32_t>(x, j);
    case TSDS_U64: return (double)static_cast<const unsigned long long*>(x)[j];
    case TSDS_F16: return (double)__half2float(static_cast<const __half*>(x)[j]);
    case TSDS_F32: return xval<float>(x, j);
    default: return xval<double>(x, j);
  }
}

// One warp per query: resolve [lo, hi) and fill the binned descriptor.
__global__ void k_resolve(const QueryDev* __restrict__ qd, SeriesDev* __restrict__ sd, int64_t* __restrict__ windows,
                          int8_t* __restrict__ small, int count, int x_dtype, int y_size, int x_size, int64_t welems,
                          int64_t small_bin_bytes) {
  const int lane = threadIdx.x & 31;
  const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (q >= count) return;
  const QueryDev Q = qd[q];
  int64_t lo, hi;
  if (Q.by_x) {
    lo = warp_lower_bound(0, Q.n, [&](int64_t j) { return x_as_double(Q.x, x_dtype, j) >= Q.x_lo; });
    hi = warp_lower_bound(0, Q.n, [&](int64_t j) { return x_as_double(Q.x, x_dtype, j) > Q.x_hi; });
    if (hi < lo) hi = lo;
  } else {
    lo = min(max(Q.lo, (int64_t)0), Q.n);
    hi = min(max(Q.hi, lo), Q.n);
  }
  if (lane != 0) return;
  const int64_t L = hi - lo;
  SeriesDev S;
  memset(&S, 0, sizeof S);
  int64_t off, per = Q.algo == TSDS_ALGO_M4 ? 4 : 2;
  if (Q.algo == 2) {   // MinMaxLTTB: MinMax over the interior, results into R[1..]
    const int64_t n_in = L > 2 ? L - 2 : 0;
    off = lo + 1;
    S.n = n_in;
    S.nb = (L > Q.n_out && Q.n_sel < n_in) ? Q.n_sel / 2 : 0;
    S.idx_bias = lo + 1;
    S.out = Q.R + 1;
    S.out_count = Q.info + 3;
  } else {
    off = lo;
    S.n = L;
    S.nb = L > Q.n_out ? Q.n_out / per : 0;
    S.idx_bias = lo;
    S.out = Q.out;
    S.out_count = Q.info;
  }
  if (S.n > 0) {
    S.y = static_cast<const char*>(Q.y) + off * y_size;
    S.x = Q.x ? static_cast<const char*>(Q.x) + off * x_size : nullptr;
  }
  // scratch pointers were placed by the host into sd[q] already: keep them
  SeriesDev& D = sd[q];
  D.y = S.y;
  D.x = S.x;
  D.n = S.n;
  D.nb = S.nb;
  D.idx_bias = S.idx_bias;
  D.out = S.out;
  D.out_count = S.out_count;
  // bins under the small-bin size go to the lane-group launch (mode 3: tiles
  // of whole bins, plus windows for a register-streaming pass over the bins
  // above the lane-group size limit), bins from there to kSmallMaxBinBytes to
  // a warp per bin (mode 1, no windows), larger ones to the register-streaming
  // launch
  const int64_t bytes = S.n * y_size;
  const int8_t g = S.nb <= 0 ? 0 : bytes < small_bin_bytes * S.nb ? 1 : bytes <= kSmallMaxBinBytes * S.nb ? 2 : 0;
  small[q] = g;
  D.mode = g == 2 ? 1 : g == 1 ? 3 : 0;
  if (g == 1) {
    const GrpShape sh = grp_shape(bytes / S.nb, y_size);
    D.grp = grp_pack(sh.g_log2, sh.tile_rounds);
  }
  windows[q] = S.nb > 0 && g != 2 ? (S.n + welems - 1) / welems : 0;
  Q.info[1] = L;
  Q.info[2] = lo;
}

__device__ __forceinline__ int64_t grp_tiles_of(const SeriesDev& S) {
  const int64_t tile_bins = (int64_t)(32 >> (S.grp & 0xff)) * (S.grp >> 8);
  return (S.nb + tile_bins - 1) / tile_bins;
}

// Exclusive prefix sum over the CTA's threads (blockDim.x a multiple of 32, at
// most 1024); *total gets the sum.  Every thread calls it.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* warp_tot, int64_t* total) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
  int64_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    const int64_t wv = lane < nw ? warp_tot[lane] : 0;
    int64_t wi = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t u = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += u;
    }
    if (lane < nw) warp_tot[lane] = wi - wv;
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  const int64_t r = warp_tot[w] + incl - v;
  __syncthreads();   // warp_tot is reused by the next scan
  return r;
}

// Window bases of the queries: those with large bins first, then those with
// small bins; total[0] = all windows, total[1] = the large-bin windows (where
// the small-bin range starts).  Queries in mode 1 get CTA bases instead, and
// total[2] = their CTAs; small-bin queries (mode 3) also get tile bases, and
// total[3] = their tiles.  One CTA: each thread takes a run of queries, and
// the runs are placed with block-wide scans.
__global__ void k_scan_windows(SeriesDev* __restrict__ sd, const int64_t* __restrict__ windows,
                               const int8_t* __restrict__ small, int count, int64_t* __restrict__ total) {
  __shared__ int64_t warp_tot[32];
  __shared__ int64_t tot[4];
  const int t = threadIdx.x;
  const int per = (count + blockDim.x - 1) / blockDim.x;
  const int a = min(t * per, count), b = min(a + per, count);
  int64_t s[4] = {0, 0, 0, 0};
  for (int i = a; i < b; ++i) {
    s[small[i]] += small[i] == 2 ? (sd[i].nb + kBinsPerCta - 1) / kBinsPerCta : windows[i];
    if (small[i] == 1) s[3] += grp_tiles_of(sd[i]);
  }
  int64_t r[4];
  for (int g = 0; g < 4; ++g) r[g] = block_exclusive_scan(s[g], warp_tot, &tot[g]);
  r[1] += tot[0];   // the small-bin windows follow the large-bin ones
  if (t == 0) {
    total[0] = tot[0] + tot[1];
    total[1] = tot[0];
    total[2] = tot[2];
    total[3] = tot[3];
  }
  for (int i = a; i < b; ++i) {
    const int g = small[i];
    sd[i].win_base = r[g];
    r[g] += g == 2 ? (sd[i].nb + kBinsPerCta - 1) / kBinsPerCta : windows[i];
    if (g == 1) {
      sd[i].tile_base = r[3];
      r[3] += grp_tiles_of(sd[i]);
    }
  }
}

// MinMaxLTTB: complete the point set R = [lo, preselection..., hi-1] and its
// size m; small ranges keep every point.
__global__ void k_close_queries(const QueryDev* __restrict__ qd, int count) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const QueryDev Q = qd[q];
  if (Q.algo != 2) return;
  const int64_t L = Q.info[1], lo = Q.info[2];
  int64_t m;
  if (L <= 2) {
    for (int64_t i = 0; i < L; ++i) Q.R[i] = lo + i;
    m = L;
  } else {
    const int64_t k = Q.info[3];
    Q.R[0] = lo;
    Q.R[k + 1] = lo + L - 1;
    m = k + 2;
  }
  Q.info[4] = m;
}

// Device-output batches: each query's count goes to the caller's count word.
__global__ void k_copy_counts(const QueryDev* __restrict__ qd, int count) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const QueryDev Q = qd[q];
  if (Q.user_count) *Q.user_count = Q.info[0];
}
}  // namespace tsds

using namespace tsds;

namespace {

double now_us() {
  return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

struct SeriesHost {
  const void* x;
  const void* y;
  int64_t n;
};

struct Ticket {
  tsds_query q;
  double t_submit = 0, t_done = 0;
  bool done = false;
  tsds_status status = TSDS_OK;
  int64_t L = 0;
  std::vector<int64_t> result;
};

struct Slot;

struct Server {
  tsds_server_config cfg;
  tsds_dtype x_dtype, y_dtype;
  int device = 0;
  std::vector<SeriesHost> series;
  std::mutex mu;
  std::condition_variable cv, cv_done;
  std::deque<int64_t> queue;
  std::unordered_map<int64_t, Ticket> tickets;
  std::vector<Slot*> slots;
  std::thread th;
  bool stop = false;
  int64_t next_id = 1;
  int64_t inflight_bytes = 0;
  // statistics
  std::vector<double> latencies;
  int64_t submitted = 0, completed = 0, batches = 0, points = 0;
  double t_first = -1, t_last = 0;
  tsds_status sticky = TSDS_OK;
  char sticky_msg[256] = "";
};

struct Slot {
  Server* srv = nullptr;
  cudaStream_t st = nullptr;
  bool busy = false;
  volatile bool finished = false;
  std::vector<int64_t> ids;
  std::vector<size_t> out_off;   // per query: offset (in int64) of its results in the output slab
  std::vector<int64_t> n_outs;
  size_t bytes = 0;              // scratch admitted
  size_t out_words = 0;
  void* pin_in = nullptr;
  size_t pin_in_cap = 0;
  int64_t* pin_out = nullptr;
  size_t pin_out_cap = 0;
};

void CUDART_CB on_batch_done(void* p) {
  Slot* s = static_cast<Slot*>(p);
  {
    std::lock_guard<std::mutex> lk(s->srv->mu);
    s->finished = true;
  }
  s->srv->cv.notify_all();
}

int64_t nb_of(const tsds_query& q);
int64_t lttb_m_max(const tsds_query& q);

// Device scratch one query may need (upper bound: its range may be the whole series).
size_t query_bytes(const Server& S, const tsds_query& q, int64_t window_bytes) {
  const int64_t n = S.series[(size_t)q.series].n;
  const int64_t ys = dtype_size(S.y_dtype);
  const int64_t nb = nb_of(q);
  const int64_t windows = (n * ys + window_bytes - 1) / window_bytes + 1;
  size_t b = sizeof(QueryDev) + sizeof(SeriesDev) + 8 + up256((size_t)(nb + 1) * 8) + up256((size_t)nb * 16) +
             (size_t)nb * 4 + (size_t)windows * (4 + 2 * sizeof(Piece)) + 1024;
  b += (size_t)(q.n_out + kInfoSlots) * 8;
  if (q.algo == 2) {
    const int64_t m_max = lttb_m_max(q);
    const int64_t B = q.n_out - 2;
    const int64_t K = (m_max - 2 + B - 1) / B;
    b += up256((size_t)m_max * 8 * 3) + lttb_job_scratch(m_max, B, K) +
         sizeof(LttbJob) + sizeof(PointsJob) + 512;
  }
  return b;
}

#define SV_CK(call)                                                                   \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      snprintf(err, errlen, "%s: %s", #call, cudaGetErrorString(e_));                 \
      return e_ == cudaErrorMemoryAllocation ? TSDS_ENOMEM : TSDS_ECUDA;              \
    }                                                                                 \
  } while (0)

int64_t nb_of(const tsds_query& q) {
  if (q.algo == 2) return (2 * ((q.n_out * q.minmax_ratio) / 2)) / 2;
  return q.n_out / (q.algo == TSDS_ALGO_M4 ? 4 : 2);
}

int64_t lttb_m_max(const tsds_query& q) { return std::max(2 * ((q.n_out * q.minmax_ratio) / 2) + 2, q.n_out) + 2; }

// Enqueues one batch on the slot's stream.  Called without the server lock:
// everything it needs from the server is in `qs` and `ser` (the series of
// each query) and the server's fixed dtypes.  With dev_out (one batched call
// rather than the server), query i writes its indices to dev_out[i] and its
// count to dev_count[i] on the device, the descriptors are staged from
// pageable memory, and nothing is copied back.
tsds_status launch_batch(const Server& S, Slot& sl, const std::vector<tsds_query>& qs,
                         const std::vector<SeriesHost>& ser, bool has_x, char* err, size_t errlen,
                         int64_t* const* dev_out = nullptr, int64_t* const* dev_count = nullptr) {
  const bool device_out = dev_out != nullptr;
  const int count = (int)qs.size();
  const int64_t window_bytes = kWindowBytes;
  const int64_t ys = dtype_size(S.y_dtype);
  const int64_t welems = window_bytes / ys;
  std::vector<int> lt;
  for (int i = 0; i < count; ++i)
    if (qs[i].algo == 2) lt.push_back(i);
  const int nlt = (int)lt.size();
  // ---- device layout: the descriptor block first, in the same order as the
  // pinned staging block, so one copy places all descriptors
  const size_t sz_q = (size_t)count * sizeof(QueryDev), sz_s = (size_t)count * sizeof(SeriesDev);
  const size_t sz_l = (size_t)nlt * sizeof(LttbJob), sz_p = (size_t)nlt * sizeof(PointsJob);
  const size_t off_q = 0, off_sd = off_q + sz_q, off_ljobs = off_sd + sz_s, off_pjobs = off_ljobs + sz_l;
  const size_t in_bytes = off_pjobs + sz_p;
  size_t o = up256(in_bytes);
  const size_t off_win = o; o = up256(o + (size_t)count * 8 + 32);   // windows; all, large-bin windows; CTAs; tiles
  const size_t off_small = o; o = up256(o + (size_t)count);
  std::vector<size_t> off_edges(count), off_res(count), off_cnt(count), off_R(count), off_lt(count);
  int64_t max_nb = 0, win_ub = 0, cta_ub = 0, tile_ub = 0;
  for (int i = 0; i < count; ++i) {
    const int64_t nb = nb_of(qs[i]);
    max_nb = std::max(max_nb, nb);
    cta_ub += (nb + kBinsPerCta - 1) / kBinsPerCta;
    tile_ub += nb;   // a tile holds at least one bin
    off_edges[i] = o; o = up256(o + (size_t)(nb + 1) * 8);
    off_res[i] = o;   o = up256(o + (size_t)nb * 16);
    win_ub += (ser[i].n * ys + window_bytes - 1) / window_bytes + 1;
  }
  const size_t zero_begin = o;    // piece counters and the work counter start at zero
  for (int i = 0; i < count; ++i) { off_cnt[i] = o; o += (size_t)nb_of(qs[i]) * 4; }
  o = up256(o);
  const size_t off_work = o; o = up256(o + 3 * sizeof(WorkCounters));   // one per launch of the split pass
  const size_t zero_end = o;
  const size_t off_map = o;   o = up256(o + (size_t)win_ub * 4);
  const size_t off_first = o; o = up256(o + (size_t)win_ub * sizeof(Piece));
  const size_t off_last = o;  o = up256(o + (size_t)win_ub * sizeof(Piece));
  const size_t off_ctas = o;  o = up256(o + (size_t)cta_ub * 4);
  const size_t off_tiles = o; o = up256(o + (size_t)tile_ub * 4);
  // results: per query n_out indices then kInfoSlots info words, contiguous for one copy back
  const size_t off_out = o;
  sl.out_off.assign(count, 0);
  sl.n_outs.assign(count, 0);
  size_t words = 0;
  for (int i = 0; i < count; ++i) {
    sl.out_off[i] = words;
    sl.n_outs[i] = device_out ? 0 : qs[i].n_out;
    words += (size_t)sl.n_outs[i] + kInfoSlots;
  }
  o = up256(o + words * 8);
  int64_t lt_max_B = 0, lt_max_m = 0;
  for (int i : lt) {
    const int64_t m_max = lttb_m_max(qs[i]);
    const int64_t B = qs[i].n_out - 2;
    const int64_t K = (m_max - 2 + B - 1) / B;
    off_R[i] = o;  o = up256(o + (size_t)m_max * 8 * 3);   // R, py, px
    off_lt[i] = o; o = up256(o + lttb_job_scratch(m_max, B, K));
    lt_max_B = std::max(lt_max_B, B);
    lt_max_m = std::max(lt_max_m, m_max);
  }
  const size_t total = o;

  // ---- staging: pinned for the server (the slot is idle, so its buffers are
  // free), pageable for a one-shot batched call
  std::vector<char> pageable;
  if (device_out) {
    pageable.assign(in_bytes, 0);
  } else if (sl.pin_in_cap < in_bytes) {
    if (sl.pin_in) cudaFreeHost(sl.pin_in);
    sl.pin_in = nullptr;
    sl.pin_in_cap = 0;
    SV_CK(cudaMallocHost(&sl.pin_in, in_bytes * 2));
    sl.pin_in_cap = in_bytes * 2;
  }
  if (!device_out && sl.pin_out_cap < words) {
    if (sl.pin_out) cudaFreeHost(sl.pin_out);
    sl.pin_out = nullptr;
    sl.pin_out_cap = 0;
    SV_CK(cudaMallocHost((void**)&sl.pin_out, words * 2 * 8));
    sl.pin_out_cap = words * 2;
  }
  sl.out_words = words;

  Scratch scr;   // returned to the library pool in stream order when this function returns
  SV_CK(scratch_alloc(scr, total, sl.st));
  char* base = static_cast<char*>(scr.p);
  char* stage = device_out ? pageable.data() : static_cast<char*>(sl.pin_in);
  QueryDev* hq = reinterpret_cast<QueryDev*>(stage + off_q);
  SeriesDev* hs = reinterpret_cast<SeriesDev*>(stage + off_sd);
  LttbJob* hl = reinterpret_cast<LttbJob*>(stage + off_ljobs);
  PointsJob* hp = reinterpret_cast<PointsJob*>(stage + off_pjobs);
  int64_t* outbase = reinterpret_cast<int64_t*>(base + off_out);
  for (int i = 0; i < count; ++i) {
    const tsds_query& q = qs[i];
    QueryDev& d = hq[i];
    memset(&d, 0, sizeof d);
    d.y = ser[i].y;
    d.x = ser[i].x;
    d.n = ser[i].n;
    d.algo = q.algo;
    d.nan = q.nan;
    d.by_x = q.by_x;
    d.x_lo = q.x_lo;
    d.x_hi = q.x_hi;
    d.lo = q.lo;
    d.hi = q.hi;
    d.n_out = q.n_out;
    d.n_sel = q.algo == 2 ? 2 * ((q.n_out * q.minmax_ratio) / 2) : 0;
    d.out = device_out ? dev_out[i] : outbase + sl.out_off[i];
    d.info = outbase + sl.out_off[i] + sl.n_outs[i];
    d.user_count = device_out ? dev_count[i] : nullptr;
    d.R = q.algo == 2 ? reinterpret_cast<int64_t*>(base + off_R[i]) : nullptr;
    SeriesDev& s = hs[i];
    memset(&s, 0, sizeof s);   // k_resolve fills the range-dependent fields
    s.edges = reinterpret_cast<int64_t*>(base + off_edges[i]);
    s.res = reinterpret_cast<int64_t*>(base + off_res[i]);
    s.cnt = reinterpret_cast<uint32_t*>(base + off_cnt[i]);
    s.status = &reinterpret_cast<WorkCounters*>(base + off_work)->status;
  }
  for (int t = 0; t < nlt; ++t) {
    const int i = lt[t];
    const tsds_query& q = qs[i];
    const int64_t m_max = lttb_m_max(q);
    int64_t* R = hq[i].R;
    double* py = reinterpret_cast<double*>(R + m_max);
    double* px = py + m_max;
    LttbJob& J = hl[t];
    memset(&J, 0, sizeof J);
    J.px = px;
    J.py = py;
    J.m_dev = hq[i].info + 4;
    J.B = q.n_out - 2;
    J.K = (m_max - 2 + J.B - 1) / J.B;
    J.nan = q.nan;
    J.R = R;
    J.out = hq[i].out;
    J.out_count = hq[i].info;
    lttb_job_bind(J, base + off_lt[i], m_max);
    PointsJob& P = hp[t];
    memset(&P, 0, sizeof P);
    P.x = ser[i].x;
    P.x_dtype = S.x_dtype;
    P.y = ser[i].y;
    P.y_dtype = S.y_dtype;
    P.R = R;
    P.m_dev = hq[i].info + 4;
    P.px = px;
    P.py = py;
  }
  // ---- launches
  cudaStream_t st = sl.st;
  SV_CK(cudaMemcpyAsync(base, stage, in_bytes, cudaMemcpyHostToDevice, st));
  const QueryDev* dq = reinterpret_cast<const QueryDev*>(base + off_q);
  SeriesDev* dsd = reinterpret_cast<SeriesDev*>(base + off_sd);
  SV_CK(cudaMemsetAsync(base + zero_begin, 0, zero_end - zero_begin, st));
  SV_CK(cudaMemsetAsync(outbase, 0, words * 8, st));
  int64_t* windows = reinterpret_cast<int64_t*>(base + off_win);
  int64_t* total_dev = windows + count;   // [all windows, large-bin windows, CTAs, tiles]
  int8_t* small = reinterpret_cast<int8_t*>(base + off_small);
  const bool can_split = true;
  note_launch();
  k_resolve<<<(count + 7) / 8, 256, 0, st>>>(dq, dsd, windows, small, count, (int)S.x_dtype, (int)ys,
                                             has_x ? (int)dtype_size(S.x_dtype) : 0, welems,
                                             can_split ? kGrpServedMaxBinBytes : 0);
  SV_CK(cudaGetLastError());
  note_launch();
  k_scan_windows<<<1, 1024, 0, st>>>(dsd, windows, small, count, total_dev);
  SV_CK(cudaGetLastError());
  SV_CK(launch_window_map(dsd, count, reinterpret_cast<int32_t*>(base + off_map), S.y_dtype, st, window_bytes));
  SV_CK(launch_cta_map(dsd, count, reinterpret_cast<int32_t*>(base + off_ctas), st));
  SV_CK(launch_tile_map(dsd, count, reinterpret_cast<int32_t*>(base + off_tiles), st));
  SV_CK(launch_edges(dsd, count, nullptr, has_x, S.x_dtype, max_nb, st));
  SeriesDev none;
  memset(&none, 0, sizeof none);
  // a batch holds one NaN mode and either M4 or the MinMax-like algorithms (the admission groups them)
  const tsds_nan_mode nan = (tsds_nan_mode)qs[0].nan;
  const bool m4 = qs[0].algo == TSDS_ALGO_M4;
  // the streaming pass: register streaming over the large-bin queries' windows
  // [0, total[1]), the segmented kernel over the small-bin ones [total[1], total[0])
  // (ranges read on the device; an empty range is a launch with nothing to claim)
  const int32_t* map = reinterpret_cast<const int32_t*>(base + off_map);
  Piece* fp = reinterpret_cast<Piece*>(base + off_first);
  Piece* lp = reinterpret_cast<Piece*>(base + off_last);
  WorkCounters* work = reinterpret_cast<WorkCounters*>(base + off_work);
  // mid-size bins: a warp per bin over the CTAs counted on the device
  SV_CK(launch_bins_multi(dsd, reinterpret_cast<const int32_t*>(base + off_ctas), std::max<int64_t>(cta_ub, 1), S.y_dtype,
                          nan, st, total_dev + 2));
  StreamConfig big;
  big.variant = STREAM_LDG;
  big.total_windows_dev = can_split ? total_dev + 1 : total_dev;
  SV_CK(launch_argminmax(dsd, count, none, map, std::max<int64_t>(win_ub, 1), fp, lp, work, S.y_dtype, nan, st, big));
  if (can_split) {
    // small bins: lane groups over the tiles counted on the device, then a
    // register-streaming pass over the small-bin queries' windows
    // [total[1], total[0]) for the bins above the lane-group size limit (it
    // exits at once when there is none)
    GrpShape shp;
    shp.max_bin = kGrpMaxBinBytes / ys;
    SV_CK(launch_argminmax_grp(dsd, none, reinterpret_cast<const int32_t*>(base + off_tiles),
                               std::max<int64_t>(tile_ub, 1), work + 1, S.y_dtype, nan, shp, st, total_dev + 3));
    StreamConfig sm;
    sm.variant = STREAM_LDG;
    sm.total_windows_dev = total_dev;
    sm.window_first_dev = total_dev + 1;
    sm.mean_bin_bytes = kPrefetchOffBinBytes;
    sm.min_bin = shp.max_bin;
    sm.large_dev = &work[1].large;
    SV_CK(launch_argminmax(dsd, count, none, map, std::max<int64_t>(win_ub, 1), fp, lp, work + 2, S.y_dtype, nan, st,
                           sm));
  }
  SV_CK(launch_emit(dsd, count, none, m4 ? ALGO_M4 : ALGO_MINMAX, st));
  SV_CK(launch_iota_batched(dsd, count, st));
  if (nlt > 0) {
    note_launch();
    k_close_queries<<<(count + 255) / 256, 256, 0, st>>>(dq, count);
    SV_CK(cudaGetLastError());
    tsds_status r = launch_points_jobs(reinterpret_cast<const PointsJob*>(base + off_pjobs), nlt, lt_max_m, st);
    if (r != TSDS_OK) { snprintf(err, errlen, "points: %s", tsds_last_error()); return r; }
    r = run_lttb_jobs(hl, reinterpret_cast<const LttbJob*>(base + off_ljobs), nlt, lt_max_B, lt_max_m, st);
    if (r != TSDS_OK) { snprintf(err, errlen, "lttb: %s", tsds_last_error()); return r; }
  }
  if (device_out) {
    note_launch();
    k_copy_counts<<<(count + 255) / 256, 256, 0, st>>>(dq, count);
    SV_CK(cudaGetLastError());
    return TSDS_OK;
  }
  SV_CK(cudaMemcpyAsync(sl.pin_out, outbase, words * 8, cudaMemcpyDeviceToHost, st));
  SV_CK(cudaLaunchHostFunc(st, on_batch_done, &sl));
  return TSDS_OK;
}

// Moves a finished slot's results into its tickets.  Server lock held.
void reap(Server& S, Slot& sl) {
  const double t = now_us();
  for (size_t i = 0; i < sl.ids.size(); ++i) {
    auto it = S.tickets.find(sl.ids[i]);
    if (it == S.tickets.end()) continue;
    Ticket& tk = it->second;
    const int64_t* res = sl.pin_out + sl.out_off[i];
    const int64_t* info = res + sl.n_outs[i];
    int64_t c = info[0];
    if (c < 0 || c > sl.n_outs[i]) {
      tk.status = TSDS_EINTERNAL;
      c = 0;
    }
    tk.result.assign(res, res + c);
    tk.L = info[1];
    tk.done = true;
    tk.t_done = t;
    S.latencies.push_back(t - tk.t_submit);
    S.points += tk.L;
    ++S.completed;
  }
  S.t_last = t;
  S.inflight_bytes -= (int64_t)sl.bytes;
  sl.bytes = 0;
  sl.ids.clear();
  sl.busy = false;
  sl.finished = false;
}

void server_loop(Server* sp) {
  Server& S = *sp;
  cudaSetDevice(S.device);
  char err[256];
  std::unique_lock<std::mutex> lk(S.mu);
  for (;;) {
    for (Slot* sl : S.slots) {
      if (sl->busy && sl->finished) {
        reap(S, *sl);
        S.cv_done.notify_all();
      }
    }
    // admit queued queries into free slots (continuous batching)
    bool blocked = false;
    for (Slot* sl : S.slots) {
      if (sl->busy || S.queue.empty()) continue;
      std::vector<tsds_query> qs;
      std::vector<int64_t> ids;
      std::vector<SeriesHost> ser;
      size_t bytes = 0;
      const tsds_query& head = S.tickets[S.queue.front()].q;
      const int nan = head.nan;
      const bool m4 = head.algo == TSDS_ALGO_M4;
      for (auto it = S.queue.begin(); it != S.queue.end() && (int)qs.size() < S.cfg.max_batch;) {
        const tsds_query& q = S.tickets[*it].q;
        if (q.nan != nan || (q.algo == TSDS_ALGO_M4) != m4) { ++it; continue; }
        const size_t b = query_bytes(S, q, kWindowBytes);
        const bool fits = S.inflight_bytes + (int64_t)(bytes + b) <= S.cfg.memory_budget;
        if (!fits && !(qs.empty() && S.inflight_bytes == 0)) break;   // an oversized query runs alone when idle
        bytes += b;
        qs.push_back(q);
        ser.push_back(S.series[(size_t)q.series]);
        ids.push_back(*it);
        it = S.queue.erase(it);
      }
      if (qs.empty()) { blocked = true; break; }
      sl->ids = ids;
      sl->bytes = bytes;
      sl->busy = true;
      sl->finished = false;
      S.inflight_bytes += (int64_t)bytes;
      ++S.batches;
      const bool has_x = !S.series.empty() && S.series[0].x != nullptr;
      lk.unlock();
      const tsds_status r = launch_batch(S, *sl, qs, ser, has_x, err, sizeof err);
      if (r != TSDS_OK) cudaStreamSynchronize(sl->st);   // no host callback was enqueued for this batch
      lk.lock();
      if (r != TSDS_OK) {
        for (int64_t id : ids) {
          Ticket& tk = S.tickets[id];
          tk.done = true;
          tk.status = r;
          tk.t_done = now_us();
        }
        S.sticky = r;
        snprintf(S.sticky_msg, sizeof S.sticky_msg, "%s", err);
        S.inflight_bytes -= (int64_t)bytes;
        sl->busy = false;
        sl->ids.clear();
        S.cv_done.notify_all();
      }
    }
    bool any_busy = false;
    for (Slot* sl : S.slots) any_busy |= sl->busy;
    if (S.stop && S.queue.empty() && !any_busy) break;
    S.cv.wait(lk, [&] {
      if (S.stop && S.queue.empty()) return true;
      for (Slot* sl : S.slots) {
        if (sl->busy && sl->finished) return true;
        if (!blocked && !sl->busy && !S.queue.empty()) return true;
      }
      return false;
    });
  }
}

}  // namespace

struct tsds_server_s {
  Server s;
};

extern "C" {

tsds_status tsds_server_create(tsds_server* out, const tsds_server_config* cfg, tsds_dtype x_dtype,
                               tsds_dtype y_dtype) {
  if (!out) return fail(TSDS_EINVAL, "tsds_server_create: out is NULL");
  *out = nullptr;
  if (!dtype_valid(y_dtype)) return fail(TSDS_EINVAL, "tsds_server_create: unknown y dtype");
  tsds_server_config c = {2, 256, (int64_t)1 << 30};
  if (cfg) c = *cfg;
  if (c.streams < 1 || c.streams > 16 || c.max_batch < 1 || c.max_batch > 4096 || c.memory_budget < 1)
    return fail(TSDS_EINVAL, "tsds_server_create: streams in [1,16], max_batch in [1,4096], memory_budget > 0");
  tsds_server_s* h = new tsds_server_s();
  Server& S = h->s;
  S.cfg = c;
  S.x_dtype = x_dtype;
  S.y_dtype = y_dtype;
  cudaGetDevice(&S.device);
  for (int i = 0; i < c.streams; ++i) {
    Slot* sl = new Slot();
    sl->srv = &S;
    if (cudaStreamCreateWithFlags(&sl->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete sl;
      tsds_server_destroy(h);
      return fail(TSDS_ECUDA, "tsds_server_create: stream creation failed");
    }
    S.slots.push_back(sl);
    // pinned staging sized for a full batch of typical queries (it grows if a
    // batch needs more), so the first batches do not pay for page-locking
    const size_t in0 = (size_t)c.max_batch * 1024;
    const size_t out0 = (size_t)c.max_batch * (4096 + kInfoSlots);
    if (cudaMallocHost(&sl->pin_in, in0) == cudaSuccess) sl->pin_in_cap = in0;
    else sl->pin_in = nullptr;
    if (cudaMallocHost((void**)&sl->pin_out, out0 * 8) == cudaSuccess) sl->pin_out_cap = out0;
    else sl->pin_out = nullptr;
  }
  {
    // map the device-memory budget into the library's pool once (the pool
    // keeps freed memory), so batches do not wait for the pool to grow
    Scratch warm;
    if (scratch_alloc(warm, (size_t)c.memory_budget, S.slots[0]->st) == cudaSuccess) {
      cudaFreeAsync(warm.p, warm.st);
      warm.p = nullptr;
    }
    cudaStreamSynchronize(S.slots[0]->st);
    cudaGetLastError();
  }
  S.th = std::thread(server_loop, &S);
  *out = h;
  return TSDS_OK;
}

tsds_status tsds_server_add_series(tsds_server h, const void* x, const void* y, int64_t n, int64_t* id) {
  if (!h || !id) return fail(TSDS_EINVAL, "tsds_server_add_series: NULL argument");
  Server& S = h->s;
  if (n < 0 || (n > 0 && !y)) return fail(TSDS_EINVAL, "tsds_server_add_series: bad series");
  if (x && dtype_valid(S.x_dtype)) {
    const tsds_status c = check_sorted_x("tsds_server_add_series", x, S.x_dtype, n, nullptr);
    if (c != TSDS_OK) return c;
  }
  std::lock_guard<std::mutex> lk(S.mu);
  if (!S.series.empty() && (S.series[0].x != nullptr) != (x != nullptr))
    return fail(TSDS_EINVAL, "tsds_server_add_series: either every series has x or none");
  if (x && !dtype_valid(S.x_dtype)) return fail(TSDS_EINVAL, "tsds_server_add_series: the server's x dtype is invalid");
  S.series.push_back(SeriesHost{x, y, n});
  *id = (int64_t)S.series.size() - 1;
  return TSDS_OK;
}

tsds_status tsds_server_submit(tsds_server h, const tsds_query* q, int64_t* ticket) {
  if (!h || !q || !ticket) return fail(TSDS_EINVAL, "tsds_server_submit: NULL argument");
  Server& S = h->s;
  std::lock_guard<std::mutex> lk(S.mu);
  if (q->series < 0 || q->series >= (int64_t)S.series.size()) return fail(TSDS_EINVAL, "tsds_server_submit: unknown series");
  if (q->algo == TSDS_ALGO_MINMAX) {
    if (q->n_out < 2 || q->n_out % 2) return fail(TSDS_EINVAL, "tsds_server_submit: MinMax needs an even n_out >= 2");
  } else if (q->algo == TSDS_ALGO_M4) {
    if (q->n_out < 4 || q->n_out % 4) return fail(TSDS_EINVAL, "tsds_server_submit: M4 needs n_out a multiple of 4");
  } else if (q->algo == 2) {
    if (q->n_out < 3 || q->minmax_ratio < 1 || q->minmax_ratio > (INT64_MAX / 4) / q->n_out)
      return fail(TSDS_EINVAL, "tsds_server_submit: MinMaxLTTB needs n_out >= 3 and minmax_ratio >= 1");
  } else {
    return fail(TSDS_EINVAL, "tsds_server_submit: unknown algorithm %d", q->algo);
  }
  if (q->nan != TSDS_NAN_PROPAGATE && q->nan != TSDS_NAN_IGNORE) return fail(TSDS_EINVAL, "tsds_server_submit: NaN mode");
  if (q->by_x && !S.series[(size_t)q->series].x) return fail(TSDS_EINVAL, "tsds_server_submit: x range on a series without x");
  const int64_t id = S.next_id++;
  Ticket& t = S.tickets[id];
  t.q = *q;
  t.t_submit = now_us();
  if (S.t_first < 0) S.t_first = t.t_submit;
  S.queue.push_back(id);
  ++S.submitted;
  *ticket = id;
  S.cv.notify_all();
  return TSDS_OK;
}

tsds_status tsds_server_result(tsds_server h, int64_t ticket, int64_t timeout_us, int64_t* out, int64_t cap,
                               int64_t* count, int* done, double* latency_us) {
  if (!h) return fail(TSDS_EINVAL, "tsds_server_result: NULL server");
  Server& S = h->s;
  std::unique_lock<std::mutex> lk(S.mu);
  auto it = S.tickets.find(ticket);
  if (it == S.tickets.end()) return fail(TSDS_EINVAL, "tsds_server_result: unknown ticket %lld", (long long)ticket);
  if (!it->second.done && timeout_us != 0) {
    auto pred = [&] { return S.tickets[ticket].done; };
    if (timeout_us < 0) S.cv_done.wait(lk, pred);
    else S.cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred);
    it = S.tickets.find(ticket);
  }
  Ticket& t = it->second;
  if (done) *done = t.done ? 1 : 0;
  if (!t.done) return TSDS_OK;
  if (t.status != TSDS_OK) {
    const tsds_status s = t.status;
    S.tickets.erase(it);
    return fail(s, "tsds_server_result: the batch failed: %s", S.sticky_msg);
  }
  const int64_t c = (int64_t)t.result.size();
  if (count) *count = c;
  if (latency_us) *latency_us = t.t_done - t.t_submit;
  if (out) {
    if (cap < c) return fail(TSDS_EINVAL, "tsds_server_result: out holds %lld, result has %lld", (long long)cap, (long long)c);
    memcpy(out, t.result.data(), (size_t)c * 8);
  }
  S.tickets.erase(it);
  return TSDS_OK;
}

tsds_status tsds_server_stats_get(tsds_server h, tsds_server_stats* st) {
  if (!h || !st) return fail(TSDS_EINVAL, "tsds_server_stats_get: NULL argument");
  Server& S = h->s;
  std::lock_guard<std::mutex> lk(S.mu);
  memset(st, 0, sizeof *st);
  st->submitted = S.submitted;
  st->completed = S.completed;
  st->batches = S.batches;
  st->points = S.points;
  st->bytes = S.points * dtype_size(S.y_dtype);
  st->span_s = S.t_first < 0 ? 0.0 : (S.t_last - S.t_first) / 1e6;
  if (!S.latencies.empty()) {
    std::vector<double> v = S.latencies;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) { return v[(size_t)std::min<double>(v.size() - 1, p * (v.size() - 1) + 0.5)]; };
    st->p50_us = pct(0.50);
    st->p99_us = pct(0.99);
    double s = 0;
    for (double x : v) s += x;
    st->mean_us = s / v.size();
    st->max_us = v.back();
  }
  return TSDS_OK;
}

tsds_status tsds_server_reset_stats(tsds_server h) {
  if (!h) return fail(TSDS_EINVAL, "tsds_server_reset_stats: NULL server");
  Server& S = h->s;
  std::lock_guard<std::mutex> lk(S.mu);
  S.latencies.clear();
  S.submitted = S.completed = S.batches = S.points = 0;
  S.t_first = -1;
  S.t_last = 0;
  return TSDS_OK;
}

tsds_status tsds_server_destroy(tsds_server h) {
  if (!h) return TSDS_OK;
  Server& S = h->s;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    S.stop = true;
  }
  S.cv.notify_all();
  if (S.th.joinable()) S.th.join();
  for (Slot* sl : S.slots) {
    if (sl->st) {
      cudaStreamSynchronize(sl->st);
      cudaStreamDestroy(sl->st);
    }
    if (sl->pin_in) cudaFreeHost(sl->pin_in);
    if (sl->pin_out) cudaFreeHost(sl->pin_out);
    delete sl;
  }
  delete h;
  return TSDS_OK;
}

tsds_status tsds_batched_minmaxlttb(const tsds_series* series, int64_t count, tsds_dtype x_dtype, tsds_dtype y_dtype,
                                    int64_t minmax_ratio, tsds_nan_mode nan, void* stream) {
  if (count < 1 || count > 65535)
    return fail(TSDS_EINVAL, "tsds_batched_minmaxlttb: count must be in [1, 65535] (got %lld)", (long long)count);
  if (!series) return fail(TSDS_EINVAL, "tsds_batched_minmaxlttb: series is NULL");
  if (!dtype_valid(y_dtype)) return fail(TSDS_EINVAL, "tsds_batched_minmaxlttb: unknown y dtype %d", (int)y_dtype);
  if (nan != TSDS_NAN_PROPAGATE && nan != TSDS_NAN_IGNORE)
    return fail(TSDS_EINVAL, "tsds_batched_minmaxlttb: unknown NaN mode %d", (int)nan);
  if (minmax_ratio < 1) return fail(TSDS_EINVAL, "tsds_batched_minmaxlttb: minmax_ratio must be >= 1");
  bool has_x = false;
  for (int64_t i = 0; i < count; ++i)
    if (series[i].n > 0) { has_x = series[i].x != nullptr; break; }
  if (has_x && !dtype_valid(x_dtype)) return fail(TSDS_EINVAL, "tsds_batched_minmaxlttb: unknown x dtype %d", (int)x_dtype);
  for (int64_t i = 0; i < count; ++i) {
    const tsds_series& q = series[i];
    if (q.n < 0) return fail(TSDS_EINVAL, "tsds_batched_minmaxlttb: series %lld: n < 0", (long long)i);
    if (q.n > 0 && (q.x != nullptr) != has_x)
      return fail(TSDS_EINVAL, "tsds_batched_minmaxlttb: series %lld: either every non-empty series has x or none",
                  (long long)i);
    if (q.n_out < 3) return fail(TSDS_EINVAL, "tsds_batched_minmaxlttb: series %lld: n_out must be >= 3", (long long)i);
    if (minmax_ratio > (INT64_MAX / 4) / q.n_out)
      return fail(TSDS_EINVAL, "tsds_batched_minmaxlttb: series %lld: n_out * minmax_ratio overflows", (long long)i);
    if ((q.n > 0 && (!q.y || !q.out)) || !q.out_count)
      return fail(TSDS_EINVAL, "tsds_batched_minmaxlttb: series %lld: NULL buffer", (long long)i);
    if (reinterpret_cast<uintptr_t>(q.y) % dtype_size(y_dtype) ||
        (has_x && reinterpret_cast<uintptr_t>(q.x) % dtype_size(x_dtype)))
      return fail(TSDS_EINVAL, "tsds_batched_minmaxlttb: series %lld: x or y not aligned to its element size",
                  (long long)i);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  tsds_status c = check_batch_sorted(series, count, x_dtype, st);
  if (c != TSDS_OK) return c;
  Server S;
  S.x_dtype = has_x ? x_dtype : TSDS_F64;
  S.y_dtype = y_dtype;
  std::vector<tsds_query> qs((size_t)count);
  std::vector<SeriesHost> ser((size_t)count);
  std::vector<int64_t*> outs((size_t)count), counts((size_t)count);
  for (int64_t i = 0; i < count; ++i) {
    const tsds_series& in = series[i];
    tsds_query& q = qs[(size_t)i];
    memset(&q, 0, sizeof q);
    q.series = i;
    q.algo = TSDS_ALGO_MINMAXLTTB;
    q.nan = nan;
    q.lo = 0;
    q.hi = in.n;
    q.n_out = in.n_out;
    q.minmax_ratio = minmax_ratio;
    ser[(size_t)i] = SeriesHost{has_x ? in.x : nullptr, in.y, in.n};
    outs[(size_t)i] = in.out;
    counts[(size_t)i] = in.out_count;
  }
  Slot sl;
  sl.st = st;
  char err[256] = "";
  const tsds_status r = launch_batch(S, sl, qs, ser, has_x, err, sizeof err, outs.data(), counts.data());
  if (r != TSDS_OK) return fail(r, "tsds_batched_minmaxlttb: %s", err);
  return TSDS_OK;
}

}  // extern "C"
