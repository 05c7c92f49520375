// noalloc.cu -- tsds_minmax_noalloc: MinMax whose scratch memory is a fixed
// array compiled into the library, for callers that cannot allocate.
//
// Who needs it: a caller whose device memory is entirely owned by another
// allocator (a framework's caching allocator, a memory-capped service) where
// a fresh cudaMalloc can fail; a latency-bound interaction loop (the
// zoom/pan redraws downsampling serves) where cudaMalloc/cudaFree may
// synchronise the whole device and stall other streams; code that must do
// all of its allocation at start-up.  tsds_minmax draws scratch from the
// library's stream-ordered pool instead, which allocates on first use and
// when a call needs more than the pool holds.
//
// How: the per-call scratch of the MinMax pipeline (bin edges, per-bin
// results, per-bin piece counters, the work counter and the per-window piece
// slots) lives in g_scratch below.  Host code cannot use g_scratch's name as
// a device address, so the first call on each device, with that device
// current, looks its address up with cudaGetSymbolAddress and caches it.
// Nothing on this path calls cudaMalloc, cudaFree, a pool or any allocating
// routine, and it does not create the library's memory pool.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>

#include <mutex>

#include <string.h>

#include "internal.h"

namespace tsds {

// The static scratch: 8 MiB on every device that loads this library, held
// until the process exits.
constexpr size_t kNoallocScratchBytes = 8u << 20;
static __device__ __align__(256) unsigned char g_scratch[kNoallocScratchBytes];

tsds_status fail(tsds_status s, const char* fmt, ...);

namespace {

constexpr int kMaxDevices = 64;

struct NoallocDevice {
  unsigned char* scratch = nullptr;   // device address of g_scratch
  int sm_count = 0;
};
std::mutex g_na_mu;
NoallocDevice g_na_dev[kMaxDevices];

// Address of g_scratch and the SM count on the current device, looked up once
// per device with that device current.
cudaError_t noalloc_device(NoallocDevice** out) {
  int d = 0;
  cudaError_t e = cudaGetDevice(&d);
  if (e != cudaSuccess) return e;
  if (d < 0 || d >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_na_mu);
  NoallocDevice& s = g_na_dev[d];
  if (!s.scratch) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
    if (e != cudaSuccess) return e;
    s.sm_count = sms;
    s.scratch = static_cast<unsigned char*>(p);
  }
  *out = &s;
  return cudaSuccess;
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

// Forgets every looked-up address (tsds_shutdown): after a device reset the
// old address would be stale, so the next call looks it up again.
void noalloc_forget_devices() {
  std::lock_guard<std::mutex> lk(g_na_mu);
  for (auto& d : g_na_dev) d = NoallocDevice{};
}

namespace {

__global__ void k_iota_na(int64_t* out, int64_t n, int64_t* count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = i;
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = n;
}

#define NA_CK(call)                                                                   \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(TSDS_ECUDA, "tsds_minmax_noalloc: %s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

}  // namespace
}  // namespace tsds

using namespace tsds;

extern "C" tsds_status tsds_minmax_noalloc(const void* x, tsds_dtype x_dtype, const void* y,
                                           tsds_dtype y_dtype, int64_t n, int64_t n_out,
                                           tsds_nan_mode nan, int64_t* out, int64_t* out_count,
                                           void* stream) {
  if (n < 0) return fail(TSDS_EINVAL, "tsds_minmax_noalloc: n must be >= 0");
  if (!dtype_valid(y_dtype)) return fail(TSDS_EINVAL, "tsds_minmax_noalloc: unknown y dtype %d", (int)y_dtype);
  if (x && !dtype_valid(x_dtype)) return fail(TSDS_EINVAL, "tsds_minmax_noalloc: unknown x dtype %d", (int)x_dtype);
  if (nan != TSDS_NAN_PROPAGATE && nan != TSDS_NAN_IGNORE)
    return fail(TSDS_EINVAL, "tsds_minmax_noalloc: unknown NaN mode %d", (int)nan);
  if ((n > 0 && (!y || !out)) || !out_count) return fail(TSDS_EINVAL, "tsds_minmax_noalloc: NULL buffer");
  if (reinterpret_cast<uintptr_t>(y) % dtype_size(y_dtype) != 0 ||
      (x && reinterpret_cast<uintptr_t>(x) % dtype_size(x_dtype) != 0))
    return fail(TSDS_EINVAL, "tsds_minmax_noalloc: x or y is not aligned to its element size");
  if (n_out < 2 || n_out % 2 != 0)
    return fail(TSDS_EINVAL, "tsds_minmax_noalloc: MinMax needs an even n_out >= 2 (got %lld)", (long long)n_out);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // Scratch needed: edges, per-bin results, per-bin counters, work counter,
  // two piece slots per window.  Checked before any device work.
  const int64_t nb = n_out / 2;
  const int64_t welems = window_elems(y_dtype);
  const int64_t windows = n_out >= n ? 0 : (n + welems - 1) / welems;
  size_t o = 0;
  const size_t off_edges = o; o = up256(o + (size_t)(nb + 1) * 8);
  const size_t off_res = o;   o = up256(o + (size_t)nb * 16);
  const size_t off_cnt = o;   o = up256(o + (size_t)nb * 4);
  const size_t off_work = o;  o = up256(o + sizeof(WorkCounters));
  const size_t off_first = o; o = up256(o + (size_t)windows * sizeof(Piece));
  const size_t off_last = o;  o = up256(o + (size_t)windows * sizeof(Piece));
  if (n_out < n && o > kNoallocScratchBytes) {
    // what fits at this n_out: every 64 KB window of y takes 64 bytes of slots
    const size_t fixed = off_first;
    const size_t max_windows = fixed < kNoallocScratchBytes ? (kNoallocScratchBytes - fixed - 512) / (2 * sizeof(Piece)) : 0;
    return fail(TSDS_EINVAL,
                "tsds_minmax_noalloc: this call needs %zu bytes of scratch but the static scratch holds %zu; "
                "at n_out=%lld at most %zu bytes of y fit (use tsds_minmax for larger inputs)",
                o, kNoallocScratchBytes, (long long)n_out, max_windows * (size_t)kWindowBytes);
  }

  NoallocDevice* dev = nullptr;
  NA_CK(noalloc_device(&dev));
  if (n == 0) {
    NA_CK(cudaMemsetAsync(out_count, 0, sizeof(int64_t), st));
    return TSDS_OK;
  }
  if (n_out >= n) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)dev->sm_count * 8) blocks = (int64_t)dev->sm_count * 8;
    note_launch();
    k_iota_na<<<(unsigned)blocks, 256, 0, st>>>(out, n, out_count);
    NA_CK(cudaGetLastError());
    return TSDS_OK;
  }

  unsigned char* base = dev->scratch;
  // the piece counters and the work counter must start at zero; the array
  // keeps whatever the previous call left in it
  NA_CK(cudaMemsetAsync(base + off_cnt, 0, off_first - off_cnt, st));
  SeriesDev S;
  memset(&S, 0, sizeof S);
  S.y = y;
  S.x = x;
  S.n = n;
  S.nb = nb;
  S.edges = reinterpret_cast<int64_t*>(base + off_edges);
  S.res = reinterpret_cast<int64_t*>(base + off_res);
  S.cnt = reinterpret_cast<uint32_t*>(base + off_cnt);
  S.win_base = 0;
  S.out = out;
  S.out_count = out_count;
  S.idx_bias = 0;
  S.status = &reinterpret_cast<WorkCounters*>(base + off_work)->status;
  NA_CK(launch_edges(nullptr, 1, &S, x != nullptr, x_dtype, nb, st));
  StreamConfig cfg;
  cfg.mean_bin_bytes = n / nb * dtype_size(y_dtype);
  NA_CK(launch_argminmax_sm(S, windows, reinterpret_cast<Piece*>(base + off_first),
                            reinterpret_cast<Piece*>(base + off_last), reinterpret_cast<WorkCounters*>(base + off_work),
                            y_dtype, nan, cfg, dev->sm_count, st));
  NA_CK(launch_emit(nullptr, 1, S, ALGO_MINMAX, st));
  return TSDS_OK;
}
