// emit.cu -- turns per-bin selections into the output index list.
//
// MinMax emits {argmin, argmax} of each non-empty bin, M4 {first, argmin,
// argmax, last} and EveryNth {first} (Section 1); each bin's selections are written once
// each, in increasing order, and bins follow each other, so the output is
// strictly increasing.  Empty bins (possible with gaps in x) emit nothing,
// which is why fewer than n_out indices can come back (Section 2.3 footnote).
// One CTA per series: per-thread runs of bins, a block-wide exclusive scan of
// their counts, then a second pass that writes.  A single series with many
// bins takes the tiled form below (many CTAs).
#include "device.cuh"
#include "internal.h"

namespace tsds {

constexpr int kEmitThreads = 1024;

template <int ALGO>
__device__ __forceinline__ int bin_select(const SeriesDev& S, int64_t b, int64_t (&v)[4]) {
  const int64_t lo = __ldg(S.edges + b), hi = __ldg(S.edges + b + 1);
  if (hi <= lo) return 0;
  if (ALGO == ALGO_EVERYNTH) {
    v[0] = lo;
    return 1;
  }
  const int64_t mn = S.res[2 * b], mx = S.res[2 * b + 1];
  int k = 0;
  if (ALGO == ALGO_MINMAX) {
    v[0] = min(mn, mx); v[1] = max(mn, mx);
    k = v[0] == v[1] ? 1 : 2;
  } else {
    // sort {lo, mn, mx, hi-1}: lo is the smallest and hi-1 the largest
    int64_t a = min(mn, mx), c = max(mn, mx);
    int64_t t[4] = {lo, a, c, hi - 1};
    k = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (k == 0 || t[i] != v[k - 1]) v[k++] = t[i];
  }
  return k;
}

template <int ALGO>
__global__ void __launch_bounds__(kEmitThreads) k_emit(const SeriesDev* __restrict__ sd, SeriesDev single) {
  const SeriesDev S = sd ? sd[blockIdx.x] : single;
  const int64_t nb = S.nb;
  if (nb <= 0) return;
  if (S.status && *S.status) {
    // the streaming pass failed on the device (a bounded wait ran out): report it as -status
    if (threadIdx.x == 0 && S.out_count) *S.out_count = -(int64_t)*S.status;
    return;
  }
  __shared__ int64_t warp_tot[kEmitThreads / 32];
  __shared__ int64_t total_sh;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t per = (nb + blockDim.x - 1) / blockDim.x;
  const int64_t b0 = min((int64_t)tid * per, nb), b1 = min(b0 + per, nb);
  int64_t v[4];
  int64_t local = 0;
  for (int64_t b = b0; b < b1; ++b) local += bin_select<ALGO>(S, b, v);
  // block exclusive scan of `local`
  int64_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    int64_t wv = lane < nw ? warp_tot[lane] : 0;
    int64_t wi = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < nw) warp_tot[lane] = wi - wv;   // exclusive prefix of warp totals
    if (lane == nw - 1) total_sh = wi;
  }
  __syncthreads();
  int64_t off = warp_tot[warp] + incl - local;
  for (int64_t b = b0; b < b1; ++b) {
    const int k = bin_select<ALGO>(S, b, v);
    for (int i = 0; i < k; ++i) emit_point(S, off + i, v[i]);
    off += k;
  }
  if (tid == 0 && S.out_count) *S.out_count = total_sh;
}

// Many bins in one series: tiles of kTileBins bins, one CTA each.  Pass 1
// counts every tile's selections, one CTA turns the counts into exclusive
// prefix sums, pass 2 places each tile at its prefix, scans within it and
// writes.  The last tile also writes the total.
constexpr int kTileThreads = 256;
constexpr int kTileItems = 4;
constexpr int64_t kTileBins = kTileThreads * kTileItems;

template <int ALGO>
__device__ __forceinline__ int64_t tile_thread_count(const SeriesDev& S, int64_t b0, int64_t b1) {
  int64_t v[4], c = 0;
  for (int64_t b = b0; b < b1; ++b) c += bin_select<ALGO>(S, b, v);
  return c;
}

// Block-wide exclusive scan of one value per thread (kTileThreads); returns
// the thread's prefix and sets *total.
__device__ __forceinline__ int64_t tile_scan(int64_t x, int64_t* warp_tot, int64_t* total) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int64_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = kTileThreads / 32;
    const int64_t wv = lane < nw ? warp_tot[lane] : 0;
    int64_t wi = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < nw) warp_tot[lane] = wi - wv;
    if (lane == nw - 1) *total = wi;
  }
  __syncthreads();
  return warp_tot[warp] + incl - x;
}

template <int ALGO>
__global__ void __launch_bounds__(kTileThreads) k_emit_count(SeriesDev S, int64_t* __restrict__ tile_count) {
  __shared__ int64_t warp_tot[kTileThreads / 32];
  __shared__ int64_t total;
  const int64_t b0 = (int64_t)blockIdx.x * kTileBins + (int64_t)threadIdx.x * kTileItems;
  const int64_t c = tile_thread_count<ALGO>(S, min(b0, S.nb), min(b0 + kTileItems, S.nb));
  tile_scan(c, warp_tot, &total);
  if (threadIdx.x == 0) tile_count[blockIdx.x] = total;
}

template <int ALGO>
__global__ void __launch_bounds__(kTileThreads) k_emit_write(SeriesDev S, const int64_t* __restrict__ tile_count) {
  __shared__ int64_t warp_tot[kTileThreads / 32];
  __shared__ int64_t total, before_sh;
  if (S.status && *S.status) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && S.out_count) *S.out_count = -(int64_t)*S.status;
    return;
  }
  // selections of the tiles before this one (k_scan_tiles made tile_count exclusive)
  if (threadIdx.x == 0) before_sh = tile_count[blockIdx.x];
  __syncthreads();
  const int64_t base = before_sh;
  const int64_t b0 = min((int64_t)blockIdx.x * kTileBins + (int64_t)threadIdx.x * kTileItems, S.nb);
  const int64_t b1 = min(b0 + kTileItems, S.nb);
  const int64_t c = tile_thread_count<ALGO>(S, b0, b1);
  int64_t off = base + tile_scan(c, warp_tot, &total);
  int64_t v[4];
  for (int64_t b = b0; b < b1; ++b) {
    const int k = bin_select<ALGO>(S, b, v);
    for (int i = 0; i < k; ++i) emit_point(S, off + i, v[i]);
    off += k;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0 && S.out_count) *S.out_count = base + total;
}

// Exclusive prefix sums of the tiles' counts, in place (one CTA; each thread
// scans a contiguous run of tiles).
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(int64_t* __restrict__ tile_count, int64_t tiles) {
  __shared__ int64_t warp_tot[kScanThreads / 32];
  __shared__ int64_t total;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t per = (tiles + kScanThreads - 1) / kScanThreads;
  const int64_t t0 = min((int64_t)tid * per, tiles), t1 = min(t0 + per, tiles);
  int64_t local = 0;
  for (int64_t t = t0; t < t1; ++t) local += tile_count[t];
  int64_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int64_t wv = warp_tot[lane];
    int64_t wi = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t v = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += v;
    }
    warp_tot[lane] = wi - wv;
    if (lane == 31) total = wi;
  }
  __syncthreads();
  int64_t run = warp_tot[warp] + incl - local;
  for (int64_t t = t0; t < t1; ++t) {
    const int64_t c = tile_count[t];
    tile_count[t] = run;
    run += c;
  }
}

int64_t emit_tiles(int64_t nb) { return (nb + kTileBins - 1) / kTileBins; }

cudaError_t launch_emit_tiled(const SeriesDev& single, Algo algo, int64_t* tile_count, cudaStream_t st) {
  const int64_t tiles = emit_tiles(single.nb);
  if (tiles <= 0) return cudaSuccess;
  note_launch(3);
  if (algo == ALGO_MINMAX) {
    k_emit_count<ALGO_MINMAX><<<(unsigned)tiles, kTileThreads, 0, st>>>(single, tile_count);
    k_scan_tiles<<<1, kScanThreads, 0, st>>>(tile_count, tiles);
    k_emit_write<ALGO_MINMAX><<<(unsigned)tiles, kTileThreads, 0, st>>>(single, tile_count);
  } else if (algo == ALGO_EVERYNTH) {
    k_emit_count<ALGO_EVERYNTH><<<(unsigned)tiles, kTileThreads, 0, st>>>(single, tile_count);
    k_scan_tiles<<<1, kScanThreads, 0, st>>>(tile_count, tiles);
    k_emit_write<ALGO_EVERYNTH><<<(unsigned)tiles, kTileThreads, 0, st>>>(single, tile_count);
  } else {
    k_emit_count<ALGO_M4><<<(unsigned)tiles, kTileThreads, 0, st>>>(single, tile_count);
    k_scan_tiles<<<1, kScanThreads, 0, st>>>(tile_count, tiles);
    k_emit_write<ALGO_M4><<<(unsigned)tiles, kTileThreads, 0, st>>>(single, tile_count);
  }
  return cudaGetLastError();
}

cudaError_t launch_emit(const SeriesDev* s_dev, int count, const SeriesDev& single, Algo algo,
                        cudaStream_t st) {
  const SeriesDev* arr = (count > 1 || s_dev) ? s_dev : nullptr;
  // a batch: 256 threads per series, so that eight series' CTAs share an SM
  int64_t threads = arr ? 256 : kEmitThreads;
  if (!arr && single.nb < 1024) threads = ((single.nb + 31) / 32) * 32;
  if (threads < 32) threads = 32;
  note_launch();
  if (algo == ALGO_MINMAX)
    k_emit<ALGO_MINMAX><<<count, (unsigned)threads, 0, st>>>(arr, single);
  else if (algo == ALGO_EVERYNTH)
    k_emit<ALGO_EVERYNTH><<<count, (unsigned)threads, 0, st>>>(arr, single);
  else
    k_emit<ALGO_M4><<<count, (unsigned)threads, 0, st>>>(arr, single);
  return cudaGetLastError();
}

}  // namespace tsds
