// stream_small.cuh -- the MinMax/M4 pass of a single series with small bins
// as a warp per bin (included by argminmax.cu after the other variants).
//
// For an input of up to a few hundred MB in bins of at most 64 KB the window
// machinery is all latency: claiming windows, searching bin starts,
// publishing pieces, and separate launches for the bin starts and the emit
// step.  Here one warp takes one bin (a few register-streaming steps):
// index-bin starts are computed in place (x-space starts come from the edge
// kernel), the warp reduces its bin and writes its selections, and with few
// bins the CTA whose arrival on a device counter is the last one emits the
// sorted output of every bin (a block-wide scan, as the emit kernel does);
// with more, the emit kernels follow.
#pragma once

constexpr int kSmallThreads = 256;          // 8 warps, 8 bins per CTA

// A bin's selections for the emit, read with loads that bypass L1 (the
// selections were written by other CTAs of the same launch).
template <int ALGO>
__device__ __forceinline__ int small_select(const SeriesDev& S, int64_t b, int64_t (&v)[4]) {
  const int64_t lo = __ldcg(S.edges + b), hi = __ldcg(S.edges + b + 1);
  if (hi <= lo) return 0;
  const int64_t mn = __ldcg(S.res + 2 * b), mx = __ldcg(S.res + 2 * b + 1);
  const int64_t a = min(mn, mx), c = max(mn, mx);
  if (ALGO == ALGO_MINMAX) {
    v[0] = a;
    v[1] = c;
    return a == c ? 1 : 2;
  }
  const int64_t t[4] = {lo, a, c, hi - 1};
  int k = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (k == 0 || t[i] != v[k - 1]) v[k++] = t[i];
  return k;
}

// A warp owns its whole bin and reads it in 2 KB steps, one round trip each.
// Before the first step it asks L2 for the bin's bytes from 2 KB on, up to
// kBinPrefetchBytes, so that the later steps find them there (a hint: the
// addresses stay inside the bin).
constexpr int64_t kBinPrefetchBytes = 16384;
template <class T>
__device__ __forceinline__ void prefetch_bin(const T* y, int64_t lo, int64_t hi, int lane) {
  const char* base = reinterpret_cast<const char*>(y + lo);
  const int64_t end = min((hi - lo) * (int64_t)sizeof(T), kBinPrefetchBytes);
  for (int64_t q = 2048 + 128 * lane; q < end; q += 4096) asm volatile("prefetch.global.L2 [%0];" ::"l"(base + q));
}

template <class P, int NM, int ALGO, bool HASX, bool EMIT>
__global__ void __launch_bounds__(kSmallThreads) k_small(SeriesDev S, unsigned* __restrict__ done) {
  using T = typename P::T;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nb = S.nb;
  const int64_t b = (int64_t)blockIdx.x * (kSmallThreads / 32) + warp;
  if (b < nb) {
    int64_t lo, hi;
    if (HASX) {
      lo = __ldg(S.edges + b);
      hi = __ldg(S.edges + b + 1);
    } else {
      lo = (int64_t)muldiv_ceil((uint64_t)b, (uint64_t)(S.n - 1), (uint64_t)nb);
      hi = b + 1 == nb ? S.n : (int64_t)muldiv_ceil((uint64_t)(b + 1), (uint64_t)(S.n - 1), (uint64_t)nb);
      if (lane == 0) {
        S.edges[b] = lo;
        if (b + 1 == nb) S.edges[nb] = S.n;
      }
    }
    if (hi > lo) {
      prefetch_bin(static_cast<const T*>(S.y), lo, hi, lane);
      Cand c = piece_ldg<P>(static_cast<const T*>(S.y), lo, hi);
      finish_bin<P, NM>(c, lo);
      if (lane == 0) {
        S.res[2 * b] = c.imin;
        S.res[2 * b + 1] = c.imax;
      }
    }
  }
  if (!EMIT) return;   // many bins: the emit kernels run next
  // the last CTA to arrive emits every bin
  __shared__ unsigned last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1 ? 1u : 0u;
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ int64_t warp_tot[kSmallThreads / 32];
  __shared__ int64_t total;
  const int64_t per = (nb + kSmallThreads - 1) / kSmallThreads;
  const int64_t b0 = min((int64_t)threadIdx.x * per, nb), b1 = min(b0 + per, nb);
  int64_t v[4];
  int64_t local = 0;
  for (int64_t q = b0; q < b1; ++q) local += small_select<ALGO>(S, q, v);
  int64_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    constexpr int nw = kSmallThreads / 32;
    const int64_t wv = lane < nw ? warp_tot[lane] : 0;
    int64_t wi = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < nw) warp_tot[lane] = wi - wv;
    if (lane == nw - 1) total = wi;
  }
  __syncthreads();
  int64_t off = warp_tot[warp] + incl - local;
  for (int64_t q = b0; q < b1; ++q) {
    const int k = small_select<ALGO>(S, q, v);
    for (int i = 0; i < k; ++i) emit_point(S, off + i, v[i]);
    off += k;
  }
  if (threadIdx.x == 0 && S.out_count) *S.out_count = total;
}

template <class P, int NM, bool EMIT>
static void launch_small_emit(const SeriesDev& S, Algo algo, bool has_x, unsigned* done, unsigned blocks,
                              cudaStream_t st) {
  if (algo == ALGO_MINMAX) {
    if (has_x) k_small<P, NM, ALGO_MINMAX, true, EMIT><<<blocks, kSmallThreads, 0, st>>>(S, done);
    else k_small<P, NM, ALGO_MINMAX, false, EMIT><<<blocks, kSmallThreads, 0, st>>>(S, done);
  } else {
    if (has_x) k_small<P, NM, ALGO_M4, true, EMIT><<<blocks, kSmallThreads, 0, st>>>(S, done);
    else k_small<P, NM, ALGO_M4, false, EMIT><<<blocks, kSmallThreads, 0, st>>>(S, done);
  }
}

template <class P, int NM>
static cudaError_t launch_small_pol(const SeriesDev& S, Algo algo, bool has_x, unsigned* done, bool emit,
                                    cudaStream_t st) {
  const unsigned blocks = (unsigned)((S.nb + kSmallThreads / 32 - 1) / (kSmallThreads / 32));
  note_launch();
  if (emit) launch_small_emit<P, NM, true>(S, algo, has_x, done, blocks, st);
  else launch_small_emit<P, NM, false>(S, algo, has_x, done, blocks, st);
  return cudaGetLastError();
}

// Batched series in mode 1 (bins of a few hundred bytes to 64 KB): CTA c
// takes bins kBinsPerCta*(c - win_base) .. of series cta_series[c], a warp
// each, with the bin starts the edge kernel wrote; the per-series emit runs
// after it.
template <class P, int NM>
__global__ void __launch_bounds__(kSmallThreads) k_bins_multi(const SeriesDev* __restrict__ sd,
                                                              const int32_t* __restrict__ cta_series,
                                                              const int64_t* __restrict__ ctas_dev) {
  using T = typename P::T;
  static_assert(kSmallThreads / 32 == kBinsPerCta, "a warp per bin");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (ctas_dev && (int64_t)blockIdx.x >= *ctas_dev) return;   // a grid sized by a bound
  const SeriesDev S = sd[cta_series[blockIdx.x]];
  const int64_t b = ((int64_t)blockIdx.x - S.win_base) * kBinsPerCta + warp;
  if (b >= S.nb) return;
  const int64_t lo = __ldg(S.edges + b), hi = __ldg(S.edges + b + 1);
  if (hi <= lo) return;
  prefetch_bin(static_cast<const T*>(S.y), lo, hi, lane);
  Cand c = piece_ldg<P>(static_cast<const T*>(S.y), lo, hi);
  finish_bin<P, NM>(c, lo);
  if (lane == 0) {
    S.res[2 * b] = c.imin;
    S.res[2 * b + 1] = c.imax;
  }
}

template <class P, int NM>
static cudaError_t launch_bins_multi_pol(const SeriesDev* sd, const int32_t* cta_series, int64_t ctas,
                                         const int64_t* ctas_dev, cudaStream_t st) {
  note_launch();
  k_bins_multi<P, NM><<<(unsigned)ctas, kSmallThreads, 0, st>>>(sd, cta_series, ctas_dev);
  return cudaGetLastError();
}
