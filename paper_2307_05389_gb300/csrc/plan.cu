// plan.cu -- bin planning: bin start indices for MinMax / M4 (and the
// MinMaxLTTB preselection), the batched window map and the n_out >= n copy.
//
// The paper's tsdownsample generates bin indices "using a search sorted
// approach" (Section 2.2).  Bin i of nb starts at
//   no x        : ceil(i*(n-1)/nb)                      (index arithmetic)
//   integer x   : first j with (x_j-x_0)*nb >= i*(x_{n-1}-x_0)   (exact, 128-bit)
//   floating x  : first j with x_j >= x_0 + ((x_{n-1}-x_0)*i)/nb (binary64,
//                 each operation rounded to nearest, no fused multiply-add)
// and the last bin ends at n.  For x = 0..n-1 the three rules agree, which is
// the paper's "equally sampled x gives the same output as no x" (Section 2.2).
#include "device.cuh"
#include "internal.h"

namespace tsds {

typedef unsigned __int128 u128;

__global__ void k_edges_index(const SeriesDev* sd, SeriesDev single, int count) {
  const SeriesDev S = count == 1 && sd == nullptr ? single : sd[blockIdx.y];
  const int64_t nb = S.nb;
  if (nb <= 0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= nb; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t v;
    if (i == nb) {
      v = S.n;
    } else {
      v = (int64_t)muldiv_ceil((uint64_t)i, (uint64_t)(S.n - 1), (uint64_t)nb);
    }
    S.edges[i] = v;
  }
}

template <class X>
struct XInt {
  static constexpr bool is_signed = (X)(-1) < (X)0;
  __device__ static u128 off(const X* x, int64_t j, X x0) {
    X v = __ldg(x + j);
    if (is_signed) return (u128)((__int128)(int64_t)v - (__int128)(int64_t)x0);
    return (u128)((uint64_t)v - (uint64_t)x0);
  }
};

template <class X>
__device__ __forceinline__ double x_as_f64(const X* x, int64_t j) { return (double)__ldg(x + j); }
template <>
__device__ __forceinline__ double x_as_f64<__half>(const __half* x, int64_t j) {
  return (double)__half2float(ldg_elem<__half>(x + j));
}

// With many small bins the edges are found in two launches: PHASE 1 searches
// all of x for every kEdgeGroup-th edge, PHASE 2 searches each other edge
// only between the two group edges around it.  Both the integer rule and the
// binary64 rule give edge values non-decreasing in i, so for sorted x edge i
// of group k lies in [s_{kG}, s_{(k+1)G}] (s_nb = n).  PHASE 0 is the single
// launch (every edge over all of x).  Measured on GB300 with 10^9 float32
// points: two levels gain 19 % per call at 256-point bins and 7 % at 512,
// and lose 2-4 % from 2048 points on (the second launch waits for the first),
// so they serve single-series calls with at least 4096 bins of at most 512
// points.
constexpr int64_t kEdgeGroup = 32;
constexpr int64_t kEdgesTwoLevelMinBins = 4096;
constexpr int64_t kEdgesTwoLevelMaxBinPoints = 512;
// The single launch with bins of at most this many points on average searches
// with kEdgeLanes lanes per edge from a window around the edge's expected
// position (four edges per warp, a few 8-way rounds) instead of a warp per
// edge over all of x.
constexpr int64_t kEdgesGuessMaxBinPoints = 8192;
constexpr int kEdgeLanes = 8;

template <class X, bool FLOATX, int PHASE>
__global__ void k_edges_x(const SeriesDev* sd, SeriesDev single, int count) {
  const SeriesDev S = count == 1 && sd == nullptr ? single : sd[blockIdx.y];
  const int64_t nb = S.nb;
  if (nb <= 0) return;
  const X* x = static_cast<const X*>(S.x);
  const int64_t n = S.n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  if (PHASE != 2 && blockIdx.x == 0 && threadIdx.x == 0) { S.edges[0] = 0; S.edges[nb] = n; }
  if (PHASE != 0 || n <= kEdgesGuessMaxBinPoints * nb) {
    // groups of kEdgeLanes lanes, one edge each, whose first round probes a
    // window around the edge's expected position: its index position for
    // evenly spread x over all of x (phases 0 and 1), or the position
    // interpolated between the two group edges around it (phase 2, which
    // searches only between them).  A miss costs a search over the rest.
    constexpr int per = 32 / kEdgeLanes;
    const int sub = lane / kEdgeLanes;
    const int64_t stride = PHASE == 1 ? kEdgeGroup : 1;
    const int64_t bin_pts = n / nb;
    for (int64_t k0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * per;; k0 += warps_total * per) {
      // this warp's edges: the k-th edge of the phase, i = stride * (k + 1)
      // (phase 2 skips the group edges), per lanes group
      int64_t i;
      if (PHASE == 2) {
        const int64_t k = k0 + sub;
        i = k / (kEdgeGroup - 1) * kEdgeGroup + k % (kEdgeGroup - 1) + 1;
        if (k0 / (kEdgeGroup - 1) * kEdgeGroup + k0 % (kEdgeGroup - 1) + 1 >= nb) break;
      } else {
        i = stride * (k0 + sub + 1);
        if (stride * (k0 + 1) >= nb) break;
      }
      const bool act = i < nb;
      int64_t lo = 0, hi = n, g = 0, radius = 0;
      if (act) {
        if (PHASE == 2) {
          const int64_t gb = i - i % kEdgeGroup;
          lo = S.edges[gb];
          hi = gb + kEdgeGroup < nb ? S.edges[gb + kEdgeGroup] : n;
          const int64_t span_bins = (gb + kEdgeGroup < nb ? kEdgeGroup : nb - gb);
          g = lo + (int64_t)muldiv_floor((uint64_t)(i - gb), (uint64_t)(hi - lo), (uint64_t)span_bins);
          radius = 4 * ((hi - lo) / span_bins) + 2 * (int64_t)sqrtf((float)(hi - lo)) + 32;
        } else {
          g = (int64_t)muldiv_floor((uint64_t)i, (uint64_t)(n - 1), (uint64_t)nb);
          radius = 4 * bin_pts + 2 * (int64_t)sqrtf((float)n) + 32;
        }
      }
      int64_t e;
      if constexpr (FLOATX) {
        const double x0 = x_as_f64<X>(x, 0);
        const double xl = x_as_f64<X>(x, n - 1);
        const double span = __dsub_rn(xl, x0);
        const double edge = __dadd_rn(x0, __ddiv_rn(__dmul_rn(span, (double)i), (double)nb));
        e = group_lower_bound<kEdgeLanes>(lo, hi, g - radius, g + radius, act,
                                          [&](int64_t j) { return x_as_f64<X>(x, j) >= edge; });
      } else {
        const X x0 = __ldg(x);
        const u128 span = XInt<X>::off(x, n - 1, x0);
        const u128 rhs = (u128)i * span;
        e = group_lower_bound<kEdgeLanes>(lo, hi, g - radius, g + radius, act,
                                          [&](int64_t j) { return XInt<X>::off(x, j, x0) * (u128)nb >= rhs; });
      }
      if (act && lane % kEdgeLanes == 0) S.edges[i] = e;
    }
    return;
  }
  const int64_t step = PHASE == 1 ? kEdgeGroup : 1;
  for (int64_t i = step + ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * step; i < nb; i += warps_total * step) {
    if (PHASE == 2 && i % kEdgeGroup == 0) continue;
    int64_t lo = 0, hi = n;
    if (PHASE == 2) {
      const int64_t g = i - i % kEdgeGroup;
      lo = S.edges[g];
      hi = g + kEdgeGroup < nb ? S.edges[g + kEdgeGroup] : n;
    }
    int64_t e;
    if constexpr (FLOATX) {
      double x0 = x_as_f64<X>(x, 0);
      double xl = x_as_f64<X>(x, n - 1);
      double span = __dsub_rn(xl, x0);
      double edge = __dadd_rn(x0, __ddiv_rn(__dmul_rn(span, (double)i), (double)nb));
      e = warp_lower_bound(lo, hi, [&](int64_t j) { return x_as_f64<X>(x, j) >= edge; });
    } else {
      X x0 = __ldg(x);
      u128 span = XInt<X>::off(x, n - 1, x0);
      u128 rhs = (u128)i * span;
      e = warp_lower_bound(lo, hi, [&](int64_t j) { return XInt<X>::off(x, j, x0) * (u128)nb >= rhs; });
    }
    if (lane == 0) S.edges[i] = e;
  }
}

template <class X, bool FLOATX>
static void launch_edges_x(dim3 grid, int threads, const SeriesDev* arr, const SeriesDev& single, int count,
                           int64_t max_nb, bool two_level, cudaStream_t st) {
  if (!two_level) {
    note_launch();
    k_edges_x<X, FLOATX, 0><<<grid, threads, 0, st>>>(arr, single, count);
    return;
  }
  int64_t cblocks = (max_nb / kEdgeGroup + 7) / 8;
  if (cblocks < 1) cblocks = 1;
  if (cblocks > 65535) cblocks = 65535;
  note_launch(2);
  k_edges_x<X, FLOATX, 1><<<dim3((unsigned)cblocks, grid.y), threads, 0, st>>>(arr, single, count);
  k_edges_x<X, FLOATX, 2><<<grid, threads, 0, st>>>(arr, single, count);
}

cudaError_t launch_edges(const SeriesDev* s_dev, int count, const SeriesDev* s_host_single,
                         bool has_x, tsds_dtype x_dtype, int64_t max_nb, cudaStream_t st) {
  SeriesDev single = s_host_single ? *s_host_single : SeriesDev{};
  const SeriesDev* arr = s_host_single ? nullptr : s_dev;
  if (max_nb <= 0) return cudaSuccess;
  if (!has_x) {
    int threads = 256;
    int64_t blocks = (max_nb + 1 + threads - 1) / threads;
    if (blocks > 65535) blocks = 65535;
    dim3 grid((unsigned)blocks, (unsigned)count);
    note_launch();
    k_edges_index<<<grid, threads, 0, st>>>(arr, single, count);
    return cudaGetLastError();
  }
  int threads = 256;   // 8 warps, one edge each
  int64_t blocks = (max_nb + 7) / 8;
  if (blocks < 1) blocks = 1;
  if (blocks > 65535) blocks = 65535;
  dim3 grid((unsigned)blocks, (unsigned)count);
  const bool two_level = s_host_single && max_nb >= kEdgesTwoLevelMinBins &&
                         single.n <= kEdgesTwoLevelMaxBinPoints * single.nb;
  switch (x_dtype) {
    case TSDS_I8: launch_edges_x<int8_t, false>(grid, threads, arr, single, count, max_nb, two_level, st); break;
    case TSDS_I16: launch_edges_x<int16_t, false>(grid, threads, arr, single, count, max_nb, two_level, st); break;
    case TSDS_I32: launch_edges_x<int32_t, false>(grid, threads, arr, single, count, max_nb, two_level, st); break;
    case TSDS_I64: launch_edges_x<int64_t, false>(grid, threads, arr, single, count, max_nb, two_level, st); break;
    case TSDS_U8: launch_edges_x<uint8_t, false>(grid, threads, arr, single, count, max_nb, two_level, st); break;
    case TSDS_U16: launch_edges_x<uint16_t, false>(grid, threads, arr, single, count, max_nb, two_level, st); break;
    case TSDS_U32: launch_edges_x<uint32_t, false>(grid, threads, arr, single, count, max_nb, two_level, st); break;
    case TSDS_U64: launch_edges_x<uint64_t, false>(grid, threads, arr, single, count, max_nb, two_level, st); break;
    case TSDS_F16: launch_edges_x<__half, true>(grid, threads, arr, single, count, max_nb, two_level, st); break;
    case TSDS_F32: launch_edges_x<float, true>(grid, threads, arr, single, count, max_nb, two_level, st); break;
    case TSDS_F64: launch_edges_x<double, true>(grid, threads, arr, single, count, max_nb, two_level, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

__global__ void k_window_map(const SeriesDev* sd, int32_t* win_series, int64_t welems) {
  const SeriesDev S = sd[blockIdx.x];
  if (S.nb <= 0 || S.mode == 1 || S.mode == 2) return;
  int64_t k = (S.n + welems - 1) / welems;
  for (int64_t w = threadIdx.x; w < k; w += blockDim.x) win_series[S.win_base + w] = (int32_t)blockIdx.x;
}

cudaError_t launch_window_map(const SeriesDev* s_dev, int count, int32_t* win_series,
                              tsds_dtype y_dtype, cudaStream_t st, int64_t window_bytes) {
  note_launch();
  k_window_map<<<count, 256, 0, st>>>(s_dev, win_series, window_bytes / dtype_size(y_dtype));
  return cudaGetLastError();
}

// cta_series[win_base + c] = the series, for each CTA c of a series in mode 1.
__global__ void k_cta_map(const SeriesDev* sd, int32_t* cta_series) {
  const SeriesDev S = sd[blockIdx.x];
  if (S.nb <= 0 || S.mode != 1) return;
  const int64_t ctas = (S.nb + kBinsPerCta - 1) / kBinsPerCta;
  for (int64_t c = threadIdx.x; c < ctas; c += blockDim.x) cta_series[S.win_base + c] = (int32_t)blockIdx.x;
}

cudaError_t launch_cta_map(const SeriesDev* s_dev, int count, int32_t* cta_series, cudaStream_t st) {
  note_launch();
  k_cta_map<<<count, 256, 0, st>>>(s_dev, cta_series);
  return cudaGetLastError();
}

// tile_series[tile_base + t] = the series, for each lane-group tile t of a series in mode 2 or 3.
__global__ void k_tile_map(const SeriesDev* sd, int32_t* tile_series) {
  const SeriesDev S = sd[blockIdx.x];
  if (S.nb <= 0 || (S.mode != 2 && S.mode != 3)) return;
  const int64_t tile_bins = (int64_t)(32 >> (S.grp & 0xff)) * (S.grp >> 8);
  const int64_t tiles = (S.nb + tile_bins - 1) / tile_bins;
  for (int64_t t = threadIdx.x; t < tiles; t += blockDim.x) tile_series[S.tile_base + t] = (int32_t)blockIdx.x;
}

cudaError_t launch_tile_map(const SeriesDev* s_dev, int count, int32_t* tile_series, cudaStream_t st) {
  note_launch();
  k_tile_map<<<count, 256, 0, st>>>(s_dev, tile_series);
  return cudaGetLastError();
}

// One CTA per series; only series whose n_out >= n (nb == 0) write.
__global__ void k_iota_batched(const SeriesDev* sd) {
  const SeriesDev S = sd[blockIdx.x];
  if (S.nb != 0) return;
  for (int64_t i = threadIdx.x; i < S.n; i += blockDim.x) emit_point(S, i, i);
  if (threadIdx.x == 0) *S.out_count = S.n;
}

cudaError_t launch_iota_batched(const SeriesDev* s_dev, int count, cudaStream_t st) {
  note_launch();
  k_iota_batched<<<count, 256, 0, st>>>(s_dev);
  return cudaGetLastError();
}

__global__ void k_iota(int64_t* out, int64_t n, int64_t* count, const void* y, const void* x, Gather g) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    out[i] = i;
    gather_point(g, i, y, x, i);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && count) *count = n;
}

cudaError_t launch_iota(int64_t* out, int64_t n, int64_t* count, cudaStream_t st, const void* y, const void* x,
                        const Gather* g) {
  int64_t blocks = (n + 255) / 256;
  if (blocks < 1) blocks = 1;
  int cap = device_sm_count() * 8;
  if (blocks > cap) blocks = cap;
  Gather none{nullptr, nullptr, 0, 0};
  note_launch();
  k_iota<<<(unsigned)blocks, 256, 0, st>>>(out, n, count, y, x, g ? *g : none);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- checked mode

// The bin searches need x sorted non-decreasing (Section 3: x gives the
// position of each point on the horizontal axis).  Element i is out of order
// when it is NaN or larger than element i+1; the smallest such i lands in
// *first_bad (left untouched when x is in order).
template <class X>
__device__ __forceinline__ bool x_gt(X a, X b) { return a > b; }
template <>
__device__ __forceinline__ bool x_gt<__half>(__half a, __half b) { return __half2float(a) > __half2float(b); }
template <class X>
__device__ __forceinline__ bool x_nan(X) { return false; }
template <>
__device__ __forceinline__ bool x_nan<__half>(__half a) { return __hisnan(a); }
template <>
__device__ __forceinline__ bool x_nan<float>(float a) { return isnan(a); }
template <>
__device__ __forceinline__ bool x_nan<double>(double a) { return isnan(a); }

template <class X>
__global__ void k_check_sorted(const X* __restrict__ x, int64_t n, unsigned long long* first_bad) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const X a = x[i];
    const bool bad = x_nan<X>(a) || (i + 1 < n && x_gt<X>(a, x[i + 1]));
    if (bad) atomicMin(first_bad, (unsigned long long)i);
  }
}

cudaError_t launch_check_sorted(const void* x, tsds_dtype xd, int64_t n, unsigned long long* first_bad,
                                cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t need = (n + 255) / 256;
  const int64_t full = (int64_t)device_sm_count() * 8;
  const unsigned grid = (unsigned)(need < full ? need : full);
  note_launch();
  switch (xd) {
    case TSDS_I8: k_check_sorted<<<grid, 256, 0, st>>>(static_cast<const int8_t*>(x), n, first_bad); break;
    case TSDS_I16: k_check_sorted<<<grid, 256, 0, st>>>(static_cast<const int16_t*>(x), n, first_bad); break;
    case TSDS_I32: k_check_sorted<<<grid, 256, 0, st>>>(static_cast<const int32_t*>(x), n, first_bad); break;
    case TSDS_I64: k_check_sorted<<<grid, 256, 0, st>>>(static_cast<const int64_t*>(x), n, first_bad); break;
    case TSDS_U8: k_check_sorted<<<grid, 256, 0, st>>>(static_cast<const uint8_t*>(x), n, first_bad); break;
    case TSDS_U16: k_check_sorted<<<grid, 256, 0, st>>>(static_cast<const uint16_t*>(x), n, first_bad); break;
    case TSDS_U32: k_check_sorted<<<grid, 256, 0, st>>>(static_cast<const uint32_t*>(x), n, first_bad); break;
    case TSDS_U64: k_check_sorted<<<grid, 256, 0, st>>>(static_cast<const uint64_t*>(x), n, first_bad); break;
    case TSDS_F16: k_check_sorted<<<grid, 256, 0, st>>>(static_cast<const __half*>(x), n, first_bad); break;
    case TSDS_F32: k_check_sorted<<<grid, 256, 0, st>>>(static_cast<const float*>(x), n, first_bad); break;
    case TSDS_F64: k_check_sorted<<<grid, 256, 0, st>>>(static_cast<const double*>(x), n, first_bad); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace tsds
