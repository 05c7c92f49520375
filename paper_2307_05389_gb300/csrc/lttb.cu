// lttb.cu -- LTTB and MinMaxLTTB (Section 1; LTTB is sequential over its
// buckets, Table 1 caption).  Built with -fmad=false, and every binary64
// operation of the area and the means goes through an explicit
// round-to-nearest intrinsic, so no multiply-add is ever fused and the
// selected indices equal those of the plain binary64 definition.
//
// Points are (x_k, y_k) in binary64: x is the point's x or its index.
// B = n_out-2 buckets cover points 1..m-2, bucket j = [1+floor(j(m-2)/B),
// 1+floor((j+1)(m-2)/B)).  The chain keeps point 0, then for j = 0..B-1 picks
// the b in bucket j maximising |(xa-xm)(yb-ya) - (xa-xb)(ym-ya)|, where a is
// the previous pick and (xm, ym) the mean of bucket j+1 (sums in index order
// divided by the count) or, for the last bucket, the last point; ties go to
// the lowest index.  NaN-propagate: a NaN area beats every number and the
// first NaN wins.  NaN-ignore: NaN areas never win and the means leave out
// points whose y is NaN; a bucket with no winner keeps its first index.
//
// GPU shape: the bucket means are independent and run one bucket per thread
// over the whole GPU; the chain is one CTA that walks the buckets, each step a
// block-wide argmax of the areas.
#include "device.cuh"
#include "internal.h"
#include "lttb.h"

namespace tsds {

typedef unsigned __int128 u128;

constexpr int kChainThreads = 512;

__device__ __forceinline__ int64_t bucket_start(int64_t j, int64_t m, int64_t B) {
  return 1 + (int64_t)(((u128)j * (u128)(m - 2)) / (u128)B);
}

__device__ __forceinline__ double load_as_f64(const void* p, int dt, int64_t i) {
  switch (dt) {
    case TSDS_I8: return (double)static_cast<const int8_t*>(p)[i];
    case TSDS_I16: return (double)static_cast<const int16_t*>(p)[i];
    case TSDS_I32: return (double)static_cast<const int32_t*>(p)[i];
    case TSDS_I64: return __ll2double_rn(static_cast<const long long*>(p)[i]);
    case TSDS_U8: return (double)static_cast<const uint8_t*>(p)[i];
    case TSDS_U16: return (double)static_cast<const uint16_t*>(p)[i];
    case TSDS_U32: return (double)static_cast<const uint32_t*>(p)[i];
    case TSDS_U64: return __ull2double_rn(static_cast<const unsigned long long*>(p)[i]);
    case TSDS_F16: return (double)__half2float(static_cast<const __half*>(p)[i]);
    case TSDS_F32: return (double)static_cast<const float*>(p)[i];
    default: return static_cast<const double*>(p)[i];
  }
}

// Points as binary64: py[k] = y[idx(k)], px[k] = x[idx(k)] or idx(k), where
// idx(k) = R[k] when a selection R is given and k otherwise.
__global__ void k_to_f64(const void* x, int x_dtype, const void* y, int y_dtype, const int64_t* R,
                         const int64_t* m_dev, int64_t m_host, double* px, double* py) {
  const int64_t m = m_dev ? *m_dev : m_host;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = R ? R[k] : k;
    py[k] = load_as_f64(y, y_dtype, i);
    if (px) px[k] = x ? load_as_f64(x, x_dtype, i) : (double)i;
  }
}

__device__ __forceinline__ double px_at(const double* px, int64_t k) { return px ? px[k] : (double)k; }

// Means of buckets 1..B-1 (the third vertex of steps 0..B-2).
__global__ void k_lttb_means(const double* __restrict__ px, const double* __restrict__ py,
                             const int64_t* m_dev, int64_t m_host, int64_t B, int nan, double2* means) {
  const int64_t m = m_dev ? *m_dev : m_host;
  if (m <= B + 2) return;   // every point is kept
  for (int64_t j = 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < B; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lo = bucket_start(j, m, B), hi = bucket_start(j + 1, m, B);
    double sx = 0.0, sy = 0.0;
    int64_t c = 0;
    for (int64_t k = lo; k < hi; ++k) {
      const double yk = py[k];
      if (nan == TSDS_NAN_IGNORE && isnan(yk)) continue;
      sx = __dadd_rn(sx, px_at(px, k));
      sy = __dadd_rn(sy, yk);
      ++c;
    }
    means[j] = make_double2(__ddiv_rn(sx, (double)c), __ddiv_rn(sy, (double)c));
  }
}

// Area as an ordered key: larger area, larger key.  NaN-propagate maps a NaN
// area above every number; NaN-ignore maps it to 0, below every area (areas
// are >= +0, whose key is 2^63), so it can never be picked.
template <int NM>
__device__ __forceinline__ uint64_t area_key(double ar) {
  if (isnan(ar)) return NM == TSDS_NAN_PROPAGATE ? kKeyMax : 0ull;
  return f64_bits_key(f64_bits(ar));
}

template <int NM>
__global__ void __launch_bounds__(kChainThreads)
k_lttb_chain(const double* __restrict__ px, const double* __restrict__ py, const int64_t* m_dev,
             int64_t m_host, int64_t B, const double2* __restrict__ means, const int64_t* __restrict__ R,
             int64_t* __restrict__ out, int64_t* __restrict__ out_count) {
  const int64_t m = m_dev ? *m_dev : m_host;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (m <= B + 2) {
    for (int64_t i = tid; i < m; i += blockDim.x) out[i] = R ? R[i] : i;
    if (tid == 0) *out_count = m;
    return;
  }
  __shared__ uint64_t sk[kChainThreads / 32];
  __shared__ int64_t si[kChainThreads / 32];
  int64_t a = 0;
  double xa = px_at(px, 0), ya = py[0];
  if (tid == 0) out[0] = R ? R[0] : 0;
  for (int64_t j = 0; j < B; ++j) {
    const int64_t lo = bucket_start(j, m, B), hi = bucket_start(j + 1, m, B);
    double xm, ym;
    if (j == B - 1) {
      xm = px_at(px, m - 1);
      ym = py[m - 1];
    } else {
      const double2 mm = means[j + 1];
      xm = mm.x;
      ym = mm.y;
    }
    const double dxm = __dsub_rn(xa, xm);   // xa - xm
    const double dym = __dsub_rn(ym, ya);   // ym - ya
    uint64_t bk = 0;
    int64_t bi = kIdxNone;
    for (int64_t b = lo + tid; b < hi; b += blockDim.x) {
      const double t1 = __dmul_rn(dxm, __dsub_rn(py[b], ya));
      const double t2 = __dmul_rn(__dsub_rn(xa, px_at(px, b)), dym);
      const uint64_t k = area_key<NM>(fabs(__dsub_rn(t1, t2)));
      if (k > bk || (k == bk && b < bi)) { bk = k; bi = b; }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const uint64_t k2 = __shfl_xor_sync(0xffffffffu, bk, o);
      const int64_t i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      if (k2 > bk || (k2 == bk && i2 < bi)) { bk = k2; bi = i2; }
    }
    if (lane == 0) { sk[warp] = bk; si[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      const int nw = blockDim.x >> 5;
      bk = lane < nw ? sk[lane] : 0ull;
      bi = lane < nw ? si[lane] : kIdxNone;
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const uint64_t k2 = __shfl_xor_sync(0xffffffffu, bk, o);
        const int64_t i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        if (k2 > bk || (k2 == bk && i2 < bi)) { bk = k2; bi = i2; }
      }
      if (lane == 0) {
        const int64_t pick = (bk == 0ull) ? lo : bi;   // no candidate (NaN-ignore): first index
        si[0] = pick;
        out[j + 1] = R ? R[pick] : pick;
      }
    }
    __syncthreads();
    a = si[0];
    xa = px_at(px, a);
    ya = py[a];
    __syncthreads();
  }
  if (tid == 0) {
    out[B + 1] = R ? R[m - 1] : m - 1;
    *out_count = B + 2;
  }
}

// Completes the MinMaxLTTB point set: R[0] = 0, R[k+1] = n-1, m = k+2 where k
// is the preselection's count.
__global__ void k_close_selection(int64_t* R, const int64_t* k_dev, int64_t n, int64_t* m_dev) {
  const int64_t k = *k_dev;
  R[0] = 0;
  R[k + 1] = n - 1;
  *m_dev = k + 2;
}

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

#define TSDS_CK(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(e_ == cudaErrorMemoryAllocation ? TSDS_ENOMEM : TSDS_ECUDA, "%s: %s", \
                  #call, cudaGetErrorString(e_));                                       \
  } while (0)

// LTTB over m points already in binary64 (m on the device when m_dev is set,
// otherwise m_host), writing R[pick] (or pick) to out.
static tsds_status lttb_core(const double* px, const double* py, const int64_t* m_dev, int64_t m_host,
                             int64_t m_max, int64_t n_out, tsds_nan_mode nan, const int64_t* R,
                             int64_t* out, int64_t* out_count, cudaStream_t st) {
  const int64_t B = n_out - 2;
  Scratch s;
  TSDS_CK(scratch_alloc(s, (size_t)(B + 1) * sizeof(double2), st));
  double2* means = static_cast<double2*>(s.p);
  if (m_max > B + 2) {
    int64_t blocks = (B + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    note_launch();
    note_launch();
  k_lttb_means<<<(unsigned)blocks, 256, 0, st>>>(px, py, m_dev, m_host, B, nan, means);
    TSDS_CK(cudaGetLastError());
  }
  note_launch();
  if (nan == TSDS_NAN_IGNORE)
    k_lttb_chain<TSDS_NAN_IGNORE><<<1, kChainThreads, 0, st>>>(px, py, m_dev, m_host, B, means, R, out, out_count);
  else
    k_lttb_chain<TSDS_NAN_PROPAGATE><<<1, kChainThreads, 0, st>>>(px, py, m_dev, m_host, B, means, R, out, out_count);
  TSDS_CK(cudaGetLastError());
  return TSDS_OK;
}

static unsigned grid_for(int64_t n) {
  int64_t blocks = (n + 255) / 256;
  const int64_t cap = (int64_t)device_sm_count() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (unsigned)blocks;
}

tsds_status run_lttb(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype, int64_t n,
                     int64_t n_out, tsds_nan_mode nan, int64_t* out, int64_t* out_count, cudaStream_t st) {
  if (n == 0) {
    TSDS_CK(cudaMemsetAsync(out_count, 0, sizeof(int64_t), st));
    return TSDS_OK;
  }
  if (n_out >= n) {
    TSDS_CK(launch_iota(out, n, out_count, st));
    return TSDS_OK;
  }
  Scratch s;
  const size_t ybytes = align_up((size_t)n * 8, 256);
  TSDS_CK(scratch_alloc(s, ybytes + (x ? (size_t)n * 8 : 0), st));
  double* py = static_cast<double*>(s.p);
  double* px = x ? reinterpret_cast<double*>(static_cast<char*>(s.p) + ybytes) : nullptr;
  note_launch();
  k_to_f64<<<grid_for(n), 256, 0, st>>>(x, x_dtype, y, y_dtype, nullptr, nullptr, n, px, py);
  TSDS_CK(cudaGetLastError());
  return lttb_core(px, py, nullptr, n, n, n_out, nan, nullptr, out, out_count, st);
}

tsds_status run_minmaxlttb(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                           int64_t n, int64_t n_out, int64_t minmax_ratio, tsds_nan_mode nan,
                           int64_t* out, int64_t* out_count, cudaStream_t st) {
  if (n == 0) {
    TSDS_CK(cudaMemsetAsync(out_count, 0, sizeof(int64_t), st));
    return TSDS_OK;
  }
  if (n_out >= n) {
    TSDS_CK(launch_iota(out, n, out_count, st));
    return TSDS_OK;
  }
  const int64_t n_sel = 2 * ((n_out * minmax_ratio) / 2);
  const int64_t n_in = n - 2;
  if (n_sel >= n_in) {
    // the preselection keeps every interior point: plain LTTB
    return run_lttb(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, st);
  }
  const int64_t m_max = n_sel + 2;
  Scratch s;
  const size_t rbytes = align_up((size_t)m_max * 8, 256);
  const size_t pbytes = align_up((size_t)m_max * 8, 256);
  TSDS_CK(scratch_alloc(s, rbytes + 2 * pbytes + 256, st));
  char* base = static_cast<char*>(s.p);
  int64_t* R = reinterpret_cast<int64_t*>(base);
  double* py = reinterpret_cast<double*>(base + rbytes);
  double* px = reinterpret_cast<double*>(base + rbytes + pbytes);
  int64_t* counts = reinterpret_cast<int64_t*>(base + rbytes + 2 * pbytes);   // [k, m]
  const size_t es_y = (size_t)dtype_size(y_dtype);
  const void* y_in = static_cast<const char*>(y) + es_y;
  const void* x_in = x ? static_cast<const char*>(x) + dtype_size(x_dtype) : nullptr;
  tsds_status r = run_binned_series(x_in, x_dtype, y_in, y_dtype, n_in, n_sel / 2, nan, ALGO_MINMAX,
                                    R + 1, counts, 1, st);
  if (r != TSDS_OK) return r;
  note_launch();
  k_close_selection<<<1, 1, 0, st>>>(R, counts, n, counts + 1);
  TSDS_CK(cudaGetLastError());
  note_launch();
  k_to_f64<<<grid_for(m_max), 256, 0, st>>>(x, x_dtype, y, y_dtype, R, counts + 1, 0, px, py);
  TSDS_CK(cudaGetLastError());
  return lttb_core(px, py, counts + 1, 0, m_max, n_out, nan, R, out, out_count, st);
}

}  // namespace tsds
