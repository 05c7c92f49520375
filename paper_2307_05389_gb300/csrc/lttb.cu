// lttb.cu -- LTTB and MinMaxLTTB (Section 1; LTTB walks its buckets
// sequentially, Table 1 caption).  Built with -fmad=false, and every binary64
// operation of the means and of the areas that decide a pick goes through an
// explicit round-to-nearest intrinsic, so no multiply-add is ever fused and
// each pick equals the one the plain binary64 definition makes.
//
// Points are (x_k, y_k) in binary64 (x is the point's x or its index).  With
// B = n_out-2 buckets over points 1..m-2, bucket j = [1+floor(j(m-2)/B),
// 1+floor((j+1)(m-2)/B)); the chain keeps point 0, then for j = 0..B-1 picks
// the b in bucket j maximising |(xa-xm)(yb-ya) - (xa-xb)(ym-ya)| (a: the
// previous pick; (xm, ym): the mean of bucket j+1, index-order sums divided by
// the count, or the last point after the last bucket); ties go to the lowest
// index.  NaN-propagate: a NaN area beats every number, first NaN wins.
// NaN-ignore: NaN areas never win, means leave out points whose y is NaN, and
// a bucket with no winner keeps its first index.
//
// GPU shape.  The chain is sequential in j (the paper's reason LTTB is not
// parallel), but its cost can move off the critical path:
//  * Small buckets (at most 32 points, the MinMaxLTTB case): the pick of
//    bucket j depends on the chain only through which point a of bucket j-1
//    was picked.  A transition table best[j][a] is filled for every bucket in
//    parallel (one warp per bucket, exact binary64 areas), and the chain
//    becomes a walk through the table that one warp does from registers,
//    with the next rows loaded ahead.
//  * Large buckets: one CTA walks the buckets.  Each step first scores every
//    point with an FP32 estimate of its area and a rigorous bound on the
//    estimate's error, then evaluates the exact binary64 area only for the
//    points whose bound reaches the best lower bound (usually one or two).
//    Any non-finite or out-of-range value sends the step to the exact path.
//    The next bucket's points are copied into shared memory with cp.async
//    while the current step reduces.
#include "device.cuh"
#include "internal.h"
#include "lttb.h"

namespace tsds {

typedef unsigned __int128 u128;

constexpr int kChainThreads = 256;
constexpr int kTableMaxK = kLttbTableMaxK;  // table mode when every bucket has <= 32 points
constexpr int kPrefetchMaxK = 4096; // chain prefetches buckets up to this size (48 B/point, two buffers)

__device__ __forceinline__ int64_t job_m(const LttbJob& J) { return J.m_dev ? *J.m_dev : J.m_host; }

__device__ __forceinline__ int64_t bucket_start(int64_t j, int64_t m, int64_t B) {
  return 1 + (int64_t)(((u128)j * (u128)(m - 2)) / (u128)B);
}

// The bucket that holds point k (1 <= k <= m-2).
__device__ __forceinline__ int64_t bucket_of(int64_t k, int64_t m, int64_t B) {
  const u128 q1 = (u128)k;   // (k-1) + 1
  int64_t j = (int64_t)((q1 * (u128)B - 1) / (u128)(m - 2));
  if (j > B - 1) j = B - 1;
  if (j < 0) j = 0;
  while (j > 0 && bucket_start(j, m, B) > k) --j;
  while (j < B - 1 && bucket_start(j + 1, m, B) <= k) ++j;
  return j;
}

__device__ __forceinline__ int64_t out_index(const LttbJob& J, int64_t k) { return J.R ? J.R[k] : k + J.bias; }

// Bucket starts walked incrementally: start(j) = 1 + floor(j*(m-2)/B).
struct BucketWalk {
  int64_t q, r, dq, dr, B;
  __device__ void init(int64_t m, int64_t B_) {
    B = B_;
    q = 0;
    r = 0;
    dq = (m - 2) / B_;
    dr = (m - 2) % B_;
  }
  __device__ int64_t start() const { return 1 + q; }
  __device__ void next() {
    q += dq;
    r += dr;
    if (r >= B) { r -= B; ++q; }
  }
};

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

// Doubled triangle area of (a, b, m) exactly as defined: every operation
// rounded to nearest, nothing fused.  dxm = xa - xm and dym = ym - ya.
__device__ __forceinline__ double exact_area(double xa, double ya, double dxm, double dym, double xb, double yb) {
  const double t1 = __dmul_rn(dxm, __dsub_rn(yb, ya));
  const double t2 = __dmul_rn(__dsub_rn(xa, xb), dym);
  return fabs(__dsub_rn(t1, t2));
}

// Area as an ordered key: larger area, larger key.  NaN-propagate maps a NaN
// area above every number; NaN-ignore maps it to 0, below every area (areas
// are >= +0, whose key is 2^63), so it can never be picked.
__device__ __forceinline__ uint64_t area_key(double ar, int nan) {
  if (isnan(ar)) return nan == TSDS_NAN_PROPAGATE ? kKeyMax : 0ull;
  return f64_bits_key(f64_bits(ar));
}

// (key desc, index asc) argmax helpers.
__device__ __forceinline__ void amax_merge(uint64_t& k, int64_t& i, uint64_t k2, int64_t i2) {
  if (k2 > k || (k2 == k && i2 < i)) { k = k2; i = i2; }
}
__device__ __forceinline__ void amax_warp(uint64_t& k, int64_t& i) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const uint64_t k2 = __shfl_xor_sync(0xffffffffu, k, o);
    const int64_t i2 = __shfl_xor_sync(0xffffffffu, i, o);
    amax_merge(k, i, k2, i2);
  }
}

// ---------------------------------------------------------------- points and means

// px[k] = x[i] or i, py[k] = y[i], with i = R[k] or k.
__global__ void k_points(const PointsJob* __restrict__ jobs) {
  const PointsJob J = jobs[blockIdx.y];
  const int64_t m = J.m_dev ? *J.m_dev : J.m_host;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = J.R ? J.R[k] : k;
    J.py[k] = load_as_f64(J.y, J.y_dtype, i);
    J.px[k] = J.x ? load_as_f64(J.x, J.x_dtype, i) : (double)i;
  }
}

// means[j] for buckets 1..B-1 (the third vertex of steps 0..B-2).
__global__ void k_means(const LttbJob* __restrict__ jobs) {
  const LttbJob& J = jobs[blockIdx.y];
  const int64_t m = job_m(J), B = J.B;
  if (m <= B + 2) return;
  for (int64_t j = 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < B; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lo = bucket_start(j, m, B), hi = bucket_start(j + 1, m, B);
    double sx = 0.0, sy = 0.0;
    int64_t c = 0;
    for (int64_t k = lo; k < hi; ++k) {
      const double yk = J.py[k];
      if (J.nan == TSDS_NAN_IGNORE && isnan(yk)) continue;
      sx = __dadd_rn(sx, J.px[k]);
      sy = __dadd_rn(sy, yk);
      ++c;
    }
    J.means[j] = make_double2(__ddiv_rn(sx, (double)c), __ddiv_rn(sy, (double)c));
  }
}

// ---------------------------------------------------------------- table mode

// table[j*K + ai] = (pick in bucket j) - start(j) when the previous pick is
// point start(j-1) + ai (for j = 0 the previous pick is point 0, slot 0).
// One warp per bucket; lanes are the candidates b.
__global__ void k_table(const LttbJob* __restrict__ jobs) {
  const LttbJob& J = jobs[blockIdx.y];
  if (J.mode != 0) return;
  const int64_t m = job_m(J), B = J.B;
  if (m <= B + 2) return;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < B; j += warps) {
    const int64_t lo = bucket_start(j, m, B), hi = bucket_start(j + 1, m, B);
    double xm, ym;
    if (j == B - 1) { xm = J.px[m - 1]; ym = J.py[m - 1]; }
    else { const double2 c = J.means[j + 1]; xm = c.x; ym = c.y; }
    const int64_t b = lo + lane;
    const bool has_b = b < hi;
    const double xb = has_b ? J.px[b] : 0.0, yb = has_b ? J.py[b] : 0.0;
    int64_t alo, ahi;
    if (j == 0) { alo = 0; ahi = 1; }
    else { alo = bucket_start(j - 1, m, B); ahi = lo; }
    for (int64_t a = alo; a < ahi; ++a) {
      const double xa = J.px[a], ya = J.py[a];
      const double dxm = __dsub_rn(xa, xm), dym = __dsub_rn(ym, ya);
      uint64_t k = 0ull;
      int64_t idx = kIdxNone;
      if (has_b) { k = area_key(exact_area(xa, ya, dxm, dym, xb, yb), J.nan); idx = b; }
      amax_warp(k, idx);
      if (lane == 0) J.table[j * J.K + (a - alo)] = (int32_t)((k == 0ull ? lo : idx) - lo);
    }
  }
}

// One warp walks the table.  Rows are loaded kRing steps ahead into
// registers (lane l holds entry l of a row); each step is one shuffle.
constexpr int kRing = 8;

__global__ void k_chase(const LttbJob* __restrict__ jobs) {
  const LttbJob& J = jobs[blockIdx.x];
  const int lane = threadIdx.x & 31;
  const int64_t m = job_m(J), B = J.B;
  if (m <= B + 2) {
    for (int64_t i = lane; i < m; i += 32) J.out[i] = out_index(J, i);
    if (lane == 0) *J.out_count = m;
    return;
  }
  if (J.mode != 0) return;
  const int64_t K = J.K;
  int32_t ring[kRing];
#pragma unroll
  for (int s = 0; s < kRing; ++s) ring[s] = (s < B && lane < K) ? J.table[(int64_t)s * K + lane] : 0;
  BucketWalk w;
  w.init(m, B);
  int64_t a = 0, prev_lo = 0;
  if (lane == 0) J.out[0] = out_index(J, 0);
  for (int64_t j0 = 0; j0 < B; j0 += kRing) {
#pragma unroll
    for (int s = 0; s < kRing; ++s) {
      const int64_t j = j0 + s;
      if (j < B) {
        const int64_t lo = w.start();
        const int ai = (int)(a - prev_lo);   // slot of the previous pick in bucket j-1 (0 for j = 0)
        const int32_t rel = __shfl_sync(0xffffffffu, ring[s], ai);
        const int64_t pick = lo + rel;
        if (lane == 0) J.out[j + 1] = out_index(J, pick);
        a = pick;
        prev_lo = lo;
        w.next();
        const int64_t jn = j + kRing;
        ring[s] = (jn < B && lane < K) ? J.table[jn * K + lane] : 0;
      }
    }
  }
  if (lane == 0) {
    J.out[B + 1] = out_index(J, m - 1);
    *J.out_count = B + 2;
  }
}

// ---------------------------------------------------------------- chain mode

// p32[k] = point k relative to its bucket's first point, rounded to FP32.
__global__ void k_p32(const LttbJob* __restrict__ jobs) {
  const LttbJob& J = jobs[blockIdx.y];
  if (J.mode != 1) return;
  const int64_t m = job_m(J), B = J.B;
  if (m <= B + 2) return;
  for (int64_t k = 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m - 1; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lo = bucket_start(bucket_of(k, m, B), m, B);
    J.p32[k] = make_float2(__double2float_rn(__dsub_rn(J.px[k], J.px[lo])),
                           __double2float_rn(__dsub_rn(J.py[k], J.py[lo])));
  }
}

// A value the FP32 filter accepts: finite, 0 or within [2^-60, 2^60] in magnitude.
__device__ __forceinline__ bool filt_ok(float v) {
  const float a = fabsf(v);
  return a == 0.0f || (a >= 8.6736174e-19f && a <= 1.1529215e18f);
}

struct ChainShared {
  uint64_t key[kChainThreads / 32];
  int64_t idx[kChainThreads / 32];
  float fmax[kChainThreads / 32];
  int bad[kChainThreads / 32];
  int64_t pick;
};

__device__ __forceinline__ float block_max_f(float v, ChainShared& sh, int lane, int warp) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) sh.fmax[warp] = v;
  __syncthreads();
  float r = sh.fmax[0];
  for (int w = 1; w < kChainThreads / 32; ++w) r = fmaxf(r, sh.fmax[w]);
  __syncthreads();
  return r;
}

__device__ __forceinline__ int block_or(int v, ChainShared& sh, int lane, int warp) {
  v = __any_sync(0xffffffffu, v) ? 1 : 0;
  if (lane == 0) sh.bad[warp] = v;
  __syncthreads();
  int r = 0;
  for (int w = 0; w < kChainThreads / 32; ++w) r |= sh.bad[w];
  __syncthreads();
  return r;
}

__device__ __forceinline__ void block_amax(uint64_t& k, int64_t& i, ChainShared& sh, int lane, int warp) {
  amax_warp(k, i);
  if (lane == 0) { sh.key[warp] = k; sh.idx[warp] = i; }
  __syncthreads();
  k = sh.key[0];
  i = sh.idx[0];
  for (int w = 1; w < kChainThreads / 32; ++w) amax_merge(k, i, sh.key[w], sh.idx[w]);
  __syncthreads();
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" :: "r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Copies bucket [lo, hi) (p32, px, py) into shared buffer `buf` with cp.async.
__device__ __forceinline__ void prefetch_bucket(const LttbJob& J, int64_t lo, int64_t hi, float2* s32, double* sx,
                                                double* sy) {
  for (int64_t b = lo + threadIdx.x; b < hi; b += blockDim.x) {
    const int64_t o = b - lo;
    cp_async8(&s32[o], &J.p32[b]);
    cp_async8(&sx[o], &J.px[b]);
    cp_async8(&sy[o], &J.py[b]);
  }
  cp_async_commit();
}

__global__ void __launch_bounds__(kChainThreads) k_chain(const LttbJob* __restrict__ jobs) {
  const LttbJob& J = jobs[blockIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t m = job_m(J), B = J.B;
  if (m <= B + 2 || J.mode != 1) return;   // table-mode jobs and short jobs are done by k_chase
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ ChainShared sh;
  const bool pre = J.K <= kPrefetchMaxK;
  const int64_t K = pre ? J.K : 0;
  // two buffers of (p32, px, py) for K points each
  float2* s32[2];
  double* sx[2];
  double* sy[2];
  {
    unsigned char* p = smem_raw;
    for (int t = 0; t < 2; ++t) {
      sx[t] = reinterpret_cast<double*>(p); p += K * 8;
      sy[t] = reinterpret_cast<double*>(p); p += K * 8;
      s32[t] = reinterpret_cast<float2*>(p); p += K * 8;
    }
  }
  BucketWalk w;
  w.init(m, B);
  int64_t a = 0;
  double xa = J.px[0], ya = J.py[0];
  if (tid == 0) J.out[0] = out_index(J, 0);
  int64_t lo = w.start();
  w.next();
  int64_t hi = w.start();
  if (pre) prefetch_bucket(J, lo, hi, s32[0], sx[0], sy[0]);
  const float u8 = 4.7683716e-07f;   // 8 * 2^-24
  const float u4 = 2.3841858e-07f;   // 4 * 2^-24
  const float tiny = 7.5231638e-37f; // 2^-120
  for (int64_t j = 0; j < B; ++j) {
    const int cur = (int)(j & 1);
    // next bucket's bounds and its prefetch (overlaps this step)
    w.next();
    const int64_t nhi = w.start();
    if (pre) {
      cp_async_wait_all();
      __syncthreads();
      if (j + 1 < B) prefetch_bucket(J, hi, nhi, s32[cur ^ 1], sx[cur ^ 1], sy[cur ^ 1]);
    }
    double xm, ym;
    if (j == B - 1) { xm = J.px[m - 1]; ym = J.py[m - 1]; }
    else { const double2 c = J.means[j + 1]; xm = c.x; ym = c.y; }
    const double dxm = __dsub_rn(xa, xm), dym = __dsub_rn(ym, ya);
    const double X0 = pre ? sx[cur][0] : J.px[lo];
    const double Y0 = pre ? sy[cur][0] : J.py[lo];
    const float al = __double2float_rn(dxm), be = __double2float_rn(dym);
    const float ax = __double2float_rn(__dsub_rn(xa, X0)), ay = __double2float_rn(__dsub_rn(ya, Y0));
    const bool fast = filt_ok(al) && filt_ok(be) && filt_ok(ax) && filt_ok(ay) &&
                      !isnan(dxm) && !isnan(dym) && !isinf(dxm) && !isinf(dym);
    uint64_t bk = 0ull;
    int64_t bi = kIdxNone;
    bool done = false;
    if (fast) {
      // pass 1: best lower bound of the area over the bucket
      float lmax = -INFINITY;
      int bad = 0;
      for (int64_t b = lo + tid; b < hi; b += blockDim.x) {
        const float2 p = pre ? s32[cur][b - lo] : J.p32[b];
        if (!(filt_ok(p.x) && filt_ok(p.y))) { bad = 1; continue; }
        const float d1 = p.y - ay, d2 = ax - p.x;
        const float t1 = al * d1, t2 = d2 * be;
        const float est = fabsf(t1 - t2);
        const float err = u8 * (fabsf(al) * (fabsf(p.y) + fabsf(ay) + fabsf(d1)) +
                                fabsf(be) * (fabsf(p.x) + fabsf(ax) + fabsf(d2))) + u4 * est + tiny;
        lmax = fmaxf(lmax, est - err);
      }
      if (!block_or(bad, sh, lane, warp)) {
        const float L = block_max_f(lmax, sh, lane, warp);
        // pass 2: exact areas of the points whose upper bound reaches L
        for (int64_t b = lo + tid; b < hi; b += blockDim.x) {
          const float2 p = pre ? s32[cur][b - lo] : J.p32[b];
          const float d1 = p.y - ay, d2 = ax - p.x;
          const float t1 = al * d1, t2 = d2 * be;
          const float est = fabsf(t1 - t2);
          const float err = u8 * (fabsf(al) * (fabsf(p.y) + fabsf(ay) + fabsf(d1)) +
                                  fabsf(be) * (fabsf(p.x) + fabsf(ax) + fabsf(d2))) + u4 * est + tiny;
          if (est + err >= L) {
            const double xb = pre ? sx[cur][b - lo] : J.px[b];
            const double yb = pre ? sy[cur][b - lo] : J.py[b];
            amax_merge(bk, bi, area_key(exact_area(xa, ya, dxm, dym, xb, yb), J.nan), b);
          }
        }
        done = true;
      }
    }
    if (!done) {
      // exact path: every point of the bucket
      for (int64_t b = lo + tid; b < hi; b += blockDim.x) {
        const double xb = pre ? sx[cur][b - lo] : J.px[b];
        const double yb = pre ? sy[cur][b - lo] : J.py[b];
        amax_merge(bk, bi, area_key(exact_area(xa, ya, dxm, dym, xb, yb), J.nan), b);
      }
    }
    block_amax(bk, bi, sh, lane, warp);
    const int64_t pick = (bk == 0ull) ? lo : bi;   // no candidate (NaN-ignore): first index
    if (tid == 0) J.out[j + 1] = out_index(J, pick);
    a = pick;
    xa = pre ? sx[cur][pick - lo] : J.px[pick];
    ya = pre ? sy[cur][pick - lo] : J.py[pick];
    lo = hi;
    hi = nhi;
  }
  if (pre) cp_async_wait_all();
  if (tid == 0) {
    J.out[B + 1] = out_index(J, m - 1);
    *J.out_count = B + 2;
  }
  (void)a;
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

static unsigned grid_for(int64_t n, int per_sm = 8) {
  int64_t blocks = (n + 255) / 256;
  const int64_t cap = (int64_t)device_sm_count() * per_sm;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (unsigned)blocks;
}

size_t lttb_job_scratch(int64_t m_max, int64_t B, int64_t K, int mode) {
  size_t s = align_up((size_t)(B + 1) * sizeof(double2), 256);
  if (mode == 0) s += align_up((size_t)B * (size_t)K * 4, 256);
  else s += align_up((size_t)m_max * sizeof(float2), 256);
  return s;
}

tsds_status launch_points_jobs(const PointsJob* jobs_dev, int count, int64_t max_m, cudaStream_t st) {
  note_launch();
  k_points<<<dim3(grid_for(max_m), (unsigned)count), 256, 0, st>>>(jobs_dev);
  TSDS_CK(cudaGetLastError());
  return TSDS_OK;
}

tsds_status run_lttb_jobs(const LttbJob* jobs_host, const LttbJob* jobs_dev, int count, int64_t max_B,
                          int64_t max_m, int64_t max_K_chain, cudaStream_t st) {
  bool any_table = false, any_chain = false;
  for (int i = 0; i < count; ++i) (jobs_host[i].mode == 0 ? any_table : any_chain) = true;
  dim3 gm(grid_for(max_B, 4), (unsigned)count);
  note_launch();
  k_means<<<gm, 256, 0, st>>>(jobs_dev);
  TSDS_CK(cudaGetLastError());
  if (any_table) {
    int64_t blocks = (max_B + 7) / 8;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    note_launch();
    k_table<<<dim3((unsigned)blocks, (unsigned)count), 256, 0, st>>>(jobs_dev);
    TSDS_CK(cudaGetLastError());
  }
  if (any_chain) {
    note_launch();
    k_p32<<<dim3(grid_for(max_m, 4), (unsigned)count), 256, 0, st>>>(jobs_dev);
    TSDS_CK(cudaGetLastError());
    const size_t smem = max_K_chain <= kPrefetchMaxK ? (size_t)max_K_chain * 48 : 0;
    if (smem > 48 * 1024) TSDS_CK(cudaFuncSetAttribute(k_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    note_launch();
    k_chain<<<(unsigned)count, kChainThreads, smem, st>>>(jobs_dev);
    TSDS_CK(cudaGetLastError());
  }
  // table-mode jobs, and every job whose points are all kept, finish here
  note_launch();
  k_chase<<<(unsigned)count, 32, 0, st>>>(jobs_dev);
  TSDS_CK(cudaGetLastError());
  return TSDS_OK;
}

// LTTB over points px/py already in binary64 (m on the device when m_dev is
// set, otherwise m_host; m_max bounds it), writing R[pick] (or pick) to out.
static tsds_status lttb_points_core(const double* px, const double* py, const int64_t* m_dev, int64_t m_host,
                                    int64_t m_max, int64_t n_out, tsds_nan_mode nan, const int64_t* R,
                                    int64_t* out, int64_t* out_count, cudaStream_t st) {
  LttbJob J;
  memset(&J, 0, sizeof J);
  J.px = px;
  J.py = py;
  J.m_dev = m_dev;
  J.m_host = m_host;
  J.B = n_out - 2;
  J.K = m_max > 2 ? (m_max - 2 + J.B - 1) / J.B : 1;
  J.nan = nan;
  J.mode = J.K <= kTableMaxK ? 0 : 1;
  J.R = R;
  J.out = out;
  J.out_count = out_count;
  Scratch s;
  const size_t js = lttb_job_scratch(m_max, J.B, J.K, J.mode);
  TSDS_CK(scratch_alloc(s, js + align_up(sizeof(LttbJob), 256), st));
  char* p = static_cast<char*>(s.p);
  J.means = reinterpret_cast<double2*>(p);
  p += align_up((size_t)(J.B + 1) * sizeof(double2), 256);
  if (J.mode == 0) J.table = reinterpret_cast<int32_t*>(p);
  else J.p32 = reinterpret_cast<float2*>(p);
  LttbJob* jd = reinterpret_cast<LttbJob*>(static_cast<char*>(s.p) + js);
  TSDS_CK(cudaMemcpyAsync(jd, &J, sizeof J, cudaMemcpyHostToDevice, st));
  return run_lttb_jobs(&J, jd, 1, J.B, m_max, J.mode == 1 ? J.K : 0, st);
}

static tsds_status points(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype, const int64_t* R,
                          const int64_t* m_dev, int64_t m_host, int64_t m_max, double* px, double* py, cudaStream_t st) {
  PointsJob P;
  P.x = x;
  P.x_dtype = x_dtype;
  P.y = y;
  P.y_dtype = y_dtype;
  P.R = R;
  P.m_dev = m_dev;
  P.m_host = m_host;
  P.px = px;
  P.py = py;
  Scratch s;
  TSDS_CK(scratch_alloc(s, sizeof(PointsJob), st));
  TSDS_CK(cudaMemcpyAsync(s.p, &P, sizeof P, cudaMemcpyHostToDevice, st));
  note_launch();
  k_points<<<dim3(grid_for(m_max), 1), 256, 0, st>>>(static_cast<const PointsJob*>(s.p));
  TSDS_CK(cudaGetLastError());
  return TSDS_OK;
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
  const size_t pb = align_up((size_t)n * 8, 256);
  TSDS_CK(scratch_alloc(s, 2 * pb, st));
  double* py = static_cast<double*>(s.p);
  double* px = reinterpret_cast<double*>(static_cast<char*>(s.p) + pb);
  tsds_status r = points(x, x_dtype, y, y_dtype, nullptr, nullptr, n, n, px, py, st);
  if (r != TSDS_OK) return r;
  return lttb_points_core(px, py, nullptr, n, n, n_out, nan, nullptr, out, out_count, st);
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
  TSDS_CK(scratch_alloc(s, 3 * rbytes + 256, st));
  char* base = static_cast<char*>(s.p);
  int64_t* R = reinterpret_cast<int64_t*>(base);
  double* py = reinterpret_cast<double*>(base + rbytes);
  double* px = reinterpret_cast<double*>(base + 2 * rbytes);
  int64_t* counts = reinterpret_cast<int64_t*>(base + 3 * rbytes);   // [k, m]
  const void* y_in = static_cast<const char*>(y) + dtype_size(y_dtype);
  const void* x_in = x ? static_cast<const char*>(x) + dtype_size(x_dtype) : nullptr;
  tsds_status r = run_binned_series(x_in, x_dtype, y_in, y_dtype, n_in, n_sel / 2, nan, ALGO_MINMAX,
                                    R + 1, counts, 1, st);
  if (r != TSDS_OK) return r;
  note_launch();
  k_close_selection<<<1, 1, 0, st>>>(R, counts, n, counts + 1);
  TSDS_CK(cudaGetLastError());
  r = points(x, x_dtype, y, y_dtype, R, counts + 1, 0, m_max, px, py, st);
  if (r != TSDS_OK) return r;
  return lttb_points_core(px, py, counts + 1, 0, m_max, n_out, nan, R, out, out_count, st);
}

}  // namespace tsds
