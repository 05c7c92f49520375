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
//    parallel (a group of lanes per bucket, several buckets per warp, exact
//    binary64 areas).
//  * Larger buckets: the pick of bucket j is the largest |linear form| of its
//    points, which a vertex of the bucket's convex hull attains, so the
//    picks that can feed bucket j+1 are few (a random walk's hull has about
//    2 ln K vertices).  Each bucket's candidates (hull vertices in FP32,
//    plus its first point and its first non-finite point) are found in
//    parallel, a table best[j][c] over the candidates c of bucket j-1 is
//    filled in parallel (one warp per entry: an FP32 estimate of every area
//    with a rigorous error bound, then exact binary64 areas for the points
//    the bound cannot rule out), and one warp chases the table.  A previous
//    pick that is not among the candidates (ties along hull edges, rounding
//    at near-ties, more than 32 hull vertices) is computed on the spot by
//    the same exact warp search, so the table only decides speed.
#include "device.cuh"
#include "internal.h"
#include "lttb.h"

namespace tsds {

typedef unsigned __int128 u128;


__device__ __forceinline__ int64_t job_m(const LttbJob& J) { return J.m_dev ? *J.m_dev : J.m_host; }

__device__ __forceinline__ int64_t bucket_start(int64_t j, int64_t m, int64_t B) {
  return 1 + (int64_t)muldiv_floor((uint64_t)j, (uint64_t)(m - 2), (uint64_t)B);
}

__device__ __forceinline__ int64_t out_index(const LttbJob& J, int64_t k) { return J.R ? J.R[k] : k + J.bias; }

// out[pos] = the series index of point k, with its values beside it.
__device__ __forceinline__ void lttb_emit(const LttbJob& J, int64_t pos, int64_t k) {
  const int64_t i = out_index(J, k);
  J.out[pos] = i;
  gather_point(J.g, pos, J.ysrc, J.xsrc, i);
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

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(smem)), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(smem)), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Large buckets whose mean needs the sequential sum (flagged by k_p32, which
// gives every other bucket its mean from exact sums, below) take it here, one
// chain per bucket and coordinate (table mode's small buckets, flagged by
// k_means, take k_sums_small).  A CTA covers 32 buckets with four warps,
// one per SM sub-partition: two producer warps stream the flagged buckets'
// x and y values through a ring of three 32-point chunks in shared memory
// (lane i copies point i of each bucket's chunk: coalesced cp.async), and two
// consumer warps add them up, thread t of the first the x values of bucket t
// and of the second its y values.  Named barriers hand each ring slot back
// and forth (one pair per slot, so no warp arrives twice on a barrier before
// the others have passed it).  The consumers then do nothing but
// shared-memory loads and one chain of binary64 additions each, and the two
// chains of a bucket run on different sub-partitions.
constexpr int kSumChunk = 32;
constexpr int kSumRing = 3;
constexpr int kSumThreads = 128;
constexpr int kBarReady = 1;               // named barriers 1..3: slot holds a chunk
constexpr int kBarFree = 1 + kSumRing;     // named barriers 4..6: slot may be refilled

// [ring slot][point of the chunk][bucket], rows padded by one so that both
// the copies (fixed bucket) and the adds (fixed point) spread over the banks.
typedef double SumSlots[kSumRing][kSumChunk][33];
struct SumRing {
  SumSlots x, y;
};

__device__ __forceinline__ void named_bar_sync(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(kSumThreads) : "memory");
}
__device__ __forceinline__ void named_bar_arrive(int id) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "n"(kSumThreads) : "memory");
}

// One chunk of one coordinate's chain: v are the values added, y decides
// (NaN-ignore) which points count.
template <bool IGN>
__device__ __forceinline__ void sums_consume(const SumSlots& v, const SumSlots& y, int slot, int t, int nn,
                                             double& s, int64_t& cnt) {
#pragma unroll
  for (int i0 = 0; i0 < kSumChunk; i0 += 8) {
    double a[8];
    bool keep[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      a[u] = v[slot][i0 + u][t];
      keep[u] = i0 + u < nn;
      if (IGN) keep[u] = keep[u] && !isnan(y[slot][i0 + u][t]);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (keep[u]) {
        s = __dadd_rn(s, a[u]);
        if (IGN) ++cnt;
      }
    }
  }
}

__global__ void __launch_bounds__(kSumThreads) k_sums_wide(const LttbJob* __restrict__ jobs, int mode) {
  const LttbJob J = jobs[blockIdx.y];
  if (J.mode != mode) return;
  const int64_t m = job_m(J), B = J.B;
  if (m <= B + 2) return;
  extern __shared__ __align__(16) unsigned char sum_smem[];
  SumRing& R = *reinterpret_cast<SumRing*>(sum_smem);
  __shared__ int64_t lo_s[32], n_s[32];
  __shared__ int64_t chunks_s;
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  const bool ign = J.nan == TSDS_NAN_IGNORE;
  for (int64_t jb = (int64_t)blockIdx.x * 32; jb < B; jb += (int64_t)gridDim.x * 32) {
    const int64_t j = jb + t;
    __syncthreads();                        // the previous group's readers of lo_s/n_s are done
    if (warp == 0) {
      const bool mine = j >= 1 && j < B && J.chain[j];
      const int64_t lo = mine ? bucket_start(j, m, B) : 0, hi = mine ? bucket_start(j + 1, m, B) : 0;
      lo_s[t] = lo;
      n_s[t] = hi - lo;
      int64_t chunks = (hi - lo + kSumChunk - 1) / kSumChunk;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) chunks = max(chunks, __shfl_xor_sync(0xffffffffu, chunks, o));
      if (t == 0) chunks_s = chunks;
    }
    __syncthreads();
    const int64_t chunks = chunks_s;
    if (chunks == 0) continue;
    if (warp >= 2) {
      // producers (x, then y): fill slot c % 3 with chunk c, signal chunk c - 1 once it landed
      const double* src = warp == 2 ? J.px : J.py;
      SumSlots& dst = warp == 2 ? R.x : R.y;
      for (int64_t c = 0; c <= chunks; ++c) {
        if (c < chunks) {
          const int slot = (int)(c % kSumRing);
          if (c >= kSumRing) named_bar_sync(kBarFree + slot);
          const int64_t k = c * kSumChunk + t;
#pragma unroll 8
          for (int b = 0; b < 32; ++b)
            if (k < n_s[b]) cp_async8(&dst[slot][t][b], src + lo_s[b] + k);
          cp_async_commit();
        }
        if (c >= 1) {
          if (c < chunks) cp_async_wait<1>();
          else cp_async_wait<0>();
          named_bar_arrive(kBarReady + (int)((c - 1) % kSumRing));
        }
      }
    } else {
      // consumers: thread t of warp 0 sums bucket jb + t's x values, of warp 1 its y values
      const int64_t n = n_s[t];
      const SumSlots& v = warp == 0 ? R.x : R.y;
      double s = 0.0;
      int64_t cnt = 0;
      for (int64_t c = 0; c < chunks; ++c) {
        const int slot = (int)(c % kSumRing);
        named_bar_sync(kBarReady + slot);
        const int nn = (int)max((int64_t)0, min((int64_t)kSumChunk, n - c * kSumChunk));
        if (ign) sums_consume<true>(v, R.y, slot, t, nn, s, cnt);
        else sums_consume<false>(v, R.y, slot, t, nn, s, cnt);
        if (c + kSumRing < chunks) named_bar_arrive(kBarFree + slot);
      }
      if (!ign) cnt = n;
      if (n > 0) reinterpret_cast<double*>(J.means)[2 * j + warp] = __ddiv_rn(s, (double)cnt);
    }
  }
}

// The same sequential sums for the small buckets of table mode (at most 32
// points): a thread per flagged bucket adds its x and its y values in index
// order, so the binary64 adds issued are the points' own (the ring above
// issues a full 32-point chunk per bucket, and this GPU's FP64 pipe is
// narrow).
__global__ void k_sums_small(const LttbJob* __restrict__ jobs) {
  const LttbJob J = jobs[blockIdx.y];
  if (J.mode != 0) return;
  const int64_t m = job_m(J), B = J.B;
  if (m <= B + 2) return;
  const bool ign = J.nan == TSDS_NAN_IGNORE;
  for (int64_t j = 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < B; j += (int64_t)gridDim.x * blockDim.x) {
    if (!J.chain[j]) continue;
    const int64_t lo = bucket_start(j, m, B), hi = bucket_start(j + 1, m, B);
    double sx = 0.0, sy = 0.0;
    int64_t cnt = 0;
    for (int64_t k = lo; k < hi; ++k) {
      const double x = J.px[k], y = J.py[k];
      if (ign && isnan(y)) continue;
      sx = __dadd_rn(sx, x);
      sy = __dadd_rn(sy, y);
      ++cnt;
    }
    if (hi > lo) J.means[j] = make_double2(__ddiv_rn(sx, (double)cnt), __ddiv_rn(sy, (double)cnt));
  }
}

// Exact bucket sums.  Each binary64 value is +-M * 2^q with M odd; a lane
// keeps its running sum as an integer multiple of 2^s, s its smallest q so
// far, and the largest binary exponent `top` it has seen.  With L the
// smallest q and T the largest exponent over a bucket's c added values, every
// partial sum of the index-order sum is a multiple of 2^L of magnitude below
// c * 2^(T+1); when that bound is at most 2^(53+L) every partial sum is a
// binary64 number, so no addition of the sequential sum rounds and it equals
// the exact sum, which the lanes' integers give in any order.  Otherwise (or
// for a NaN or an infinity) the integers may have wrapped and the bucket
// takes the sequential sum instead.
struct ExactSum {
  unsigned long long acc;   // two's complement, units of 2^s
  int s, top;
  bool nan;                 // a NaN was added: the sum is NaN in any order
};

__device__ __forceinline__ void exact_init(ExactSum& e) {
  e.acc = 0ull;
  e.s = 4096;
  e.top = -4096;
  e.nan = false;
}

__device__ __forceinline__ void exact_add(ExactSum& e, double v, bool& bad) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int eb = (int)((b >> 52) & 0x7ff);
  unsigned long long M = b & 0xfffffffffffffull;
  if (eb == 0x7ff) {
    if (M != 0ull) e.nan = true;
    else bad = true;                                     // an infinity: order may matter (overflow)
    return;
  }
  if (eb == 0 && M == 0ull) return;                      // a zero adds nothing
  int q = eb == 0 ? -1074 : eb - 1075;
  if (eb != 0) M |= 1ull << 52;
  const int tz = __ffsll((long long)M) - 1;
  M >>= tz;
  q += tz;
  e.top = max(e.top, q + 63 - __clzll((long long)M));
  if (q < e.s) {
    e.acc <<= min(e.s - q, 63);
    e.s = q;
  }
  const unsigned long long w = M << min(q - e.s, 63);
  e.acc += (b >> 63) ? (0ull - w) : w;
}

// The warp's exact sum of one coordinate (NaN when a NaN was added), or
// false when the bound fails.
__device__ __forceinline__ bool exact_finish(const ExactSum& e, int cnt, double& out) {
  if (__any_sync(0xffffffffu, e.nan)) {
    out = __longlong_as_double(0x7ff8000000000000ll);
    return true;
  }
  const int L = __reduce_min_sync(0xffffffffu, e.s + 8192) - 8192;
  const int T = __reduce_max_sync(0xffffffffu, e.top + 8192) - 8192;
  unsigned long long a = e.acc << min(e.s - L, 63);
  if (e.s == 4096) a = 0ull;                             // lane saw no nonzero value
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (T == -4096) {                                      // every value was zero
    out = 0.0;
    return true;
  }
  const int lg = cnt <= 1 ? 0 : 32 - __clz(cnt - 1);     // ceil(log2 cnt)
  if (T + 1 + lg > 53 + L) return false;
  double r = __ll2double_rn((long long)a);               // exact: |a| < 2^53
  int e2 = L;
  if (e2 < -1022) {                                      // scale in two exact steps
    r = __dmul_rn(r, __longlong_as_double((long long)(-600 + 1023) << 52));
    e2 += 600;
  }
  out = __dmul_rn(r, __longlong_as_double((long long)(e2 + 1023) << 52));
  return true;
}

// The same over each group of GS lanes (a power of two; lanes gs*GS ..
// gs*GS+GS-1 hold one bucket): every lane of the warp calls it, and each gets
// its group's result.
__device__ __forceinline__ bool exact_finish_g(const ExactSum& e, int cnt, double& out, int GS) {
  bool nan = e.nan;
  int L = e.s, T = e.top;
  for (int o = GS >> 1; o; o >>= 1) {
    nan = __shfl_xor_sync(0xffffffffu, nan, o) || nan;
    L = min(L, __shfl_xor_sync(0xffffffffu, L, o));
    T = max(T, __shfl_xor_sync(0xffffffffu, T, o));
  }
  unsigned long long a = e.acc << min(e.s - L, 63);
  if (e.s == 4096) a = 0ull;                             // lane saw no nonzero value
  for (int o = GS >> 1; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (nan) {
    out = __longlong_as_double(0x7ff8000000000000ll);
    return true;
  }
  if (T == -4096) {                                      // every value was zero
    out = 0.0;
    return true;
  }
  const int lg = cnt <= 1 ? 0 : 32 - __clz(cnt - 1);     // ceil(log2 cnt)
  if (T + 1 + lg > 53 + L) return false;
  double r = __ll2double_rn((long long)a);               // exact: |a| < 2^53
  int e2 = L;
  if (e2 < -1022) {                                      // scale in two exact steps
    r = __dmul_rn(r, __longlong_as_double((long long)(-600 + 1023) << 52));
    e2 += 600;
  }
  out = __dmul_rn(r, __longlong_as_double((long long)(e2 + 1023) << 52));
  return true;
}

// means[j] for buckets 1..B-1 (the third vertex of steps 0..B-2): binary64
// sums in index order divided once by the count.  Small buckets (table mode,
// at most 32 points): a group of lanes per bucket (32/GS buckets per warp for
// buckets of at most GS points), a lane per point, the exact integer
// sum (ExactSum) when no addition of the index-order sum can round; other
// buckets are flagged for the sequential sums of k_sums_wide.
__global__ void k_means(const LttbJob* __restrict__ jobs) {
  const LttbJob J = jobs[blockIdx.y];
  if (J.mode != 0) return;
  const int64_t m = job_m(J), B = J.B;
  if (m <= B + 2) return;
  constexpr unsigned FULL = 0xffffffffu;
  const bool ign = J.nan == TSDS_NAN_IGNORE;
  const int lane = threadIdx.x & 31;
  // buckets of at most GS points: 32/GS of them per warp, a lane per point
  int gs = 1;
  while (gs < J.K) gs <<= 1;
  const int GS = gs, per = 32 / GS, gi = lane / GS, gl = lane % GS;
  const unsigned shift = (unsigned)(gi * GS);
  const unsigned gm = GS == 32 ? FULL : ((1u << GS) - 1u);
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t j0 = 1 + ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * per; j0 < B;
       j0 += warps * per) {
    const int64_t j = j0 + gi;
    const bool jact = j < B;
    const int64_t lo = jact ? bucket_start(j, m, B) : 0, hi = jact ? bucket_start(j + 1, m, B) : 0;
    const bool has = gl < hi - lo;          // at most GS points in table mode
    const double x = has ? J.px[lo + gl] : 0.0, y = has ? J.py[lo + gl] : 0.0;
    const bool inc = has && !(ign && isnan(y));
    const int cnt = __popc((__ballot_sync(FULL, inc) >> shift) & gm);
    ExactSum ex, ey;
    exact_init(ex);
    exact_init(ey);
    bool bad = cnt == 0;
    if (inc) {
      exact_add(ex, x, bad);
      exact_add(ey, y, bad);
    }
    bad = ((__ballot_sync(FULL, bad) >> shift) & gm) != 0u;
    double sx = 0.0, sy = 0.0;
    const bool okx = exact_finish_g(ex, cnt, sx, GS);
    const bool oky = exact_finish_g(ey, cnt, sy, GS);
    const bool exact = !bad && okx && oky;
    if (jact && gl == 0) {
      J.chain[j] = exact ? 0 : 1;
      if (exact) J.means[j] = make_double2(__ddiv_rn(sx, (double)cnt), __ddiv_rn(sy, (double)cnt));
    }
  }
}

// p32[k] = point k relative to its bucket's first point, rounded to FP32: a
// warp per bucket, coalesced.  The same pass adds the bucket up exactly
// (ExactSum) and writes its mean, or flags the bucket for k_sums_wide.  When
// x is the index, k - start is an integer below 2^53: its FP32 rounding comes
// straight from the integer, and the x sum is an integer sum, exact while the
// bucket's indices add up to less than 2^53.
__global__ void k_p32(const LttbJob* __restrict__ jobs) {
  const LttbJob J = jobs[blockIdx.y];
  if (J.mode != 2) return;
  const int64_t m = job_m(J), B = J.B;
  if (m <= B + 2) return;
  const int lane = threadIdx.x & 31;
  const bool ign = J.nan == TSDS_NAN_IGNORE;
  const bool xi = J.x_index != 0;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < B; j += warps) {
    const int64_t lo = bucket_start(j, m, B), hi = bucket_start(j + 1, m, B);
    const double X0 = J.px[lo], Y0 = J.py[lo];
    ExactSum ex, ey;
    exact_init(ex);
    exact_init(ey);
    unsigned long long isum = 0;             // x sum when x is the index (wraps only when unused)
    bool bad = hi - lo > (int64_t)1 << 30;
    const bool small = hi - lo < (int64_t)1 << 31;   // offsets fit an int
    int cnt = 0;
    for (int64_t k0 = lo + lane; k0 < hi; k0 += 128) {
      double xv[4], yv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t k = k0 + 32 * u;
        xv[u] = !xi && k < hi ? J.px[k] : 0.0;
        yv[u] = k < hi ? J.py[k] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t k = k0 + 32 * u;
        if (k < hi) {
          const float fx = !xi ? __double2float_rn(__dsub_rn(xv[u], X0))
                           : small ? __int2float_rn((int)(k - lo)) : __ll2float_rn(k - lo);
          J.p32[k] = make_float2(fx, __double2float_rn(__dsub_rn(yv[u], Y0)));
          if (!(ign && isnan(yv[u]))) {
            ++cnt;
            if (xi) isum += (unsigned long long)k;
            else exact_add(ex, xv[u], bad);
            exact_add(ey, yv[u], bad);
          }
        }
      }
    }
    if (j == 0) continue;
    cnt = (int)__reduce_add_sync(0xffffffffu, (unsigned)cnt);
    bad = __any_sync(0xffffffffu, bad) || cnt == 0;
    double sx = 0.0, sy = 0.0;
    bool okx;
    if (xi) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) isum += __shfl_xor_sync(0xffffffffu, isum, o);
      // every partial sum is at most hi * cnt: below 2^53 they are all exact binary64 additions
      okx = (double)hi * (double)cnt < 9007199254740992.0;
      sx = __ll2double_rn((long long)isum);
    } else {
      okx = exact_finish(ex, cnt, sx);
    }
    const bool oky = exact_finish(ey, cnt, sy);
    const bool exact = !bad && okx && oky;
    if (lane == 0) {
      J.chain[j] = exact ? 0 : 1;
      if (exact) J.means[j] = make_double2(__ddiv_rn(sx, (double)cnt), __ddiv_rn(sy, (double)cnt));
    }
  }
}

// ---------------------------------------------------------------- table mode

// Jobs whose points are all kept return every index.
__global__ void __launch_bounds__(32) k_chase(const LttbJob* __restrict__ jobs) {
  const LttbJob J = jobs[blockIdx.x];
  const int lane = threadIdx.x & 31;
  const int64_t m = job_m(J), B = J.B;
  if (m <= B + 2) {
    for (int64_t i = lane; i < m; i += 32) lttb_emit(J, i, i);
    if (lane == 0) *J.out_count = m;
  }
}

// ---------------------------------------------------------------- hull-table mode

constexpr int kCandMax = kLttbCandMax;

// A value the FP32 filter accepts: finite, 0 or within [2^-60, 2^60] in magnitude.
__device__ __forceinline__ bool filt_ok(float v) {
  const float a = fabsf(v);
  return a == 0.0f || (a >= 8.6736174e-19f && a <= 1.1529215e18f);
}

// The FP32 filter.  For previous pick a and third vertex m, with al, be the
// FP32 roundings of xa - xm and ym - ya and (ax, ay) those of a relative to
// the bucket's first point, a point p of the bucket (relative to the same
// first point, FP32) gets est = |al (p.y - ay) - (ax - p.x) be| and the bound
// err = 8u (|al| (|p.y| + |ay| + |p.y - ay|) + |be| (|p.x| + |ax| + |ax - p.x|))
// + 4u est + 2^-120 (u = 2^-24) on est's distance from its exact binary64
// area, valid while every input passes filt_ok.  A point whose est + err is
// below a lower bound of the best exact area cannot be the pick.  Every
// operation is rounded to nearest and none is fused, so the computed
// est + err is a monotone function of p.x and p.y separately, which is what
// lets a slice's bounding box bound all of its points at once.
struct Filt {
  float al, be, ax, ay;
};

__device__ __forceinline__ float filt_err(const Filt& F, float apx, float apy, float ad1, float ad2, float est) {
  const float u8 = 4.7683716e-07f;   // 8 * 2^-24
  const float u4 = 2.3841858e-07f;   // 4 * 2^-24
  const float tiny = 7.5231638e-37f; // 2^-120
  const float sy = __fadd_rn(__fadd_rn(apy, fabsf(F.ay)), ad1);
  const float sx = __fadd_rn(__fadd_rn(apx, fabsf(F.ax)), ad2);
  const float t = __fadd_rn(__fmul_rn(fabsf(F.al), sy), __fmul_rn(fabsf(F.be), sx));
  return __fadd_rn(__fadd_rn(__fmul_rn(u8, t), __fmul_rn(u4, est)), tiny);
}

// The signed estimate al (py - ay) - (ax - px) be: non-decreasing in py when
// al >= 0 (non-increasing otherwise) and in px when be >= 0.
__device__ __forceinline__ float filt_signed(const Filt& F, float px, float py) {
  return __fsub_rn(__fmul_rn(F.al, __fsub_rn(py, F.ay)), __fmul_rn(__fsub_rn(F.ax, px), F.be));
}

// est + err of one point.
__device__ __forceinline__ float filt_point(const Filt& F, float2 p) {
  const float est = fabsf(filt_signed(F, p.x, p.y));
  return __fadd_rn(est, filt_err(F, fabsf(p.x), fabsf(p.y), fabsf(__fsub_rn(p.y, F.ay)),
                                 fabsf(__fsub_rn(F.ax, p.x)), est));
}

// An upper bound of filt_point over every point of the box (x0, x1, y0, y1):
// the signed estimate takes its extremes at two opposite corners, and each
// term of err its largest value at an edge of the box.
__device__ __forceinline__ float filt_box(const Filt& F, float4 bx) {
  const float yh = F.al >= 0.0f ? bx.w : bx.z, yl = F.al >= 0.0f ? bx.z : bx.w;
  const float xh = F.be >= 0.0f ? bx.y : bx.x, xl = F.be >= 0.0f ? bx.x : bx.y;
  const float est = fmaxf(fabsf(filt_signed(F, xh, yh)), fabsf(filt_signed(F, xl, yl)));
  const float ad1 = fmaxf(fabsf(__fsub_rn(bx.z, F.ay)), fabsf(__fsub_rn(bx.w, F.ay)));
  const float ad2 = fmaxf(fabsf(__fsub_rn(F.ax, bx.x)), fabsf(__fsub_rn(F.ax, bx.y)));
  const float apx = fmaxf(fabsf(bx.x), fabsf(bx.y)), apy = fmaxf(fabsf(bx.z), fabsf(bx.w));
  return __fadd_rn(est, filt_err(F, apx, apy, ad1, ad2, est));
}

// table[j*K + ai] = (pick in bucket j) - start(j) when the previous pick is
// point start(j-1) + ai (for j = 0 the previous pick is point 0, slot 0).
// One warp per bucket; lanes are the candidates b.  The FP32 filter (filt_err above) decides most
// steps without binary64 arithmetic: when exactly one candidate's upper bound
// reaches the best lower bound, that candidate is the pick.  Otherwise (a tie
// or near-tie, or a value the filter cannot take) every candidate gets its
// exact binary64 area.  The binary64 work left is per bucket, not per step:
// the FP32 copies of the bucket's points (lanes = b) and of the previous
// bucket's points and their differences from the third vertex (lanes = a).
__global__ void k_table(const LttbJob* __restrict__ jobs) {
  const LttbJob J = jobs[blockIdx.y];
  if (J.mode != 0) return;
  const int64_t m = job_m(J), B = J.B;
  if (m <= B + 2) return;
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  // buckets of at most GS points: 32/GS of them per warp, GS lanes each, so
  // the per-bucket binary64 work of several buckets shares one warp instruction
  int gs = 1;
  while (gs < J.K) gs <<= 1;
  const int GS = gs, per = 32 / GS, gi = lane / GS, gl = lane % GS;
  const unsigned shift = (unsigned)(gi * GS);
  const unsigned gm = GS == 32 ? FULL : ((1u << GS) - 1u);
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t j0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * per; j0 < B;
       j0 += warps * per) {
    const int64_t j = j0 + gi;
    const bool jact = j < B;
    int64_t lo = 0, hi = 0;
    double xm = 0.0, ym = 0.0, X0 = 0.0, Y0 = 0.0;
    if (jact) {
      lo = bucket_start(j, m, B);
      hi = bucket_start(j + 1, m, B);
      if (j == B - 1) { xm = J.px[m - 1]; ym = J.py[m - 1]; }
      else { const double2 c = J.means[j + 1]; xm = c.x; ym = c.y; }
      X0 = J.px[lo];
      Y0 = J.py[lo];
    }
    const int64_t b = lo + gl;
    const bool has_b = jact && b < hi;
    const double xb = has_b ? J.px[b] : 0.0, yb = has_b ? J.py[b] : 0.0;
    const float2 pb = make_float2(__double2float_rn(__dsub_rn(xb, X0)), __double2float_rn(__dsub_rn(yb, Y0)));
    // NaN candidates have NaN areas; the others must suit the filter
    const bool nanb = has_b && (isnan(xb) || isnan(yb));
    const bool candb = has_b && !nanb;
    const bool pts_ok = ((__ballot_sync(FULL, candb && !(filt_ok(pb.x) && filt_ok(pb.y))) >> shift) & gm) == 0u;
    const unsigned nan_mask = (__ballot_sync(FULL, nanb) >> shift) & gm;
    const unsigned cand_mask = (__ballot_sync(FULL, candb) >> shift) & gm;
    const bool prop = J.nan == TSDS_NAN_PROPAGATE;
    int64_t alo = 0, ahi = 0;
    if (jact) {
      if (j == 0) { alo = 0; ahi = 1; }
      else { alo = bucket_start(j - 1, m, B); ahi = lo; }
    }
    // lane gl of the group: the previous pick a = alo + gl
    const bool has_a = alo + gl < ahi;
    const double xa_l = has_a ? J.px[alo + gl] : 0.0, ya_l = has_a ? J.py[alo + gl] : 0.0;
    const double dxm_l = __dsub_rn(xa_l, xm), dym_l = __dsub_rn(ym, ya_l);
    const float al_l = __double2float_rn(dxm_l), be_l = __double2float_rn(dym_l);
    const float ax_l = __double2float_rn(__dsub_rn(xa_l, X0)), ay_l = __double2float_rn(__dsub_rn(ya_l, Y0));
    const bool fast_l = pts_ok && filt_ok(al_l) && filt_ok(be_l) && filt_ok(ax_l) && filt_ok(ay_l) &&
                        isfinite(dxm_l) && isfinite(dym_l);
    // a NaN difference from the third vertex makes every area NaN: the first
    // candidate (NaN-propagate: first NaN; NaN-ignore: no winner, first index)
    const bool anan_l = isnan(dxm_l) || isnan(dym_l);
    const int ka = (int)(ahi - alo);
    int kw = ka;   // the warp's largest previous bucket
#pragma unroll
    for (int o = 16; o; o >>= 1) kw = max(kw, __shfl_xor_sync(FULL, kw, o));
    for (int ai = 0; ai < kw; ++ai) {
      // every shuffle and ballot below runs on the whole warp; each group uses its own lanes
      const int src = (int)shift + ai;
      const bool step = ai < ka;
      const bool anan = __shfl_sync(FULL, anan_l, src);
      const bool fast = __shfl_sync(FULL, fast_l, src);
      const Filt F{__shfl_sync(FULL, al_l, src), __shfl_sync(FULL, be_l, src), __shfl_sync(FULL, ax_l, src),
                   __shfl_sync(FULL, ay_l, src)};
      float lowb = -INFINITY, upb = -INFINITY;
      if (candb && fast) {
        const float est = fabsf(filt_signed(F, pb.x, pb.y));
        const float err = filt_err(F, fabsf(pb.x), fabsf(pb.y), fabsf(__fsub_rn(pb.y, F.ay)),
                                   fabsf(__fsub_rn(F.ax, pb.x)), est);
        lowb = __fsub_rd(est, err);
        upb = __fadd_rn(est, err);
      }
      float L = lowb;
      for (int o = GS >> 1; o; o >>= 1) L = fmaxf(L, __shfl_xor_sync(FULL, L, o));
      const unsigned pass = (__ballot_sync(FULL, candb && upb >= L) >> shift) & gm;
      int32_t pick = -1;
      if (anan) pick = 0;
      else if (fast && prop && nan_mask) pick = __ffs(nan_mask) - 1;   // every other area is finite: first NaN wins
      else if (fast && !cand_mask) pick = 0;                           // NaN-ignore, only NaN candidates: no winner
      else if (fast && __popc(pass) == 1) pick = __ffs(pass) - 1;
      const bool need = step && pick < 0;
      if (__any_sync(FULL, need)) {
        const double xa = __shfl_sync(FULL, xa_l, src), ya = __shfl_sync(FULL, ya_l, src);
        const double dxm = __shfl_sync(FULL, dxm_l, src), dym = __shfl_sync(FULL, dym_l, src);
        uint64_t k = 0ull;
        int64_t idx = kIdxNone;
        if (need && has_b) { k = area_key(exact_area(xa, ya, dxm, dym, xb, yb), J.nan); idx = b; }
        for (int o = GS >> 1; o; o >>= 1) {
          const uint64_t k2 = __shfl_xor_sync(FULL, k, o);
          const int64_t i2 = __shfl_xor_sync(FULL, idx, o);
          amax_merge(k, idx, k2, i2);
        }
        if (need) pick = (int32_t)((k == 0ull ? lo : idx) - lo);
      }
      if (step && gl == 0) J.table[j * J.K + ai] = pick;
    }
  }
}

// The exact pick of bucket j = [lo, hi) after previous pick a, by one warp.
// Every point first gets an FP32 estimate of its area and a rigorous bound
// on the estimate's error (relative to the bucket's first point, where the
// FP32 copies are exact enough); only points whose upper bound reaches the
// best lower bound get the exact binary64 area.  Values outside the range
// where the bound holds send the step to exact areas for every point.
__device__ __noinline__ int64_t warp_pick(const LttbJob& J, int64_t j, int64_t lo, int64_t hi, int64_t a, int64_t m, int64_t B,
                             int lane) {
  double xm, ym;
  if (j == B - 1) { xm = J.px[m - 1]; ym = J.py[m - 1]; }
  else { const double2 c = J.means[j + 1]; xm = c.x; ym = c.y; }
  const double xa = J.px[a], ya = J.py[a];
  const double dxm = __dsub_rn(xa, xm), dym = __dsub_rn(ym, ya);
  const double X0 = J.px[lo], Y0 = J.py[lo];
  const float al = __double2float_rn(dxm), be = __double2float_rn(dym);
  const float ax = __double2float_rn(__dsub_rn(xa, X0)), ay = __double2float_rn(__dsub_rn(ya, Y0));
  const bool fast = filt_ok(al) && filt_ok(be) && filt_ok(ax) && filt_ok(ay) && !isnan(dxm) && !isnan(dym) &&
                    !isinf(dxm) && !isinf(dym);
  const Filt F{al, be, ax, ay};
  uint64_t bk = 0ull;
  int64_t bi = kIdxNone;
  bool done = false;
  if (fast) {
    // a lower bound of the best area: the largest est - err (rounded down)
    float lmax = -INFINITY;
    bool bad = false;
    for (int64_t b = lo + lane; b < hi; b += 32) {
      const float2 p = J.p32[b];
      if (!(filt_ok(p.x) && filt_ok(p.y))) { bad = true; continue; }
      const float est = fabsf(filt_signed(F, p.x, p.y));
      const float err = filt_err(F, fabsf(p.x), fabsf(p.y), fabsf(__fsub_rn(p.y, F.ay)), fabsf(__fsub_rn(F.ax, p.x)),
                                 est);
      lmax = fmaxf(lmax, __fsub_rd(est, err));
    }
    if (!__any_sync(0xffffffffu, bad)) {
#pragma unroll
      for (int o = 16; o; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
      for (int64_t b = lo + lane; b < hi; b += 32)
        if (filt_point(F, J.p32[b]) >= lmax)
          amax_merge(bk, bi, area_key(exact_area(xa, ya, dxm, dym, J.px[b], J.py[b]), J.nan), b);
      done = true;
    }
  }
  if (!done)
    for (int64_t b = lo + lane; b < hi; b += 32)
      amax_merge(bk, bi, area_key(exact_area(xa, ya, dxm, dym, J.px[b], J.py[b]), J.nan), b);
  amax_warp(bk, bi);
  return bk == 0ull ? lo : bi;   // no candidate (NaN-ignore): first index
}

// Candidates of every bucket, one warp per bucket: each lane builds the upper
// and lower hulls of its slice of the bucket (Andrew's monotone chain over the
// FP32 points, x ascending, after the Akl-Toussaint test against the
// bucket's extreme points has set aside the points that cannot be vertices),
// then pairs of neighbouring slice hulls are merged
// in five rounds (lane 2i takes lane 2i+1's lists, lane 4i lane 4i+2's, ...),
// all stacks in shared memory.  Lane 0 writes candidate row j+1 (the row the
// step after bucket j reads): the first point, the first non-finite point,
// then hull vertices, at most kCandMax, -1 after.  A stack that would
// overflow replaces its top, so an unusually long hull only yields fewer
// useful candidates (the chase then computes those steps directly).  The
// candidates only steer the work: the tables scan every point a candidate's
// bound cannot exclude, so FP32 hulls that miss a vertex cost time, not
// correctness.
constexpr int kHullWarps = 4;
constexpr int kSliceStack = 24;    // per lane and hull

// Per warp: entry i of lane l's stacks at [i][l] (distinct banks across lanes).
struct HullWarp {
  float2 p[2][kSliceStack][32];
  int32_t r[2][kSliceStack][32];
  int n[2][32];
};

__device__ __forceinline__ float cross3(float2 o, float2 a, float2 b) {
  return (a.x - o.x) * (b.y - o.y) - (a.y - o.y) * (b.x - o.x);
}

// Pushes (p, r) onto column `col` of stack h (upper: pops on left or straight
// turns, lower: on right or straight turns).  t1 and t2 mirror the stack's
// top two points in registers, so a push that pops nothing reads no shared
// memory.
__device__ __forceinline__ void hull_push(HullWarp& H, int h, int col, int& n, float2& t1, float2& t2, float2 p,
                                          int32_t r) {
  while (n >= 2) {
    const float c = cross3(t2, t1, p);
    if (h == 0 ? c >= 0.0f : c <= 0.0f) {
      --n;
      t1 = t2;
      if (n >= 2) t2 = H.p[h][n - 2][col];
    } else {
      break;
    }
  }
  if (n == kSliceStack) {      // full: the new point replaces the top
    H.p[h][n - 1][col] = p;
    H.r[h][n - 1][col] = r;
    t1 = p;
    return;
  }
  H.p[h][n][col] = p;
  H.r[h][n][col] = r;
  t2 = t1;
  t1 = p;
  ++n;
}

__global__ void __launch_bounds__(kHullWarps * 32) k_hull(const LttbJob* __restrict__ jobs) {
  const LttbJob J = jobs[blockIdx.y];
  if (J.mode != 2) return;
  const int64_t m = job_m(J), B = J.B;
  if (m <= B + 2) return;
  extern __shared__ __align__(16) unsigned char hull_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  HullWarp& H = reinterpret_cast<HullWarp*>(hull_smem)[wib];
  for (int64_t j = (int64_t)blockIdx.x * kHullWarps + wib; j < B; j += (int64_t)gridDim.x * kHullWarps) {
    const int64_t lo = bucket_start(j, m, B), hi = bucket_start(j + 1, m, B);
    const int64_t c = (hi - lo + 31) / 32;
    const int64_t s0 = lo + lane * c, s1 = min(s0 + c, hi);
    // Akl-Toussaint: with F, L the bucket's first and last finite points and T, D
    // its highest and lowest, a point strictly below the polyline F-T-L is no
    // vertex of the upper hull, one strictly above F-D-L none of the lower hull
    int64_t kf = INT64_MAX, kl = -1, kt = INT64_MAX, kd = INT64_MAX;
    float ty = -INFINITY, dy = INFINITY;
    for (int64_t k0 = lo + lane; k0 < hi; k0 += 128) {
      float2 pv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) pv[u] = k0 + 32 * u < hi ? J.p32[k0 + 32 * u] : make_float2(NAN, NAN);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t k = k0 + 32 * u;
        const float2 p = pv[u];
        if (!(isfinite(p.x) && isfinite(p.y))) continue;
        kf = min(kf, k);
        kl = max(kl, k);
        if (p.y > ty || (p.y == ty && k < kt)) { ty = p.y; kt = k; }
        if (p.y < dy || (p.y == dy && k < kd)) { dy = p.y; kd = k; }
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      kf = min(kf, (int64_t)__shfl_xor_sync(0xffffffffu, kf, o));
      kl = max(kl, (int64_t)__shfl_xor_sync(0xffffffffu, kl, o));
      const float ty2 = __shfl_xor_sync(0xffffffffu, ty, o), dy2 = __shfl_xor_sync(0xffffffffu, dy, o);
      const int64_t kt2 = __shfl_xor_sync(0xffffffffu, kt, o), kd2 = __shfl_xor_sync(0xffffffffu, kd, o);
      if (ty2 > ty || (ty2 == ty && kt2 < kt)) { ty = ty2; kt = kt2; }
      if (dy2 < dy || (dy2 == dy && kd2 < kd)) { dy = dy2; kd = kd2; }
    }
    const bool some = kl >= 0;
    const float2 pF = some ? J.p32[kf] : make_float2(0.f, 0.f), pL = some ? J.p32[kl] : pF;
    const float2 pT = some ? J.p32[kt] : pF, pD = some ? J.p32[kd] : pF;
    int n0 = 0, n1 = 0;
    float2 u1 = make_float2(0.f, 0.f), u2 = u1, l1 = u1, l2 = u1;   // tops of the two stacks
    int64_t bad = INT64_MAX;
    float4 box = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);   // empty: x0 > x1
    bool box_ok = true;
    for (int64_t b0 = s0; b0 < s1; b0 += 8) {
      float2 pv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) pv[u] = b0 + u < s1 ? J.p32[b0 + u] : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t b = b0 + u;
        if (b >= s1) break;
        const float2 p = pv[u];
        if (!(isfinite(p.x) && isfinite(p.y))) { bad = min(bad, b); box_ok = false; continue; }
        box_ok = box_ok && filt_ok(p.x) && filt_ok(p.y);
        box.x = fminf(box.x, p.x);
        box.y = fmaxf(box.y, p.x);
        box.z = fminf(box.z, p.y);
        box.w = fmaxf(box.w, p.y);
        const int32_t r = (int32_t)(b - lo);
        const float cu = p.x <= pT.x ? cross3(pF, pT, p) : cross3(pT, pL, p);
        const float cl = p.x <= pD.x ? cross3(pF, pD, p) : cross3(pD, pL, p);
        if (!(cu < 0.0f)) hull_push(H, 0, lane, n0, u1, u2, p, r);
        if (!(cl > 0.0f)) hull_push(H, 1, lane, n1, l1, l2, p, r);
      }
    }
    // the slice's box for k_htable; NaN marks a slice with a value the FP32 filter cannot take
    J.box[j * 32 + lane] = box_ok ? box : make_float4(NAN, NAN, NAN, NAN);
#pragma unroll
    for (int o = 16; o; o >>= 1) bad = min(bad, (int64_t)__shfl_xor_sync(0xffffffffu, bad, o));
    H.n[0][lane] = n0;
    H.n[1][lane] = n1;
    for (int d = 1; d < 32; d <<= 1) {
      __syncwarp();
      if ((lane & (2 * d - 1)) == 0) {
        const int src = lane + d;
        for (int h = 0; h < 2; ++h) {
          int n = H.n[h][lane];
          float2 t1 = make_float2(0.f, 0.f), t2 = t1;
          if (n >= 1) t1 = H.p[h][n - 1][lane];
          if (n >= 2) t2 = H.p[h][n - 2][lane];
          const int ns = H.n[h][src];
          for (int i = 0; i < ns; ++i) hull_push(H, h, lane, n, t1, t2, H.p[h][i][src], H.r[h][i][src]);
          H.n[h][lane] = n;
        }
      }
    }
    __syncwarp();
    if (j + 1 <= B) {
      // the list 0, [first non-finite point], upper hull, lower hull (lane 0's
      // merged stacks); its first occurrences, at most kCandMax, in order
      static_assert(kCandMax == 32 && 2 + 2 * kSliceStack <= 64, "one row per warp, two entries per lane");
      const int nu = H.n[0][0], nl = H.n[1][0];
      const int hb = bad < hi ? 1 : 0;
      const int total = 1 + hb + nu + nl;
      auto entry = [&](int e) -> int32_t {
        if (e == 0) return 0;
        if (hb && e == 1) return (int32_t)(bad - lo);
        e -= 1 + hb;
        return e < nu ? H.r[0][e][0] : H.r[1][e - nu][0];
      };
      int32_t v[2];
      bool keep[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int e = lane + 32 * q;
        keep[q] = e < total;
        v[q] = keep[q] ? entry(e) : -1;
        for (int f = 0; keep[q] && f < e; ++f)
          if (entry(f) == v[q]) keep[q] = false;
      }
      const unsigned k0 = __ballot_sync(0xffffffffu, keep[0]), k1 = __ballot_sync(0xffffffffu, keep[1]);
      const unsigned below = (1u << lane) - 1u;
      const int p0 = __popc(k0 & below), p1 = __popc(k0) + __popc(k1 & below);
      int32_t* row = J.cand + (j + 1) * kCandMax;
      if (keep[0] && p0 < kCandMax) row[p0] = v[0];
      if (keep[1] && p1 < kCandMax) row[p1] = v[1];
      if (lane >= __popc(k0) + __popc(k1)) row[lane] = -1;
    }
    __syncwarp();
  }
}

// table[j*kCandMax + s] = (pick of bucket j) - start(j) when the previous pick
// is candidate s of bucket j-1 (row j of cand; for j = 0: point 0, slot 0).
// One CTA per bucket: the bucket's FP32 points are staged in shared memory
// once, and each warp takes candidates in turn.  For a candidate, the exact
// areas of bucket j's own hull candidates (row j+1) give a lower bound L of
// the best area; one pass of FP32 estimates with rigorous error bounds then
// keeps only the points whose upper bound reaches L, whose exact binary64
// areas decide the pick.  Values outside the range where the bound holds,
// and non-finite areas, take the exact path over every point.
constexpr int kTableWarps = 4;
constexpr int kStageMax = 6144;    // points of a bucket staged in shared memory (48 KB)

__global__ void __launch_bounds__(kTableWarps * 32) k_htable(const LttbJob* __restrict__ jobs) {
  const LttbJob J = jobs[blockIdx.y];
  if (J.mode != 2) return;
  const int64_t m = job_m(J), B = J.B;
  if (m <= B + 2) return;
  extern __shared__ __align__(16) float2 stage[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  for (int64_t j = blockIdx.x; j < B; j += gridDim.x) {
    const int64_t lo = bucket_start(j, m, B), hi = bucket_start(j + 1, m, B);
    const int64_t K = hi - lo;
    const bool staged = K <= kStageMax;
    __syncthreads();   // the previous bucket's readers are done with the stage
    if (staged)
      for (int64_t i = threadIdx.x; i < K; i += blockDim.x) stage[i] = J.p32[lo + i];
    __syncthreads();
    // lane l's slice of the bucket (the slices k_hull used) and its box
    const int64_t cs = (K + 31) / 32;
    const float4 mybox = J.box[j * 32 + lane];
    const bool any_bad = __any_sync(0xffffffffu, isnan(mybox.x));
    double xm, ym;
    if (j == B - 1) { xm = J.px[m - 1]; ym = J.py[m - 1]; }
    else { const double2 cm = J.means[j + 1]; xm = cm.x; ym = cm.y; }
    const double X0 = J.px[lo], Y0 = J.py[lo];
    const int32_t own = J.cand[(j + 1) * kCandMax + lane];   // this bucket's hull candidates
    const int64_t alo = j == 0 ? 0 : bucket_start(j - 1, m, B);
    for (int s = wib; s < kCandMax; s += kTableWarps) {
      int32_t r;
      if (j == 0) r = s == 0 ? 0 : -1;
      else r = J.cand[j * kCandMax + s];
      if (r < 0) {   // uniform per warp
        if (lane == 0) J.fslot[j * kCandMax + s] = -1;
        continue;
      }
      const int64_t a = alo + r;
      const double xa = J.px[a], ya = J.py[a];
      const double dxm = __dsub_rn(xa, xm), dym = __dsub_rn(ym, ya);
      uint64_t bk = 0ull;
      int64_t bi = kIdxNone;
      const float al = __double2float_rn(dxm), be = __double2float_rn(dym);
      const float ax = __double2float_rn(__dsub_rn(xa, X0)), ay = __double2float_rn(__dsub_rn(ya, Y0));
      const bool fast = !any_bad && filt_ok(al) && filt_ok(be) && filt_ok(ax) && filt_ok(ay) && !isnan(dxm) &&
                        !isnan(dym) && !isinf(dxm) && !isinf(dym);
      bool done = false;
      if (fast) {
        // lower bound: the exact area of the bucket's own candidate with the
        // largest FP32 estimate
        const Filt F{al, be, ax, ay};
        float e = -1.0f;
        if (own >= 0) {
          const float2 p = staged ? stage[own] : J.p32[lo + own];
          e = fabsf(filt_signed(F, p.x, p.y));
        }
        float emax = e;
#pragma unroll
        for (int o = 16; o; o >>= 1) emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        const unsigned who = __ballot_sync(0xffffffffu, own >= 0 && e == emax);
        const int32_t r_best = __shfl_sync(0xffffffffu, own, who ? __ffs(who) - 1 : 0);
        double best = -1.0;
        if (who) {
          const double ar = exact_area(xa, ya, dxm, dym, J.px[lo + r_best], J.py[lo + r_best]);
          if (isfinite(ar)) best = ar;
        }
        if (best >= 0.0) {
          // slices whose box can reach L, then their points that can
          const float L = __double2float_rd(best);
          unsigned live = __ballot_sync(0xffffffffu, mybox.x <= mybox.y && filt_box(F, mybox) >= L);
          while (live) {
            const int l = __ffs(live) - 1;
            live &= live - 1;
            const int64_t r1 = min((int64_t)(l + 1) * cs, K);
            for (int64_t i = (int64_t)l * cs + lane; i < r1; i += 32) {
              const float2 p = staged ? stage[i] : J.p32[lo + i];
              if (filt_point(F, p) >= L)
                amax_merge(bk, bi, area_key(exact_area(xa, ya, dxm, dym, J.px[lo + i], J.py[lo + i]), J.nan),
                           lo + i);
            }
          }
          done = true;
        }
      }
      if (!done) {
        bk = 0ull;
        bi = kIdxNone;
        for (int64_t b = lo + lane; b < hi; b += 32)
          amax_merge(bk, bi, area_key(exact_area(xa, ya, dxm, dym, J.px[b], J.py[b]), J.nan), b);
      }
      amax_warp(bk, bi);
      const int32_t rel = (int32_t)((bk == 0ull ? lo : bi) - lo);
      // its slot among the next step's inputs (this bucket's candidates, row j+1)
      const unsigned hit = __ballot_sync(0xffffffffu, own == rel);
      if (lane == 0) {
        J.table[j * kCandMax + s] = rel;
        J.fslot[j * kCandMax + s] = hit ? __ffs(hit) - 1 : -1;
      }
    }
  }
}

// ---------------------------------------------------------------- the chain
//
// With the tables in place the chain is a composition of small functions:
// step j maps the slot of the previous pick (its place among step j's
// inputs: the points of bucket j-1 in table mode, its candidates in
// hull-table mode) to the slot of its own pick among step j+1's inputs
// (fslot), and emits the pick (table).  Functions compose associatively, so
// the B steps are cut into segments of 32: one warp per segment follows all
// 32 possible input slots through its segment at once (k_compose), one warp
// then chains the segments, 32 steps per lookup (k_chain_seg), and one warp
// per segment replays its segment from the known input to write the picks
// (k_replay).  A path that leaves the tables (a previous pick that is not a
// candidate) marks its segment, and k_chain_seg walks such a segment step by
// step with the exact warp search.
constexpr int kSeg = 32;
constexpr int kSegWarpsC = 8;
constexpr int kBlk = 32;          // segments per block of the chain's shared-memory ring
constexpr int kChaseRing = 4;     // blocks in the ring (three in flight)

__device__ __forceinline__ int job_width(const LttbJob& J) { return J.mode == 0 ? (int)J.K : kCandMax; }

__global__ void __launch_bounds__(kSegWarpsC * 32) k_compose(const LttbJob* __restrict__ jobs) {
  const LttbJob J = jobs[blockIdx.y];
  const int64_t m = job_m(J), B = J.B;
  if (m <= B + 2) return;
  __shared__ int32_t rows[kSegWarpsC][kSeg][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int W = job_width(J);
  const int64_t nseg = (B + kSeg - 1) / kSeg;
  for (int64_t seg = (int64_t)blockIdx.x * kSegWarpsC + w; seg < nseg; seg += (int64_t)gridDim.x * kSegWarpsC) {
    const int64_t j0 = seg * kSeg;
    const int len = (int)min((int64_t)kSeg, B - j0);
    // the segment's rows, eight loads in flight per lane
    for (int t0 = 0; t0 < len; t0 += 8) {
      int32_t v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = (t0 + u < len && lane < W) ? J.fslot[(j0 + t0 + u) * W + lane] : -1;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (t0 + u < len) rows[w][t0 + u][lane] = v[u];
    }
    __syncwarp();
    int32_t cur = lane;
    for (int t = 0; t < len; ++t) {
      if (j0 + t == B - 1) break;   // the last step's slot feeds nothing
      cur = (cur >= 0 && cur < W) ? rows[w][t][cur] : -1;
    }
    J.comp[seg * kSeg + lane] = cur;
    __syncwarp();
  }
}

// The slot of point `rel` of bucket j among step j+1's inputs (-1: none).
__device__ __forceinline__ int32_t next_slot(const LttbJob& J, int64_t j, int32_t rel, int lane) {
  if (J.mode == 0) return rel;
  const unsigned hit = __ballot_sync(0xffffffffu, J.cand[(j + 1) * kCandMax + lane] == rel);
  return hit ? __ffs(hit) - 1 : -1;
}

// Walks segment `seg` step by step from input slot s (or, for s < 0, from
// the previous pick a), writing its picks; leaves s and a at the segment's end.
__device__ __noinline__ void walk_segment(const LttbJob& J, int64_t seg, int64_t m, int64_t B, int W, int lane,
                                          int32_t& s, int64_t& a) {
  const int64_t j0 = seg * kSeg, j1 = min(j0 + kSeg, B);
  int64_t lo = bucket_start(j0, m, B);
  for (int64_t j = j0; j < j1; ++j) {
    const int64_t hi = bucket_start(j + 1, m, B);
    int32_t rel;
    if (s >= 0) rel = J.table[j * W + s];
    else rel = (int32_t)(warp_pick(J, j, lo, hi, a, m, B, lane) - lo);
    if (lane == 0) lttb_emit(J, j + 1, lo + rel);
    a = lo + rel;
    s = j + 1 < B ? next_slot(J, j, rel, lane) : 0;
    lo = hi;
  }
}

__global__ void __launch_bounds__(32) k_chain_seg(const LttbJob* __restrict__ jobs) {
  const LttbJob J = jobs[blockIdx.x];
  const int lane = threadIdx.x & 31;
  const int64_t m = job_m(J), B = J.B;
  if (m <= B + 2) return;
  __shared__ __align__(16) int32_t ring[kChaseRing][kBlk * kSeg];
  const int W = job_width(J);
  const int64_t nseg = (B + kSeg - 1) / kSeg;
  const int64_t nblk = (nseg + kBlk - 1) / kBlk;
  auto issue = [&](int64_t b) {
    if (b < nblk) {
      const int64_t n16 = min((int64_t)kBlk, nseg - b * kBlk) * kSeg / 4;
      for (int64_t i = lane; i < n16; i += 32)
        cp_async16(&ring[b % kChaseRing][4 * i], J.comp + b * kBlk * kSeg + 4 * i);
    }
    cp_async_commit();
  };
  for (int b = 0; b < kChaseRing - 1; ++b) issue(b);
  if (lane == 0) lttb_emit(J, 0, 0);
  int32_t s = 0;        // input slot of the current segment (-1: the previous pick is not a table input)
  int64_t a = 0;        // the previous pick, when s < 0
  for (int64_t b = 0; b < nblk; ++b) {
    issue(b + kChaseRing - 1);
    cp_async_wait<kChaseRing - 1>();
    __syncwarp();
    const int n = (int)min((int64_t)kBlk, nseg - b * kBlk);
    const int32_t* blk = ring[b % kChaseRing];
    for (int t = 0; t < n; ++t) {
      const int64_t seg = b * kBlk + t;
      const int32_t nxt = s >= 0 ? blk[t * kSeg + s] : -1;
      if (lane == 0) J.seg_start[seg] = nxt >= 0 ? s : -1;
      if (nxt >= 0) s = nxt;
      else walk_segment(J, seg, m, B, W, lane, s, a);   // the path leaves the tables in this segment
    }
    __syncwarp();
  }
  if (lane == 0) {
    lttb_emit(J, B + 1, m - 1);
    *J.out_count = B + 2;
  }
}

__global__ void __launch_bounds__(kSegWarpsC * 32) k_replay(const LttbJob* __restrict__ jobs) {
  const LttbJob J = jobs[blockIdx.y];
  const int64_t m = job_m(J), B = J.B;
  if (m <= B + 2) return;
  __shared__ int32_t pr[kSegWarpsC][kSeg][32], fr[kSegWarpsC][kSeg][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int W = job_width(J);
  const int64_t nseg = (B + kSeg - 1) / kSeg;
  for (int64_t seg = (int64_t)blockIdx.x * kSegWarpsC + w; seg < nseg; seg += (int64_t)gridDim.x * kSegWarpsC) {
    int32_t s = J.seg_start[seg];
    if (s < 0) continue;   // written by k_chain_seg
    const int64_t j0 = seg * kSeg;
    const int len = (int)min((int64_t)kSeg, B - j0);
    for (int t0 = 0; t0 < len; t0 += 8) {
      int32_t pv[8], fv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const bool ok = t0 + u < len && lane < W;
        pv[u] = ok ? J.table[(j0 + t0 + u) * W + lane] : 0;
        fv[u] = ok ? J.fslot[(j0 + t0 + u) * W + lane] : 0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (t0 + u < len) {
          pr[w][t0 + u][lane] = pv[u];
          fr[w][t0 + u][lane] = fv[u];
        }
      }
    }
    __syncwarp();
    int32_t mine = 0;
    for (int t = 0; t < len; ++t) {
      const int32_t rel = pr[w][t][s];
      if (lane == t) mine = rel;
      s = fr[w][t][s];
      s = (s >= 0 && s < W) ? s : 0;   // only the last step's slot can be outside the table
    }
    if (lane < len) lttb_emit(J, j0 + lane + 1, bucket_start(j0 + lane, m, B) + mine);
    __syncwarp();
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

static unsigned grid_for(int64_t n, int per_sm = 8) {
  int64_t blocks = (n + 255) / 256;
  const int64_t cap = (int64_t)device_sm_count() * per_sm;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (unsigned)blocks;
}

size_t lttb_job_scratch(int64_t m_max, int64_t B, int64_t K) {
  const int64_t nseg = (B + kSeg - 1) / kSeg;
  size_t s = align_up((size_t)(B + 1) * sizeof(double2), 256);
  s += align_up((size_t)nseg * kSeg * 4, 256) + align_up((size_t)nseg * 4, 256);   // comp, seg_start
  if (lttb_mode(K) == 0) {
    s += align_up((size_t)B * (size_t)K * 4, 256);
    s += align_up((size_t)B, 256);                                // chain flags
  } else {
    s += align_up((size_t)m_max * sizeof(float2), 256);           // p32
    s += align_up((size_t)(B + 1) * kCandMax * 4, 256);           // candidate rows 0..B
    s += 2 * align_up((size_t)B * kCandMax * 4, 256);             // table, fslot
    s += align_up((size_t)B, 256);                                // chain flags
    s += align_up((size_t)B * 32 * sizeof(float4), 256);          // slice boxes
  }
  return s;
}

void lttb_job_bind(LttbJob& J, char* p, int64_t m_max) {
  J.mode = lttb_mode(J.K);
  const int64_t nseg = (J.B + kSeg - 1) / kSeg;
  J.means = reinterpret_cast<double2*>(p);
  p += align_up((size_t)(J.B + 1) * sizeof(double2), 256);
  J.comp = reinterpret_cast<int32_t*>(p);
  p += align_up((size_t)nseg * kSeg * 4, 256);
  J.seg_start = reinterpret_cast<int32_t*>(p);
  p += align_up((size_t)nseg * 4, 256);
  if (J.mode == 0) {
    J.table = reinterpret_cast<int32_t*>(p);
    J.fslot = J.table;
    p += align_up((size_t)J.B * (size_t)J.K * 4, 256);
    J.chain = reinterpret_cast<uint8_t*>(p);
    return;
  }
  J.p32 = reinterpret_cast<float2*>(p);
  p += align_up((size_t)m_max * sizeof(float2), 256);
  J.cand = reinterpret_cast<int32_t*>(p);
  p += align_up((size_t)(J.B + 1) * kCandMax * 4, 256);
  J.table = reinterpret_cast<int32_t*>(p);
  p += align_up((size_t)J.B * kCandMax * 4, 256);
  J.fslot = reinterpret_cast<int32_t*>(p);
  p += align_up((size_t)J.B * kCandMax * 4, 256);
  J.chain = reinterpret_cast<uint8_t*>(p);
  p += align_up((size_t)J.B, 256);
  J.box = reinterpret_cast<float4*>(p);
}

tsds_status launch_points_jobs(const PointsJob* jobs_dev, int count, int64_t max_m, cudaStream_t st) {
  note_launch();
  k_points<<<dim3(grid_for(max_m), (unsigned)count), 256, 0, st>>>(jobs_dev);
  TSDS_CK(cudaGetLastError());
  return TSDS_OK;
}

// The sequential sums of the flagged buckets of the jobs in `mode`.
static tsds_status launch_sums(const LttbJob* jobs_dev, int count, int64_t max_B, int mode, cudaStream_t st) {
  const int ssmem = (int)sizeof(SumRing);
  TSDS_CK(cudaFuncSetAttribute(k_sums_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, ssmem));
  note_launch();
  k_sums_wide<<<dim3((unsigned)((max_B + 31) / 32), (unsigned)count), kSumThreads, ssmem, st>>>(jobs_dev, mode);
  TSDS_CK(cudaGetLastError());
  return TSDS_OK;
}

tsds_status run_lttb_jobs(const LttbJob* jobs_host, const LttbJob* jobs_dev, int count, int64_t max_B,
                          int64_t max_m, cudaStream_t st) {
  bool any_table = false, any_hull = false;
  for (int i = 0; i < count; ++i) (jobs_host[i].mode == 0 ? any_table : any_hull) = true;
  const int64_t cap = (int64_t)device_sm_count() * 16;
  if (any_table) {
    note_launch();
    k_means<<<dim3(grid_for(max_B * 32, 8), (unsigned)count), 256, 0, st>>>(jobs_dev);   // lane groups per bucket
    TSDS_CK(cudaGetLastError());
    note_launch();
    k_sums_small<<<dim3(grid_for(max_B), (unsigned)count), 256, 0, st>>>(jobs_dev);   // flagged buckets
    TSDS_CK(cudaGetLastError());
    int64_t blocks = (max_B + 7) / 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    note_launch();
    k_table<<<dim3((unsigned)blocks, (unsigned)count), 256, 0, st>>>(jobs_dev);
    TSDS_CK(cudaGetLastError());
  }
  // table-mode jobs, and every job whose points are all kept, finish here
  note_launch();
  k_chase<<<(unsigned)count, 32, 0, st>>>(jobs_dev);
  TSDS_CK(cudaGetLastError());
  if (any_hull) {
    int64_t pb = (max_B + 7) / 8;
    if (pb > cap) pb = cap;
    note_launch();
    k_p32<<<dim3((unsigned)pb, (unsigned)count), 256, 0, st>>>(jobs_dev);
    TSDS_CK(cudaGetLastError());
    {
      const tsds_status r = launch_sums(jobs_dev, count, max_B, 2, st);
      if (r != TSDS_OK) return r;
    }
    int64_t hb = (max_B + kHullWarps - 1) / kHullWarps;
    if (hb > cap) hb = cap;
    if (hb < 1) hb = 1;
    const int hsmem = (int)(kHullWarps * sizeof(HullWarp));
    TSDS_CK(cudaFuncSetAttribute(k_hull, cudaFuncAttributeMaxDynamicSharedMemorySize, hsmem));
    note_launch();
    k_hull<<<dim3((unsigned)hb, (unsigned)count), kHullWarps * 32, hsmem, st>>>(jobs_dev);
    TSDS_CK(cudaGetLastError());
    int64_t tb = max_B;
    if (tb > cap) tb = cap;
    if (tb < 1) tb = 1;
    const int tsmem = (int)(kStageMax * sizeof(float2));
    note_launch();
    k_htable<<<dim3((unsigned)tb, (unsigned)count), kTableWarps * 32, tsmem, st>>>(jobs_dev);
    TSDS_CK(cudaGetLastError());
  }
  {
    const int64_t nseg = (max_B + kSeg - 1) / kSeg;
    int64_t cb = (nseg + kSegWarpsC - 1) / kSegWarpsC;
    if (cb > cap) cb = cap;
    if (cb < 1) cb = 1;
    note_launch();
    k_compose<<<dim3((unsigned)cb, (unsigned)count), kSegWarpsC * 32, 0, st>>>(jobs_dev);
    TSDS_CK(cudaGetLastError());
    note_launch();
    k_chain_seg<<<(unsigned)count, 32, 0, st>>>(jobs_dev);
    TSDS_CK(cudaGetLastError());
    note_launch();
    k_replay<<<dim3((unsigned)cb, (unsigned)count), kSegWarpsC * 32, 0, st>>>(jobs_dev);
    TSDS_CK(cudaGetLastError());
  }
  return TSDS_OK;
}

// LTTB over points px/py already in binary64 (m on the device when m_dev is
// set, otherwise m_host; m_max bounds it), writing R[pick] (or pick) to out.
static tsds_status lttb_points_core(const double* px, const double* py, const int64_t* m_dev, int64_t m_host,
                                    int64_t m_max, int64_t n_out, tsds_nan_mode nan, const int64_t* R,
                                    int64_t* out, int64_t* out_count, cudaStream_t st, bool x_index,
                                    double* means_out, const void* y, const void* x, const Gather* g) {
  LttbJob J;
  memset(&J, 0, sizeof J);
  J.px = px;
  J.py = py;
  J.m_dev = m_dev;
  J.m_host = m_host;
  J.B = n_out - 2;
  J.K = m_max > 2 ? (m_max - 2 + J.B - 1) / J.B : 1;
  J.nan = nan;
  J.R = R;
  J.out = out;
  J.out_count = out_count;
  J.x_index = x_index ? 1 : 0;
  if (g) {
    J.g = *g;
    J.ysrc = y;
    J.xsrc = x;
  }
  Scratch s;
  const size_t js = lttb_job_scratch(m_max, J.B, J.K);
  TSDS_CK(scratch_alloc(s, js + align_up(sizeof(LttbJob), 256), st));
  lttb_job_bind(J, static_cast<char*>(s.p), m_max);
  LttbJob* jd = reinterpret_cast<LttbJob*>(static_cast<char*>(s.p) + js);
  TSDS_CK(cudaMemcpyAsync(jd, &J, sizeof J, cudaMemcpyHostToDevice, st));
  const tsds_status r = run_lttb_jobs(&J, jd, 1, J.B, m_max, st);
  if (r == TSDS_OK && means_out && J.B > 1)
    TSDS_CK(cudaMemcpyAsync(means_out, J.means + 1, (size_t)(J.B - 1) * sizeof(double2), cudaMemcpyDeviceToDevice,
                            st));
  return r;
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
                     int64_t n_out, tsds_nan_mode nan, int64_t* out, int64_t* out_count, cudaStream_t st,
                     double* means_out, const Gather* g) {
  if (n == 0) {
    TSDS_CK(cudaMemsetAsync(out_count, 0, sizeof(int64_t), st));
    return TSDS_OK;
  }
  if (n_out >= n) {
    TSDS_CK(launch_iota(out, n, out_count, st, y, x, g));
    return TSDS_OK;
  }
  Scratch s;
  const size_t pb = align_up((size_t)n * 8, 256);
  TSDS_CK(scratch_alloc(s, 2 * pb, st));
  double* py = static_cast<double*>(s.p);
  double* px = reinterpret_cast<double*>(static_cast<char*>(s.p) + pb);
  tsds_status r = points(x, x_dtype, y, y_dtype, nullptr, nullptr, n, n, px, py, st);
  if (r != TSDS_OK) return r;
  return lttb_points_core(px, py, nullptr, n, n, n_out, nan, nullptr, out, out_count, st, x == nullptr, means_out,
                          y, x, g);
}

tsds_status run_minmaxlttb(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                           int64_t n, int64_t n_out, int64_t minmax_ratio, tsds_nan_mode nan,
                           int64_t* out, int64_t* out_count, cudaStream_t st, const Gather* g) {
  if (n == 0) {
    TSDS_CK(cudaMemsetAsync(out_count, 0, sizeof(int64_t), st));
    return TSDS_OK;
  }
  if (n_out >= n) {
    TSDS_CK(launch_iota(out, n, out_count, st, y, x, g));
    return TSDS_OK;
  }
  const int64_t n_sel = 2 * ((n_out * minmax_ratio) / 2);
  const int64_t n_in = n - 2;
  if (n_sel >= n_in) {
    // the preselection keeps every interior point: plain LTTB
    return run_lttb(x, x_dtype, y, y_dtype, n, n_out, nan, out, out_count, st, nullptr, g);
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
  return lttb_points_core(px, py, counts + 1, 0, m_max, n_out, nan, R, out, out_count, st, false, nullptr, y, x, g);
}

}  // namespace tsds
