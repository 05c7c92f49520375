// argminmax.cu -- the streaming per-bin argmin/argmax pass behind MinMax, M4
// and the MinMaxLTTB preselection.
//
// What it computes (Section 2.1, Listing 1): for every bin, the index of the
// smallest and of the largest value, the earliest index winning ties, NaNs
// handled by the NaN mode.  The paper's CPU kernel keeps four SIMD registers
// (lowest/highest values and their indices) and does a horizontal reduce at
// the end; it reads every value once because the work is memory-bound.
//
// GB300 design.  The pass is HBM-bound (a few integer or FP32 operations per
// byte), so the kernel is built around keeping enough bytes in flight:
//  * y is cut into fixed windows of kWindowBytes; a persistent grid of warps
//    claims windows from an atomic counter (load balance across the 152 SMs
//    whatever the bin sizes), and each warp walks the bins overlapping its
//    window.  A bin is cut where windows cut it.
//  * Within a bin piece every lane streams 16-byte vectors with coalesced
//    loads, U vectors (64 bytes) per lane per step.  Per step the lane reduces
//    its U vectors to one group minimum and maximum with packed 16x2 integer
//    or FP32/FP16x2 min/max instructions (no per-element index bookkeeping)
//    and remembers the step where the running extremum last strictly
//    improved.  After every CH steps it resolves that step's element index by
//    re-reading the 64 bytes (an L2 hit) and keeping the first element equal
//    to the extremum.  The first step whose group extremum equals the final
//    extremum holds its first occurrence, so the earliest index survives.
//  * Lanes then combine (ordered 64-bit key, index) pairs with warp shuffles.
//    A bin held by one window is written directly; pieces of a bin that
//    spans windows go to per-window slots, and the warp whose atomic
//    increment completes the bin's piece count combines them.  Nothing waits.
#include <type_traits>

#include "device.cuh"
#include "internal.h"

namespace tsds {

constexpr int kU = 4;    // 16-byte vectors per lane per step
constexpr int kCH = 8;   // steps between index resolutions

// ---------------------------------------------------------------------------
// Packed 16x2 helpers (sm_90+ PTX).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t min_s16x2(uint32_t a, uint32_t b) {
  uint32_t r; asm("min.s16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r;
}
__device__ __forceinline__ uint32_t max_s16x2(uint32_t a, uint32_t b) {
  uint32_t r; asm("max.s16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r;
}
__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b) {
  uint32_t r; asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r;
}
__device__ __forceinline__ uint32_t max_u16x2(uint32_t a, uint32_t b) {
  uint32_t r; asm("max.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r;
}
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t r; asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel)); return r;
}
__device__ __forceinline__ float fmin_nan(float a, float b) {
  float r; asm("min.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b)); return r;
}
__device__ __forceinline__ float fmax_nan(float a, float b) {
  float r; asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b)); return r;
}

template <class T, int E>
__device__ __forceinline__ T vec_elem(const uint4& v, int e) {
  T arr[E];
  memcpy(arr, &v, 16);
  return arr[e];
}

// ---------------------------------------------------------------------------
// Policies: how a dtype reduces a group of U vectors and how its running
// extremum compares, matches an element and becomes an ordered key.
// ---------------------------------------------------------------------------

// float32: FP32 min/max; NaN via min.NaN (propagate) or fminf (ignore).
template <int NM>
struct PolF32 {
  using T = float;
  using Acc = float;
  static constexpr int E = 4;
  static constexpr bool kFloat = true;
  __device__ static float mn(float a, float b) { return NM == TSDS_NAN_PROPAGATE ? fmin_nan(a, b) : fminf(a, b); }
  __device__ static float mx(float a, float b) { return NM == TSDS_NAN_PROPAGATE ? fmax_nan(a, b) : fmaxf(a, b); }
  __device__ static void group(const uint4 (&v)[kU], Acc& gmin, Acc& gmax) {
    float a[kU], b[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      float f0 = __uint_as_float(v[u].x), f1 = __uint_as_float(v[u].y);
      float f2 = __uint_as_float(v[u].z), f3 = __uint_as_float(v[u].w);
      a[u] = mn(mn(f0, f1), mn(f2, f3));
      b[u] = mx(mx(f0, f1), mx(f2, f3));
    }
    gmin = mn(mn(a[0], a[1]), mn(a[2], a[3]));
    gmax = mx(mx(b[0], b[1]), mx(b[2], b[3]));
  }
  __device__ static bool better_min(Acc g, Acc r) {
    return NM == TSDS_NAN_PROPAGATE ? (g < r || (isnan(g) && !isnan(r))) : (g < r || (isnan(r) && !isnan(g)));
  }
  __device__ static bool better_max(Acc g, Acc r) {
    return NM == TSDS_NAN_PROPAGATE ? (g > r || (isnan(g) && !isnan(r))) : (g > r || (isnan(r) && !isnan(g)));
  }
  __device__ static bool match(T e, Acc t) { return isnan(t) ? isnan(e) : e == t; }
  __device__ static bool match_min(T e, Acc t) { return match(e, t); }
  __device__ static bool match_max(T e, Acc t) { return match(e, t); }
  __device__ static uint64_t key_min(Acc a) { return fkey_min<NM>((double)a); }
  __device__ static uint64_t key_max(Acc a) { return fkey_max<NM>((double)a); }
  __device__ static uint64_t elem_key_min(T e) { return fkey_min<NM>((double)e); }
  __device__ static uint64_t elem_key_max(T e) { return fkey_max<NM>((double)e); }
};

// float16: packed half2 min/max, then one FP32 comparison per group.
template <int NM>
struct PolF16 {
  using T = __half;
  using Acc = float;
  static constexpr int E = 8;
  static constexpr bool kFloat = true;
  __device__ static __half2 mn2(__half2 a, __half2 b) { return NM == TSDS_NAN_PROPAGATE ? __hmin2_nan(a, b) : __hmin2(a, b); }
  __device__ static __half2 mx2(__half2 a, __half2 b) { return NM == TSDS_NAN_PROPAGATE ? __hmax2_nan(a, b) : __hmax2(a, b); }
  __device__ static float mnf(float a, float b) { return NM == TSDS_NAN_PROPAGATE ? fmin_nan(a, b) : fminf(a, b); }
  __device__ static float mxf(float a, float b) { return NM == TSDS_NAN_PROPAGATE ? fmax_nan(a, b) : fmaxf(a, b); }
  __device__ static __half2 h2(uint32_t w) { return *reinterpret_cast<__half2*>(&w); }
  __device__ static void group(const uint4 (&v)[kU], Acc& gmin, Acc& gmax) {
    __half2 a[kU], b[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      __half2 w0 = h2(v[u].x), w1 = h2(v[u].y), w2 = h2(v[u].z), w3 = h2(v[u].w);
      a[u] = mn2(mn2(w0, w1), mn2(w2, w3));
      b[u] = mx2(mx2(w0, w1), mx2(w2, w3));
    }
    __half2 lo = mn2(mn2(a[0], a[1]), mn2(a[2], a[3]));
    __half2 hi = mx2(mx2(b[0], b[1]), mx2(b[2], b[3]));
    gmin = mnf(__low2float(lo), __high2float(lo));
    gmax = mxf(__low2float(hi), __high2float(hi));
  }
  __device__ static bool better_min(Acc g, Acc r) { return PolF32<NM>::better_min(g, r); }
  __device__ static bool better_max(Acc g, Acc r) { return PolF32<NM>::better_max(g, r); }
  __device__ static bool match(T e, Acc t) { float f = __half2float(e); return isnan(t) ? isnan(f) : f == t; }
  __device__ static bool match_min(T e, Acc t) { return match(e, t); }
  __device__ static bool match_max(T e, Acc t) { return match(e, t); }
  __device__ static uint64_t key_min(Acc a) { return fkey_min<NM>((double)a); }
  __device__ static uint64_t key_max(Acc a) { return fkey_max<NM>((double)a); }
  __device__ static uint64_t elem_key_min(T e) { return fkey_min<NM>((double)__half2float(e)); }
  __device__ static uint64_t elem_key_max(T e) { return fkey_max<NM>((double)__half2float(e)); }
};

// 8- and 16-bit integers: widen to 16-bit lanes (PRMT) and reduce with packed
// 16x2 min/max, two elements per instruction.
template <class T_>
struct PolSmallInt {
  using T = T_;
  using Acc = int32_t;
  static constexpr int E = 16 / sizeof(T_);
  static constexpr bool kFloat = false;
  static constexpr bool kSigned = (T_)(-1) < (T_)0;
  __device__ static uint32_t mn(uint32_t a, uint32_t b) { return kSigned ? min_s16x2(a, b) : min_u16x2(a, b); }
  __device__ static uint32_t mx(uint32_t a, uint32_t b) { return kSigned ? max_s16x2(a, b) : max_u16x2(a, b); }
  __device__ static int32_t lane_lo(uint32_t w) { return kSigned ? (int32_t)(int16_t)(w & 0xFFFFu) : (int32_t)(w & 0xFFFFu); }
  __device__ static int32_t lane_hi(uint32_t w) { return kSigned ? ((int32_t)w >> 16) : (int32_t)(w >> 16); }
  __device__ static void group(const uint4 (&v)[kU], Acc& gmin, Acc& gmax) {
    uint32_t w[4 * kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) { w[4 * u] = v[u].x; w[4 * u + 1] = v[u].y; w[4 * u + 2] = v[u].z; w[4 * u + 3] = v[u].w; }
    uint32_t lo, hi;
    if (sizeof(T_) == 2) {
      lo = w[0]; hi = w[0];
#pragma unroll
      for (int i = 1; i < 4 * kU; ++i) { lo = mn(lo, w[i]); hi = mx(hi, w[i]); }
    } else {
      // bytes 0,2 and bytes 1,3 of each word as 16-bit lanes (sign- or zero-extended)
      const uint32_t sel_even = kSigned ? 0xA280u : 0x4240u;
      const uint32_t sel_odd = kSigned ? 0xB391u : 0x4341u;
      uint32_t e0 = prmt(w[0], 0u, sel_even), o0 = prmt(w[0], 0u, sel_odd);
      lo = mn(e0, o0); hi = mx(e0, o0);
#pragma unroll
      for (int i = 1; i < 4 * kU; ++i) {
        uint32_t e = prmt(w[i], 0u, sel_even), o = prmt(w[i], 0u, sel_odd);
        lo = mn(lo, mn(e, o));
        hi = mx(hi, mx(e, o));
      }
    }
    gmin = min(lane_lo(lo), lane_hi(lo));
    gmax = max(lane_lo(hi), lane_hi(hi));
  }
  __device__ static bool better_min(Acc g, Acc r) { return g < r; }
  __device__ static bool better_max(Acc g, Acc r) { return g > r; }
  __device__ static bool match_min(T e, Acc t) { return (int32_t)e == t; }
  __device__ static bool match_max(T e, Acc t) { return (int32_t)e == t; }
  __device__ static uint64_t key_min(Acc a) { return kSigned ? skey((int64_t)a) : ukey((uint64_t)(uint32_t)a); }
  __device__ static uint64_t key_max(Acc a) { return key_min(a); }
  __device__ static uint64_t elem_key_min(T e) { return kSigned ? skey((int64_t)e) : ukey((uint64_t)e); }
  __device__ static uint64_t elem_key_max(T e) { return elem_key_min(e); }
};

// 32-bit integers: native integer min/max.
template <class T_>
struct PolInt32 {
  using T = T_;
  using Acc = T_;
  static constexpr int E = 4;
  static constexpr bool kFloat = false;
  static constexpr bool kSigned = (T_)(-1) < (T_)0;
  __device__ static void group(const uint4 (&v)[kU], Acc& gmin, Acc& gmax) {
    T a[kU], b[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      T e0 = (T)v[u].x, e1 = (T)v[u].y, e2 = (T)v[u].z, e3 = (T)v[u].w;
      a[u] = min(min(e0, e1), min(e2, e3));
      b[u] = max(max(e0, e1), max(e2, e3));
    }
    gmin = min(min(a[0], a[1]), min(a[2], a[3]));
    gmax = max(max(b[0], b[1]), max(b[2], b[3]));
  }
  __device__ static bool better_min(Acc g, Acc r) { return g < r; }
  __device__ static bool better_max(Acc g, Acc r) { return g > r; }
  __device__ static bool match_min(T e, Acc t) { return e == t; }
  __device__ static bool match_max(T e, Acc t) { return e == t; }
  __device__ static uint64_t key_min(Acc a) { return kSigned ? skey((int64_t)a) : ukey((uint64_t)a); }
  __device__ static uint64_t key_max(Acc a) { return key_min(a); }
  __device__ static uint64_t elem_key_min(T e) { return key_min(e); }
  __device__ static uint64_t elem_key_max(T e) { return key_min(e); }
};

// 64-bit types: compare ordered 64-bit keys with integer instructions (the
// FP64 pipe is narrow on this GPU).  float64 takes the raw sign-magnitude key
// first and only re-maps NaNs when a group's key range shows one.
template <int KIND, int NM>   // KIND 0: int64, 1: uint64, 2: float64
struct Pol64 {
  using T = typename std::conditional<KIND == 0, int64_t, typename std::conditional<KIND == 1, uint64_t, double>::type>::type;
  using Acc = uint64_t;
  static constexpr int E = 2;
  static constexpr bool kFloat = KIND == 2;
  __device__ static uint64_t raw(uint64_t b) {
    if (KIND == 0) return b ^ kSign64;
    if (KIND == 1) return b;
    return f64_bits_key(b);
  }
  __device__ static uint64_t kmin_of(uint64_t k) { return (KIND == 2 && raw_key_is_nan(k)) ? nan_key_min<NM>() : k; }
  __device__ static uint64_t kmax_of(uint64_t k) { return (KIND == 2 && raw_key_is_nan(k)) ? nan_key_max<NM>() : k; }
  __device__ static void group(const uint4 (&v)[kU], Acc& gmin, Acc& gmax) {
    uint64_t k[2 * kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      k[2 * u] = raw(((uint64_t)v[u].y << 32) | v[u].x);
      k[2 * u + 1] = raw(((uint64_t)v[u].w << 32) | v[u].z);
    }
    uint64_t lo = k[0], hi = k[0];
#pragma unroll
    for (int i = 1; i < 2 * kU; ++i) { lo = min(lo, k[i]); hi = max(hi, k[i]); }
    if (KIND == 2 && (raw_key_is_nan(lo) || raw_key_is_nan(hi))) {
      lo = kmin_of(k[0]); hi = kmax_of(k[0]);
#pragma unroll
      for (int i = 1; i < 2 * kU; ++i) { lo = min(lo, kmin_of(k[i])); hi = max(hi, kmax_of(k[i])); }
    }
    gmin = lo;
    gmax = hi;
  }
  __device__ static uint64_t bits(T e) {
    if constexpr (KIND == 2) {
      return f64_bits(e);   // opaque move: keeps the key arithmetic integer
    } else {
      return (uint64_t)e;
    }
  }
  __device__ static bool better_min(Acc g, Acc r) { return g < r; }
  __device__ static bool better_max(Acc g, Acc r) { return g > r; }
  __device__ static bool match_min(T e, Acc t) { return kmin_of(raw(bits(e))) == t; }
  __device__ static bool match_max(T e, Acc t) { return kmax_of(raw(bits(e))) == t; }
  __device__ static uint64_t key_min(Acc a) { return a; }
  __device__ static uint64_t key_max(Acc a) { return a; }
  __device__ static uint64_t elem_key_min(T e) { return kmin_of(raw(bits(e))); }
  __device__ static uint64_t elem_key_max(T e) { return kmax_of(raw(bits(e))); }
};

// ---------------------------------------------------------------------------
// One bin piece [a, b) of a series, reduced by one warp.
// ---------------------------------------------------------------------------
template <class P, bool MIN>
__device__ __noinline__ int find_first(const uint4* __restrict__ vp, int nvec, int t, int lane,
                                       typename P::Acc target) {
  // element offset (from the first body element) of the first match in step t
  using T = typename P::T;
  const int vb = t * (32 * kU) + lane;
#pragma unroll 1
  for (int u = 0; u < kU; ++u) {
    const int vi = vb + u * 32;
    if (vi >= nvec) break;
    const uint4 v = ldg_vec(vp + vi);
#pragma unroll
    for (int e = 0; e < P::E; ++e) {
      const T val = vec_elem<T, P::E>(v, e);
      if (MIN ? P::match_min(val, target) : P::match_max(val, target)) return vi * P::E + e;
    }
  }
  return -1;
}

template <class P>
__device__ __forceinline__ Cand piece_argminmax(const typename P::T* __restrict__ y, int64_t a, int64_t b) {
  using T = typename P::T;
  using Acc = typename P::Acc;
  constexpr int E = P::E;
  const int lane = threadIdx.x & 31;
  Cand c;
  cand_init(c);

  // body: the 16-byte aligned vectors inside [a, b); head and tail elements
  // outside it go through the scalar path
  const uintptr_t addr = reinterpret_cast<uintptr_t>(y + a);
  int64_t ia = a + (int64_t)(((16u - (unsigned)(addr & 15u)) & 15u) / sizeof(T));
  if (ia > b) ia = b;
  const int64_t nvec = (b - ia) / E;
  const int64_t ib = ia + nvec * E;
  for (int64_t i = a + lane; i < ia; i += 32) {
    const T e = ldg_elem<T>(y + i);
    cand_merge_min(c, P::elem_key_min(e), i);
    cand_merge_max(c, P::elem_key_max(e), i);
  }
  for (int64_t i = ib + lane; i < b; i += 32) {
    const T e = ldg_elem<T>(y + i);
    cand_merge_min(c, P::elem_key_min(e), i);
    cand_merge_max(c, P::elem_key_max(e), i);
  }

  if (nvec > 0) {
    // a piece never exceeds one window, so step and vector numbers fit in 32 bits
    const uint4* __restrict__ vp = reinterpret_cast<const uint4*>(y + ia);
    const int nv = (int)nvec;
    const int iters = (nv + 32 * kU - 1) / (32 * kU);
    bool rvalid = false;
    Acc rmin{}, rmax{};
    int rimin = -1, rimax = -1;
    for (int t0 = 0; t0 < iters; t0 += kCH) {
      const int t1 = min(t0 + kCH, iters);
      bool cvalid = false;
      Acc cmin{}, cmax{};
      int tmin = 0, tmax = 0;
      for (int t = t0; t < t1; ++t) {
        const int vb = t * (32 * kU) + lane;
        uint4 v[kU];
        if (vb + (kU - 1) * 32 < nv) {
#pragma unroll
          for (int u = 0; u < kU; ++u) v[u] = ldg_vec(vp + vb + u * 32);
        } else {
          if (vb >= nv) continue;
          v[0] = ldg_vec(vp + vb);
#pragma unroll
          for (int u = 1; u < kU; ++u) v[u] = (vb + u * 32 < nv) ? ldg_vec(vp + vb + u * 32) : v[0];
        }
        Acc gmin, gmax;
        P::group(v, gmin, gmax);
        if (!cvalid || P::better_min(gmin, cmin)) { cmin = gmin; tmin = t; }
        if (!cvalid || P::better_max(gmax, cmax)) { cmax = gmax; tmax = t; }
        cvalid = true;
      }
      if (cvalid) {
        if (!rvalid || P::better_min(cmin, rmin)) {
          rmin = cmin;
          rimin = find_first<P, true>(vp, nv, tmin, lane, cmin);
        }
        if (!rvalid || P::better_max(cmax, rmax)) {
          rmax = cmax;
          rimax = find_first<P, false>(vp, nv, tmax, lane, cmax);
        }
        rvalid = true;
      }
    }
    if (rvalid) {
      cand_merge_min(c, P::key_min(rmin), ia + rimin);
      cand_merge_max(c, P::key_max(rmax), ia + rimax);
    }
  }
  cand_warp_reduce(c);
  return c;
}

// NaN-ignore: an all-NaN bin keeps the sentinel keys; it selects its first index.
template <class P, int NM>
__device__ __forceinline__ void finish_bin(Cand& c, int64_t lo) {
  if (P::kFloat && NM == TSDS_NAN_IGNORE) {
    if (c.kmin == kKeyMax) c.imin = lo;
    if (c.kmax == 0) c.imax = lo;
  }
}

__device__ __forceinline__ Piece load_piece_cg(const Piece* p) {
  Piece r;
  const uint4* q = reinterpret_cast<const uint4*>(p);
  uint4 a = __ldcg(q), b = __ldcg(q + 1);
  r.kmin = ((uint64_t)a.y << 32) | a.x;
  r.imin = (int64_t)(((uint64_t)a.w << 32) | a.z);
  r.kmax = ((uint64_t)b.y << 32) | b.x;
  r.imax = (int64_t)(((uint64_t)b.w << 32) | b.z);
  return r;
}

template <class P, int NM, bool MULTI>
__global__ void __launch_bounds__(kStreamThreads)
k_argminmax(const SeriesDev* __restrict__ sd, SeriesDev single, const int32_t* __restrict__ win_series,
            int64_t total_windows, Piece* __restrict__ first_piece, Piece* __restrict__ last_piece,
            WorkCounters* __restrict__ work, int64_t welems, const int64_t* __restrict__ total_dev) {
  using T = typename P::T;
  const int lane = threadIdx.x & 31;
  if (total_dev) total_windows = *total_dev;
  for (;;) {
    unsigned long long wu = 0;
    if (lane == 0) wu = atomicAdd(&work->next_window, 1ull);
    const int64_t w = (int64_t)__shfl_sync(0xffffffffu, wu, 0);
    if (w >= total_windows) break;
    SeriesDev S = MULTI ? sd[win_series[w]] : single;
    const T* __restrict__ y = static_cast<const T*>(S.y);
    const int64_t* __restrict__ edges = S.edges;
    const int64_t nb = S.nb;
    const int64_t k = w - S.win_base;
    const int64_t ws = k * welems;
    const int64_t we = min(ws + welems, S.n);
    // the bin holding ws: the last b with edges[b] <= ws
    int64_t b = warp_lower_bound(1, nb + 1, [&](int64_t j) { return __ldg(edges + j) > ws; }) - 1;
    int64_t lo = __ldg(edges + b);
    while (b < nb && lo < we) {
      const int64_t hi = __ldg(edges + b + 1);
      if (hi > lo) {
        const int64_t pa = max(lo, ws), pb = min(hi, we);
        Cand c = piece_argminmax<P>(y, pa, pb);
        const int64_t k0 = lo / welems, k1 = (hi - 1) / welems;
        if (k0 == k1) {
          finish_bin<P, NM>(c, lo);
          if (lane == 0) { S.res[2 * b] = c.imin; S.res[2 * b + 1] = c.imax; }
        } else {
          Piece* slot = (k == k0) ? &last_piece[S.win_base + k] : &first_piece[S.win_base + k];
          unsigned done = 0;
          if (lane == 0) {
            *slot = Piece{c.kmin, c.imin, c.kmax, c.imax};
            __threadfence();
            done = atomicAdd(&S.cnt[b], 1u);
          }
          done = __shfl_sync(0xffffffffu, done, 0);
          if ((int64_t)done == k1 - k0) {
            // every other piece of this bin is published: combine them all
            __threadfence();
            Cand t;
            cand_init(t);
            for (int64_t p = lane; p <= k1 - k0; p += 32) {
              const Piece q = load_piece_cg(p == 0 ? &last_piece[S.win_base + k0] : &first_piece[S.win_base + k0 + p]);
              cand_merge_min(t, q.kmin, q.imin);
              cand_merge_max(t, q.kmax, q.imax);
            }
            cand_warp_reduce(t);
            finish_bin<P, NM>(t, lo);
            if (lane == 0) { S.res[2 * b] = t.imin; S.res[2 * b + 1] = t.imax; S.cnt[b] = 0u; }
          }
        }
      }
      lo = hi;
      ++b;
    }
  }
}

template <class P, int NM>
static cudaError_t launch_pol(const SeriesDev* s_dev, int count, const SeriesDev& single,
                              const int32_t* win_series, int64_t total_windows, Piece* fp, Piece* lp,
                              WorkCounters* work, const StreamConfig& cfg, cudaStream_t st) {
  const bool multi = count > 1 || s_dev != nullptr;
  auto kern = multi ? k_argminmax<P, NM, true> : k_argminmax<P, NM, false>;
  static int per_sm[2] = {0, 0};
  int& occ = per_sm[multi ? 1 : 0];
  if (occ == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kStreamThreads, 0);
    if (e != cudaSuccess || occ < 1) occ = 1;
  }
  const int per = (cfg.ctas_per_sm > 0 && cfg.ctas_per_sm < occ) ? cfg.ctas_per_sm : occ;
  const int64_t warps_per_block = kStreamThreads / 32;
  int64_t blocks = (total_windows + warps_per_block - 1) / warps_per_block;
  const int64_t cap = (int64_t)device_sm_count() * per;
  if (blocks > cap || cfg.total_windows_dev) blocks = cap;
  if (blocks < 1) blocks = 1;
  note_launch();
  kern<<<(unsigned)blocks, kStreamThreads, 0, st>>>(s_dev, single, win_series, total_windows, fp, lp, work,
                                                     cfg.window_bytes / (int64_t)sizeof(typename P::T),
                                                     cfg.total_windows_dev);
  return cudaGetLastError();
}

using PolI64 = Pol64<0, 0>;
using PolU64 = Pol64<1, 0>;
using PolF64Prop = Pol64<2, TSDS_NAN_PROPAGATE>;
using PolF64Ign = Pol64<2, TSDS_NAN_IGNORE>;

cudaError_t launch_argminmax(const SeriesDev* s_dev, int count, const SeriesDev& single,
                             const int32_t* win_series, int64_t total_windows,
                             Piece* first_piece, Piece* last_piece, WorkCounters* work,
                             tsds_dtype y_dtype, tsds_nan_mode nan, cudaStream_t st, const StreamConfig& cfg) {
  if (total_windows <= 0) return cudaSuccess;
  const bool ign = nan == TSDS_NAN_IGNORE;
#define TSDS_LAUNCH(POL, NM) launch_pol<POL, NM>(s_dev, count, single, win_series, total_windows, first_piece, last_piece, work, cfg, st)
  switch (y_dtype) {
    case TSDS_I8: return TSDS_LAUNCH(PolSmallInt<int8_t>, 0);
    case TSDS_U8: return TSDS_LAUNCH(PolSmallInt<uint8_t>, 0);
    case TSDS_I16: return TSDS_LAUNCH(PolSmallInt<int16_t>, 0);
    case TSDS_U16: return TSDS_LAUNCH(PolSmallInt<uint16_t>, 0);
    case TSDS_I32: return TSDS_LAUNCH(PolInt32<int32_t>, 0);
    case TSDS_U32: return TSDS_LAUNCH(PolInt32<uint32_t>, 0);
    case TSDS_I64: return TSDS_LAUNCH(PolI64, 0);
    case TSDS_U64: return TSDS_LAUNCH(PolU64, 0);
    case TSDS_F16: return ign ? TSDS_LAUNCH(PolF16<1>, 1) : TSDS_LAUNCH(PolF16<0>, 0);
    case TSDS_F32: return ign ? TSDS_LAUNCH(PolF32<1>, 1) : TSDS_LAUNCH(PolF32<0>, 0);
    case TSDS_F64: return ign ? TSDS_LAUNCH(PolF64Ign, 1) : TSDS_LAUNCH(PolF64Prop, 0);
    default: return cudaErrorInvalidValue;
  }
#undef TSDS_LAUNCH
}

// Single-series launch with the SM count given by the caller instead of the
// library's per-device state, for the entry point that must not create the
// library's memory pool (tsds_minmax_noalloc).
template <class P, int NM>
static cudaError_t launch_pol_sm(const SeriesDev& single, int64_t total_windows, Piece* fp, Piece* lp,
                                 WorkCounters* work, int sm_count, cudaStream_t st) {
  auto kern = k_argminmax<P, NM, false>;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kStreamThreads, 0) != cudaSuccess || occ < 1)
    occ = 1;
  int64_t blocks = (total_windows + kStreamThreads / 32 - 1) / (kStreamThreads / 32);
  const int64_t cap = (int64_t)sm_count * occ;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  note_launch();
  kern<<<(unsigned)blocks, kStreamThreads, 0, st>>>(nullptr, single, nullptr, total_windows, fp, lp, work,
                                                     kWindowBytes / (int64_t)sizeof(typename P::T), nullptr);
  return cudaGetLastError();
}

cudaError_t launch_argminmax_sm(const SeriesDev& single, int64_t total_windows, Piece* first_piece,
                                Piece* last_piece, WorkCounters* work, tsds_dtype y_dtype, tsds_nan_mode nan,
                                int sm_count, cudaStream_t st) {
  if (total_windows <= 0) return cudaSuccess;
  const bool ign = nan == TSDS_NAN_IGNORE;
#define TSDS_LAUNCH(POL, NM) launch_pol_sm<POL, NM>(single, total_windows, first_piece, last_piece, work, sm_count, st)
  switch (y_dtype) {
    case TSDS_I8: return TSDS_LAUNCH(PolSmallInt<int8_t>, 0);
    case TSDS_U8: return TSDS_LAUNCH(PolSmallInt<uint8_t>, 0);
    case TSDS_I16: return TSDS_LAUNCH(PolSmallInt<int16_t>, 0);
    case TSDS_U16: return TSDS_LAUNCH(PolSmallInt<uint16_t>, 0);
    case TSDS_I32: return TSDS_LAUNCH(PolInt32<int32_t>, 0);
    case TSDS_U32: return TSDS_LAUNCH(PolInt32<uint32_t>, 0);
    case TSDS_I64: return TSDS_LAUNCH(PolI64, 0);
    case TSDS_U64: return TSDS_LAUNCH(PolU64, 0);
    case TSDS_F16: return ign ? TSDS_LAUNCH(PolF16<1>, 1) : TSDS_LAUNCH(PolF16<0>, 0);
    case TSDS_F32: return ign ? TSDS_LAUNCH(PolF32<1>, 1) : TSDS_LAUNCH(PolF32<0>, 0);
    case TSDS_F64: return ign ? TSDS_LAUNCH(PolF64Ign, 1) : TSDS_LAUNCH(PolF64Prop, 0);
    default: return cudaErrorInvalidValue;
  }
#undef TSDS_LAUNCH
}

}  // namespace tsds
