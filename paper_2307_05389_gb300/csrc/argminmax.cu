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
//  * y is cut into windows (a multiple of 4 KB); a persistent grid of warps
//    claims windows from an atomic counter (load balance across the 152 SMs
//    whatever the bin sizes), and each warp walks the bins overlapping its
//    window.  A bin is cut where windows cut it.
//  * Each warp streams its window through a private ring of 4 shared-memory
//    stages of 4 KB filled by bulk asynchronous copies (cp.async.bulk with an
//    mbarrier per stage), so every warp keeps 16 KB in flight without holding
//    any of it in registers; small bins cost shared-memory latency, not DRAM
//    latency.
//  * A bin's part of a chunk is reduced by all lanes, 4 vectors of 16 bytes
//    per lane per step: packed 16x2 integer or FP32/FP16x2 min/max
//    instructions reduce a step to one group minimum and maximum (no
//    per-element index bookkeeping) and each lane remembers the step where its
//    extremum last strictly improved.  Before the chunk is released the lane
//    finds the first element equal to its extremum in that step, from shared
//    memory; the first step whose group extremum equals the final one holds
//    its first occurrence, so the earliest index survives.
//  * A second variant (stream_ldg.cuh) loads the same steps straight into
//    registers and resolves indices every 8 steps from a cached re-read; with
//    less bookkeeping per byte it is the faster one for large bins, the ring
//    for small ones.  Each launch picks one by its bytes-weighted mean bin
//    size (the batched plans can also time both).
//  * Lanes then combine (ordered 64-bit key, index) pairs with warp shuffles.
//    A bin held by one window is written directly; pieces of a bin that
//    spans windows go to per-window slots, and the warp whose atomic
//    increment completes the bin's piece count combines them.  The only waits
//    are on the ring's barriers, and they are bounded.
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <type_traits>

#include "device.cuh"
#include "internal.h"

namespace tsds {

constexpr int kU = 4;    // 16-byte vectors per lane per step

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
// three-input forms (sm_100 and later): NaN if any input is NaN (.NaN), else
// the least / greatest of the non-NaN inputs
__device__ __forceinline__ float fmin3_nan(float a, float b, float c) {
  float r; asm("min.NaN.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c)); return r;
}
__device__ __forceinline__ float fmax3_nan(float a, float b, float c) {
  float r; asm("max.NaN.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c)); return r;
}
__device__ __forceinline__ float fmin3_num(float a, float b, float c) {
  float r; asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c)); return r;
}
__device__ __forceinline__ float fmax3_num(float a, float b, float c) {
  float r; asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c)); return r;
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
  __device__ static void group1(const uint4& v, Acc& gmin, Acc& gmax) {
    const float f0 = __uint_as_float(v.x), f1 = __uint_as_float(v.y);
    const float f2 = __uint_as_float(v.z), f3 = __uint_as_float(v.w);
    if (NM == TSDS_NAN_PROPAGATE) {
      gmin = fmin3_nan(f0, f1, fmin_nan(f2, f3));
      gmax = fmax3_nan(f0, f1, fmax_nan(f2, f3));
    } else {
      gmin = fmin3_num(f0, f1, fminf(f2, f3));
      gmax = fmax3_num(f0, f1, fmaxf(f2, f3));
    }
  }
  // propagate: g < r, or g NaN and r not; ignore: g < r, or r NaN and g not
  // (!(g >= r) holds for g < r and whenever either is NaN)
  __device__ static bool better_min(Acc g, Acc r) {
    return NM == TSDS_NAN_PROPAGATE ? (!(g >= r) && r == r) : (!(g >= r) && g == g);
  }
  __device__ static bool better_max(Acc g, Acc r) {
    return NM == TSDS_NAN_PROPAGATE ? (!(g <= r) && r == r) : (!(g <= r) && g == g);
  }
  __device__ static bool match(T e, Acc t) { return isnan(t) ? isnan(e) : e == t; }
  __device__ static bool match_min(T e, Acc t) { return match(e, t); }
  __device__ static bool match_max(T e, Acc t) { return match(e, t); }
  __device__ static uint64_t key_min(Acc a) { return f32key_min<NM>(a); }
  __device__ static uint64_t key_max(Acc a) { return f32key_max<NM>(a); }
  __device__ static uint64_t elem_key_min(T e) { return f32key_min<NM>(e); }
  __device__ static uint64_t elem_key_max(T e) { return f32key_max<NM>(e); }
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
  __device__ static void group1(const uint4& v, Acc& gmin, Acc& gmax) {
    const __half2 w0 = h2(v.x), w1 = h2(v.y), w2 = h2(v.z), w3 = h2(v.w);
    const __half2 lo = mn2(mn2(w0, w1), mn2(w2, w3));
    const __half2 hi = mx2(mx2(w0, w1), mx2(w2, w3));
    gmin = mnf(__low2float(lo), __high2float(lo));
    gmax = mxf(__low2float(hi), __high2float(hi));
  }
  __device__ static bool better_min(Acc g, Acc r) { return PolF32<NM>::better_min(g, r); }
  __device__ static bool better_max(Acc g, Acc r) { return PolF32<NM>::better_max(g, r); }
  __device__ static bool match(T e, Acc t) { float f = __half2float(e); return isnan(t) ? isnan(f) : f == t; }
  __device__ static bool match_min(T e, Acc t) { return match(e, t); }
  __device__ static bool match_max(T e, Acc t) { return match(e, t); }
  __device__ static uint64_t key_min(Acc a) { return f32key_min<NM>(a); }
  __device__ static uint64_t key_max(Acc a) { return f32key_max<NM>(a); }
  __device__ static uint64_t elem_key_min(T e) { return f32key_min<NM>(__half2float(e)); }
  __device__ static uint64_t elem_key_max(T e) { return f32key_max<NM>(__half2float(e)); }
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
  __device__ static void group1(const uint4& v, Acc& gmin, Acc& gmax) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t lo, hi;
    if (sizeof(T_) == 2) {
      lo = mn(mn(w[0], w[1]), mn(w[2], w[3]));
      hi = mx(mx(w[0], w[1]), mx(w[2], w[3]));
    } else {
      const uint32_t sel_even = kSigned ? 0xA280u : 0x4240u;
      const uint32_t sel_odd = kSigned ? 0xB391u : 0x4341u;
      uint32_t e[4], o[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { e[i] = prmt(w[i], 0u, sel_even); o[i] = prmt(w[i], 0u, sel_odd); }
      lo = mn(mn(mn(e[0], o[0]), mn(e[1], o[1])), mn(mn(e[2], o[2]), mn(e[3], o[3])));
      hi = mx(mx(mx(e[0], o[0]), mx(e[1], o[1])), mx(mx(e[2], o[2]), mx(e[3], o[3])));
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
  __device__ static void group1(const uint4& v, Acc& gmin, Acc& gmax) {
    const T e0 = (T)v.x, e1 = (T)v.y, e2 = (T)v.z, e3 = (T)v.w;
    gmin = min(min(e0, e1), min(e2, e3));
    gmax = max(max(e0, e1), max(e2, e3));
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
  __device__ static void group1(const uint4& v, Acc& gmin, Acc& gmax) {
    const uint64_t k0 = raw(((uint64_t)v.y << 32) | v.x), k1 = raw(((uint64_t)v.w << 32) | v.z);
    gmin = min(k0, k1);
    gmax = max(k0, k1);
    // raw NaN keys lie outside [key(-inf), key(+inf)], so one of the two is a
    // NaN exactly when the smaller lies below that range or the larger above
    if (KIND == 2 && (gmin < kKeyNegInf || gmax > kKeyPosInf)) {
      gmin = min(kmin_of(k0), kmin_of(k1));
      gmax = max(kmax_of(k0), kmax_of(k1));
    }
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
// Per-warp shared-memory ring fed by bulk asynchronous copies (TMA).
//
// Each warp streams the 16-byte-aligned body of its window in kChunkBytes
// chunks through kRingStages stages; lane 0 arms the stage's mbarrier with
// the chunk's byte count and issues cp.async.bulk, all lanes wait on the
// barrier's phase parity.  Every wait is bounded: when it runs out the warp
// records TSDS_ETIMEOUT in the launch's status word, waits (again bounded)
// for its own copies still in flight and stops.
// ---------------------------------------------------------------------------
constexpr int kRingStages = 4;
constexpr int kChunkBytes = 4096;
constexpr int kWarpsPerCta = 4;
constexpr int kRingThreads = kWarpsPerCta * 32;
constexpr int kRingSmemBytes = kWarpsPerCta * kRingStages * kChunkBytes;
constexpr unsigned kWaitRounds = 1u << 22;   // try_wait rounds (each suspends briefly): seconds in total

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Bounded wait for the phase with the given parity; uniform across the warp.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  for (unsigned i = 0; i < kWaitRounds; ++i)
    if (mbar_try(b, parity)) return true;
  return false;
}

struct Ring {
  unsigned char* buf;   // kRingStages * kChunkBytes of this warp
  uint64_t* bar;        // kRingStages barriers of this warp
  uintptr_t bl, bh;     // window body [bl, bh): global, 16-byte aligned
  int64_t nchunks;      // chunks of the body
  int64_t issued;       // chunks issued so far (window-local)
  int64_t waited;       // chunks whose copy has completed and been observed
  int64_t head;         // first chunk not yet released
  uint64_t gbase;       // warp-wide count of chunks before this window (stage / parity)
  bool ok;
};

__device__ __forceinline__ int ring_stage(const Ring& R, int64_t c) { return (int)((R.gbase + (uint64_t)c) % kRingStages); }
__device__ __forceinline__ uint32_t ring_parity(const Ring& R, int64_t c) {
  return (uint32_t)(((R.gbase + (uint64_t)c) / kRingStages) & 1u);
}

__device__ __forceinline__ void ring_issue(Ring& R, int64_t c, int lane) {
  if (lane == 0) {
    const uintptr_t src = R.bl + (uintptr_t)c * kChunkBytes;
    const uint32_t bytes = (uint32_t)min((uintptr_t)kChunkBytes, R.bh - src);
    const int s = ring_stage(R, c);
    mbar_expect_tx(&R.bar[s], bytes);
    bulk_g2s(R.buf + (size_t)s * kChunkBytes, reinterpret_cast<const void*>(src), bytes, &R.bar[s]);
  }
}

__device__ __forceinline__ void ring_begin(Ring& R, uintptr_t bl, uintptr_t bh, int lane) {
  R.bl = bl;
  R.bh = bh;
  R.nchunks = bh > bl ? (int64_t)((bh - bl + kChunkBytes - 1) / kChunkBytes) : 0;
  R.issued = min((int64_t)kRingStages, R.nchunks);
  R.waited = 0;
  R.head = 0;
  for (int64_t c = 0; c < R.issued; ++c) ring_issue(R, c, lane);
}

// Makes chunk c resident.  The chunks before it are released first (each is
// observed complete before its stage is refilled with the chunk kRingStages
// ahead), then chunk c is waited for.  Invariant: head <= waited <= issued,
// and only issued chunks are ever waited for.
__device__ __forceinline__ void ring_ensure(Ring& R, int64_t c, int lane) {
  while (R.head < c && R.ok) {
    while (R.waited <= R.head && R.ok) {
      R.ok = mbar_wait(&R.bar[ring_stage(R, R.waited)], ring_parity(R, R.waited));
      if (R.ok) ++R.waited;
    }
    if (!R.ok) break;
    __syncwarp();   // every lane is done reading chunk `head`
    if (R.issued < R.nchunks) {
      if (lane == 0) fence_proxy_async();
      ring_issue(R, R.issued, lane);
      ++R.issued;
    }
    ++R.head;
  }
  while (R.waited <= c && R.ok) {
    R.ok = mbar_wait(&R.bar[ring_stage(R, R.waited)], ring_parity(R, R.waited));
    if (R.ok) ++R.waited;
  }
}

// Observes every issued chunk so the barriers' phases stay in step for the
// next window (bounded like every wait).
__device__ __forceinline__ void ring_end(Ring& R) {
  while (R.waited < R.issued && R.ok) {
    R.ok = mbar_wait(&R.bar[ring_stage(R, R.waited)], ring_parity(R, R.waited));
    if (R.ok) ++R.waited;
  }
  // issue the remaining chunks only if the pieces never reached them (cannot happen when
  // the pieces cover the body); keep the phase count consistent either way
  R.gbase += (uint64_t)R.issued;
}

// ---------------------------------------------------------------------------
// Reduction of one sub-range [s0, s1) (global addresses) of a resident chunk.
// ---------------------------------------------------------------------------
template <class P>
__device__ __forceinline__ typename P::T smem_elem(const unsigned char* p) {
  using T = typename P::T;
  if constexpr (sizeof(T) == 2 && std::is_same<T, __half>::value) {
    return __ushort_as_half(*reinterpret_cast<const unsigned short*>(p));
  } else {
    return *reinterpret_cast<const T*>(p);
  }
}

template <class P, bool MIN>
__device__ __noinline__ int find_first_smem(const uint4* __restrict__ sp, int nvec, int t, int lane,
                                            typename P::Acc target) {
  using T = typename P::T;
  const int vb = t * (32 * kU) + lane;
#pragma unroll 1
  for (int u = 0; u < kU; ++u) {
    const int vi = vb + u * 32;
    if (vi >= nvec) break;
    const uint4 v = sp[vi];
#pragma unroll
    for (int e = 0; e < P::E; ++e) {
      const T val = vec_elem<T, P::E>(v, e);
      if (MIN ? P::match_min(val, target) : P::match_max(val, target)) return vi * P::E + e;
    }
  }
  return -1;
}

// A lane's running extremum over the whole vectors of a piece, in the
// policy's value space; its index is found (in the resident chunk) only when
// a chunk strictly improves it.
template <class P>
struct LaneRun {
  bool valid;
  typename P::Acc mn, mx;
  int64_t imn, imx;
};

template <class P>
__device__ __forceinline__ void sub_reduce(LaneRun<P>& r, Cand& c, const unsigned char* chunk, uintptr_t cs,
                                           uintptr_t s0, uintptr_t s1, uintptr_t ya, int lane) {
  using T = typename P::T;
  using Acc = typename P::Acc;
  constexpr int S = sizeof(T);
  const uintptr_t v0 = (s0 + 15) & ~(uintptr_t)15, v1 = s1 & ~(uintptr_t)15;
  // elements outside whole vectors, one per lane
  if (v0 >= v1) {
    for (uintptr_t a = s0 + (uintptr_t)lane * S; a < s1; a += 32 * S) {
      const T e = smem_elem<P>(chunk + (a - cs));
      const int64_t i = (int64_t)((a - ya) / S);
      cand_merge_min(c, P::elem_key_min(e), i);
      cand_merge_max(c, P::elem_key_max(e), i);
    }
    return;
  }
  for (uintptr_t a = s0 + (uintptr_t)lane * S; a < v0; a += 32 * S) {
    const T e = smem_elem<P>(chunk + (a - cs));
    const int64_t i = (int64_t)((a - ya) / S);
    cand_merge_min(c, P::elem_key_min(e), i);
    cand_merge_max(c, P::elem_key_max(e), i);
  }
  for (uintptr_t a = v1 + (uintptr_t)lane * S; a < s1; a += 32 * S) {
    const T e = smem_elem<P>(chunk + (a - cs));
    const int64_t i = (int64_t)((a - ya) / S);
    cand_merge_min(c, P::elem_key_min(e), i);
    cand_merge_max(c, P::elem_key_max(e), i);
  }
  const uint4* __restrict__ sp = reinterpret_cast<const uint4*>(chunk + (v0 - cs));
  const int nv = (int)((v1 - v0) / 16);
  const int iters = (nv + 32 * kU - 1) / (32 * kU);
  bool cvalid = false;
  Acc cmin{}, cmax{};
  int tmin = 0, tmax = 0;
  for (int t = 0; t < iters; ++t) {
    const int vb = t * (32 * kU) + lane;
    if (vb >= nv) continue;
    uint4 v[kU];
    v[0] = sp[vb];
#pragma unroll
    for (int u = 1; u < kU; ++u) v[u] = (vb + u * 32 < nv) ? sp[vb + u * 32] : v[0];
    Acc gmin, gmax;
    P::group(v, gmin, gmax);
    if (!cvalid || P::better_min(gmin, cmin)) { cmin = gmin; tmin = t; }
    if (!cvalid || P::better_max(gmax, cmax)) { cmax = gmax; tmax = t; }
    cvalid = true;
  }
  if (cvalid) {
    const int64_t i0 = (int64_t)((v0 - ya) / S);
    // chunks are visited in index order, so a strict improvement is needed to move
    if (!r.valid || P::better_min(cmin, r.mn)) {
      r.mn = cmin;
      r.imn = i0 + find_first_smem<P, true>(sp, nv, tmin, lane, cmin);
    }
    if (!r.valid || P::better_max(cmax, r.mx)) {
      r.mx = cmax;
      r.imx = i0 + find_first_smem<P, false>(sp, nv, tmax, lane, cmax);
    }
    r.valid = true;
  }
}

// One bin piece [pa, pb) of the warp's window: elements outside the ring's body
// come from global memory, the body from the resident chunks.
template <class P>
__device__ __forceinline__ Cand piece_ring(Ring& R, const typename P::T* __restrict__ y, int64_t pa, int64_t pb,
                                           int lane) {
  using T = typename P::T;
  constexpr int S = sizeof(T);
  Cand c;
  cand_init(c);
  const uintptr_t ya = reinterpret_cast<uintptr_t>(y);
  const uintptr_t a0 = ya + (uintptr_t)pa * S, a1 = ya + (uintptr_t)pb * S;
  // before / after the body (array ends that are not 16-byte aligned)
  for (uintptr_t a = a0 + (uintptr_t)lane * S; a < min(a1, R.bl); a += 32 * S) {
    const int64_t i = (int64_t)((a - ya) / S);
    const T e = ldg_elem<T>(y + i);
    cand_merge_min(c, P::elem_key_min(e), i);
    cand_merge_max(c, P::elem_key_max(e), i);
  }
  for (uintptr_t a = max(a0, R.bh) + (uintptr_t)lane * S; a < a1; a += 32 * S) {
    const int64_t i = (int64_t)((a - ya) / S);
    const T e = ldg_elem<T>(y + i);
    cand_merge_min(c, P::elem_key_min(e), i);
    cand_merge_max(c, P::elem_key_max(e), i);
  }
  uintptr_t b0 = max(a0, R.bl);
  const uintptr_t b1 = min(a1, R.bh);
  LaneRun<P> r;
  r.valid = false;
  r.imn = r.imx = kIdxNone;
  while (b0 < b1 && R.ok) {
    const int64_t ci = (int64_t)((b0 - R.bl) / kChunkBytes);
    ring_ensure(R, ci, lane);
    if (!R.ok) break;
    const uintptr_t cs = R.bl + (uintptr_t)ci * kChunkBytes;
    const uintptr_t ce = min(cs + (uintptr_t)kChunkBytes, R.bh);
    const uintptr_t e = min(b1, ce);
    sub_reduce<P>(r, c, R.buf + (size_t)ring_stage(R, ci) * kChunkBytes, cs, b0, e, ya, lane);
    b0 = e;
  }
  if (r.valid) {
    cand_merge_min(c, P::key_min(r.mn), r.imn);
    cand_merge_max(c, P::key_max(r.mx), r.imx);
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

// The warp's reduction c of bin b = [lo, hi) over its part in window k: a bin
// inside one window is written at once; otherwise the part goes to the
// window's piece slot (the bin's first window uses last_piece, every later one
// first_piece) and the warp whose increment completes the bin's piece count
// combines all of them.  Warp-collective: every lane calls it with the same
// arguments.
template <class P, int NM>
__device__ __forceinline__ void bin_result(const SeriesDev& S, int64_t b, int64_t lo, int64_t hi, int64_t k,
                                           int64_t welems, Cand c, Piece* __restrict__ first_piece,
                                           Piece* __restrict__ last_piece, int lane) {
  const int64_t k0 = lo / welems, k1 = (hi - 1) / welems;
  if (k0 == k1) {
    finish_bin<P, NM>(c, lo);
    if (lane == 0) { S.res[2 * b] = c.imin; S.res[2 * b + 1] = c.imax; }
    return;
  }
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

template <class P, int NM, bool MULTI>
__global__ void __launch_bounds__(kRingThreads)
k_argminmax(const SeriesDev* __restrict__ sd, SeriesDev single, const int32_t* __restrict__ win_series,
            int64_t total_windows, Piece* __restrict__ first_piece, Piece* __restrict__ last_piece,
            WorkCounters* __restrict__ work, int64_t welems, const int64_t* __restrict__ total_dev,
            int64_t w_first, const int64_t* __restrict__ first_dev) {
  using T = typename P::T;
  extern __shared__ __align__(128) unsigned char ring_smem[];
  __shared__ __align__(8) uint64_t bars[kWarpsPerCta][kRingStages];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (total_dev) total_windows = *total_dev;
  if (first_dev) w_first = *first_dev;
  Ring R;
  R.buf = ring_smem + (size_t)warp * kRingStages * kChunkBytes;
  R.bar = bars[warp];
  R.gbase = 0;
  R.ok = true;
  if (lane == 0) {
    for (int s = 0; s < kRingStages; ++s) mbar_init(&R.bar[s], 1);
    fence_mbar_init();
  }
  __syncwarp();
  for (;;) {
    unsigned long long wu = 0;
    if (lane == 0) wu = atomicAdd(&work->next_window, 1ull);
    const int64_t w = w_first + (int64_t)__shfl_sync(0xffffffffu, wu, 0);
    if (w >= total_windows) break;
    const SeriesDev S = MULTI ? sd[win_series[w]] : single;
    const T* __restrict__ y = static_cast<const T*>(S.y);
    const int64_t* __restrict__ edges = S.edges;
    const int64_t nb = S.nb;
    const int64_t k = w - S.win_base;
    const int64_t ws = k * welems;
    const int64_t we = min(ws + welems, S.n);
    // the window's body: 16-byte aligned and inside the array
    const uintptr_t ya = reinterpret_cast<uintptr_t>(y);
    uintptr_t bl = max((ya + (uintptr_t)ws * sizeof(T)) & ~(uintptr_t)15, (ya + 15) & ~(uintptr_t)15);
    uintptr_t bh = min((ya + (uintptr_t)we * sizeof(T) + 15) & ~(uintptr_t)15,
                       (ya + (uintptr_t)S.n * sizeof(T)) & ~(uintptr_t)15);
    if (bh < bl) bh = bl;
    ring_begin(R, bl, bh, lane);
    // the bin holding ws: the last b with edges[b] <= ws
    int64_t b = warp_lower_bound(1, nb + 1, [&](int64_t j) { return __ldg(edges + j) > ws; }) - 1;
    int64_t lo = __ldg(edges + b);
    while (b < nb && lo < we && R.ok) {
      // the ends of the next 32 bins, one per lane
      const int64_t my_hi = (b + lane < nb) ? __ldg(edges + b + 1 + lane) : INT64_MAX;
      for (int q = 0; q < 32 && b < nb && lo < we && R.ok; ++q, ++b) {
        const int64_t hi = __shfl_sync(0xffffffffu, my_hi, q);
        if (hi > lo) {
          const int64_t pa = max(lo, ws), pb = min(hi, we);
          Cand c = piece_ring<P>(R, y, pa, pb, lane);
          bin_result<P, NM>(S, b, lo, hi, k, welems, c, first_piece, last_piece, lane);
        }
        lo = hi;
      }
    }
    ring_end(R);
    if (!R.ok) break;
  }
  if (!R.ok && lane == 0) atomicExch(&work->status, (unsigned long long)TSDS_ETIMEOUT);
}

// A wait nothing will satisfy, bounded by `rounds`: exercises the timeout
// path of the barrier waits without touching memory copies.
__global__ void k_wait_probe(unsigned long long* status, unsigned rounds) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  bool ok = false;
  for (unsigned i = 0; i < rounds && !ok; ++i) ok = mbar_try(&bar, 0);
  __syncthreads();
  if (threadIdx.x == 0) *status = ok ? 0ull : (unsigned long long)TSDS_ETIMEOUT;
}

cudaError_t launch_wait_probe(unsigned long long* status, unsigned rounds, cudaStream_t st) {
  note_launch();
  k_wait_probe<<<1, 32, 0, st>>>(status, rounds);
  return cudaGetLastError();
}

#include "stream_ldg.cuh"
#include "stream_seg.cuh"
#include "stream_grp.cuh"

typedef unsigned __int128 u128;
#include "stream_small.cuh"

// Resident CTAs per SM of each streaming kernel, cached per device (and
// cleared by tsds_shutdown).  The ring kernel's 64 KB of dynamic shared memory
// is opted into here, once per device, with the device current.
constexpr int kOccDevices = 64;
static std::atomic<unsigned> g_occ_epoch{1};

void forget_stream_occupancy() { g_occ_epoch.fetch_add(1); }

template <class P, int NM, bool MULTI, int VAR>
static cudaError_t stream_occupancy(int* occ_out) {
  // per device: the epoch the cached value belongs to (high 32 bits) and the value
  static std::atomic<unsigned long long> cache[kOccDevices];
  int d = 0;
  cudaError_t e = cudaGetDevice(&d);
  if (e != cudaSuccess) return e;
  const unsigned epoch = g_occ_epoch.load();
  std::atomic<unsigned long long>* slot = (d >= 0 && d < kOccDevices) ? &cache[d] : nullptr;
  if (slot) {
    const unsigned long long c = slot->load();
    if ((unsigned)(c >> 32) == epoch && (int)(c & 0xffffffffu) > 0) {
      *occ_out = (int)(c & 0xffffffffu);
      return cudaSuccess;
    }
  }
  int occ = 0;
  if constexpr (VAR == STREAM_LDG) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_argminmax_ldg<P, NM, MULTI>, kStreamThreadsLdg, 0);
  } else if constexpr (VAR == STREAM_SEG) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_argminmax_seg<P, NM, MULTI>, kSegThreads, 0);
  } else {
    auto kern = k_argminmax<P, NM, MULTI>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kRingSmemBytes);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kRingThreads, kRingSmemBytes);
  }
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  // concurrent first calls compute the same value; either store is fine
  if (slot) slot->store(((unsigned long long)epoch << 32) | (unsigned)occ);
  *occ_out = occ;
  return cudaSuccess;
}

// Process-wide override of the per-launch choice (tsds_stream_variant; at
// load, TSDS_STREAM_VARIANT=ring|ldg|seg).
static std::atomic<int> g_variant{-1};

static int variant_override() {
  int v = g_variant.load(std::memory_order_relaxed);
  if (v < 0) {
    const char* e = getenv("TSDS_STREAM_VARIANT");
    const int env = (e && !strcmp(e, "ring")) ? STREAM_RING
                    : (e && !strcmp(e, "ldg")) ? STREAM_LDG
                    : (e && !strcmp(e, "seg")) ? STREAM_SEG
                    : (e && !strcmp(e, "grp")) ? STREAM_GRP
                                               : STREAM_AUTO;
    int expect = -1;
    g_variant.compare_exchange_strong(expect, env);
    v = g_variant.load(std::memory_order_relaxed);
  }
  return v;
}

int stream_variant_for(const StreamConfig& cfg, int64_t elem_bytes) {
  int v = cfg.variant != STREAM_AUTO ? cfg.variant : variant_override();
  // the lane-group pass is not windowed: a windowed launch asked for it runs the automatic choice
  if (v == STREAM_AUTO || v == STREAM_GRP)
    v = cfg.mean_bin_bytes < seg_max_bin_bytes(elem_bytes) ? STREAM_SEG : STREAM_LDG;
  return v;
}

bool grp_call(int64_t mean_bin_bytes, int64_t bytes, bool has_x) {
  const int v = variant_override();
  if (v == STREAM_GRP) return true;
  // beyond 256 MB the lane groups also win at 8-32 KB bins (with x and without)
  (void)has_x;
  const int64_t limit = bytes > kSmallMaxBytes ? kGrpAutoMaxBinBytesLarge : kGrpAutoMaxBinBytes;
  return v == STREAM_AUTO && mean_bin_bytes < limit;
}

template <class P, int NM, int VAR, bool MULTI>
static cudaError_t launch_var(const SeriesDev* s_dev, const SeriesDev& single, const int32_t* win_series,
                              int64_t total_windows, Piece* fp, Piece* lp, WorkCounters* work,
                              const StreamConfig& cfg, int sm_count, cudaStream_t st) {
  int occ = 1;
  const cudaError_t oe = stream_occupancy<P, NM, MULTI, VAR>(&occ);
  if (oe != cudaSuccess) return oe;
  const int per = (cfg.ctas_per_sm > 0 && cfg.ctas_per_sm < occ) ? cfg.ctas_per_sm : occ;
  const int threads = VAR == STREAM_LDG ? kStreamThreadsLdg : VAR == STREAM_SEG ? kSegThreads : kRingThreads;
  const int warps_per_cta = threads / 32;
  int64_t blocks = (total_windows - cfg.window_first + warps_per_cta - 1) / warps_per_cta;
  const int64_t cap = (int64_t)(sm_count > 0 ? sm_count : device_sm_count()) * per;
  if (blocks > cap || cfg.total_windows_dev) blocks = cap;
  if (blocks < 1) blocks = 1;
  const int64_t welems = cfg.window_bytes / (int64_t)sizeof(typename P::T);
  note_launch();
  if constexpr (VAR == STREAM_LDG) {
    const int prefetch = cfg.mean_bin_bytes > 0 && cfg.mean_bin_bytes < kPrefetchMaxBinBytes ? 1 : 0;
    k_argminmax_ldg<P, NM, MULTI><<<(unsigned)blocks, threads, 0, st>>>(s_dev, single, win_series, total_windows, fp,
                                                                        lp, work, welems, cfg.total_windows_dev,
                                                                        cfg.window_first, cfg.window_first_dev,
                                                                        prefetch, cfg.min_bin, cfg.large_dev);
  } else if constexpr (VAR == STREAM_SEG) {
    k_argminmax_seg<P, NM, MULTI><<<(unsigned)blocks, threads, 0, st>>>(s_dev, single, win_series, total_windows, fp,
                                                                        lp, work, welems, cfg.total_windows_dev,
                                                                        cfg.window_first, cfg.window_first_dev);
  } else {
    k_argminmax<P, NM, MULTI><<<(unsigned)blocks, threads, kRingSmemBytes, st>>>(
        s_dev, single, win_series, total_windows, fp, lp, work, welems, cfg.total_windows_dev, cfg.window_first,
        cfg.window_first_dev);
  }
  return cudaGetLastError();
}

template <class P, int NM>
static cudaError_t launch_pol(const SeriesDev* s_dev, int count, const SeriesDev& single,
                              const int32_t* win_series, int64_t total_windows, Piece* fp, Piece* lp,
                              WorkCounters* work, const StreamConfig& cfg, int sm_count, cudaStream_t st) {
  const bool multi = count > 1 || s_dev != nullptr;
  const int var = stream_variant_for(cfg, (int64_t)sizeof(typename P::T));
#define TSDS_VAR(V)                                                                                         \
  return multi ? launch_var<P, NM, V, true>(s_dev, single, win_series, total_windows, fp, lp, work, cfg,    \
                                            sm_count, st)                                                   \
               : launch_var<P, NM, V, false>(s_dev, single, win_series, total_windows, fp, lp, work, cfg,   \
                                             sm_count, st)
  if (var == STREAM_LDG) TSDS_VAR(STREAM_LDG);
  if (var == STREAM_SEG) TSDS_VAR(STREAM_SEG);
  TSDS_VAR(STREAM_RING);
#undef TSDS_VAR
}

using PolI64 = Pol64<0, 0>;
using PolU64 = Pol64<1, 0>;
using PolF64Prop = Pol64<2, TSDS_NAN_PROPAGATE>;
using PolF64Ign = Pol64<2, TSDS_NAN_IGNORE>;

static cudaError_t launch_any(const SeriesDev* s_dev, int count, const SeriesDev& single,
                              const int32_t* win_series, int64_t total_windows, Piece* first_piece,
                              Piece* last_piece, WorkCounters* work, tsds_dtype y_dtype, tsds_nan_mode nan,
                              const StreamConfig& cfg, int sm_count, cudaStream_t st) {
  if (total_windows <= cfg.window_first) return cudaSuccess;
  // the ring consumes windows in whole 4 KB chunks; every variant needs 16-byte windows
  if (cfg.window_bytes <= 0 || cfg.window_bytes % kChunkBytes != 0) return cudaErrorInvalidValue;
  const bool ign = nan == TSDS_NAN_IGNORE;
#define TSDS_LAUNCH(POL, NM) \
  launch_pol<POL, NM>(s_dev, count, single, win_series, total_windows, first_piece, last_piece, work, cfg, sm_count, st)
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

cudaError_t launch_argminmax(const SeriesDev* s_dev, int count, const SeriesDev& single,
                             const int32_t* win_series, int64_t total_windows,
                             Piece* first_piece, Piece* last_piece, WorkCounters* work,
                             tsds_dtype y_dtype, tsds_nan_mode nan, cudaStream_t st, const StreamConfig& cfg) {
  return launch_any(s_dev, count, single, win_series, total_windows, first_piece, last_piece, work, y_dtype, nan,
                    cfg, 0, st);
}

cudaError_t launch_argminmax_sm(const SeriesDev& single, int64_t total_windows, Piece* first_piece,
                                Piece* last_piece, WorkCounters* work, tsds_dtype y_dtype, tsds_nan_mode nan,
                                const StreamConfig& cfg, int sm_count, cudaStream_t st) {
  return launch_any(nullptr, 1, single, nullptr, total_windows, first_piece, last_piece, work, y_dtype, nan, cfg,
                    sm_count, st);
}

bool small_call(int64_t n, int64_t nb, tsds_dtype y_dtype, bool has_x) {
  const int64_t bytes = n * dtype_size(y_dtype);
  if (nb < 1 || bytes > kSmallMaxBinBytes * nb || variant_override() != STREAM_AUTO) return false;
  // measured on GB300 (float32): up to 256 MB a warp per bin wins from 8 KB
  // bins on (below, the lane-group pass is faster); beyond 256 MB the lane
  // groups win up to 64 KB bins and the windowed pass from there
  (void)has_x;
  if (bytes <= kSmallMaxBytes) return nb <= 4096 || bytes >= 8192 * nb;
  return false;
}

template <class P, int NM, bool MULTI>
static cudaError_t launch_grp_var(const SeriesDev* s_dev, const SeriesDev& single, const int32_t* tile_series,
                                  int64_t total_tiles, WorkCounters* work, const GrpShape& shape, cudaStream_t st,
                                  const int64_t* total_dev, int sm_count) {
  // resident CTAs per SM, cached per device like the windowed kernels' (cleared by tsds_shutdown)
  static std::atomic<unsigned long long> cache[kOccDevices];
  int d = 0;
  cudaError_t e = cudaGetDevice(&d);
  if (e != cudaSuccess) return e;
  const unsigned epoch = g_occ_epoch.load();
  std::atomic<unsigned long long>* slot = (d >= 0 && d < kOccDevices) ? &cache[d] : nullptr;
  int occ = 0;
  const unsigned long long c = slot ? slot->load() : 0ull;
  if ((unsigned)(c >> 32) == epoch && (int)(c & 0xffffffffu) > 0) {
    occ = (int)(c & 0xffffffffu);
  } else {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_argminmax_grp<P, NM, MULTI>, kGrpThreads, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    if (slot) slot->store(((unsigned long long)epoch << 32) | (unsigned)occ);
  }
  int64_t blocks = (total_tiles + kGrpThreads / 32 - 1) / (kGrpThreads / 32);
  const int64_t cap = (int64_t)(sm_count > 0 ? sm_count : device_sm_count()) * occ;
  if (blocks > cap || total_dev) blocks = cap;
  if (blocks < 1) blocks = 1;
  note_launch();
  k_argminmax_grp<P, NM, MULTI><<<(unsigned)blocks, kGrpThreads, 0, st>>>(s_dev, single, tile_series, total_tiles, work,
                                                                       shape.g_log2, shape.tile_rounds, shape.max_bin,
                                                                       total_dev);
  return cudaGetLastError();
}

cudaError_t launch_argminmax_grp(const SeriesDev* s_dev, const SeriesDev& single, const int32_t* tile_series,
                                 int64_t total_tiles, WorkCounters* work, tsds_dtype y_dtype, tsds_nan_mode nan,
                                 const GrpShape& shape, cudaStream_t st, const int64_t* total_dev, int sm_count) {
  if (total_tiles <= 0 && !total_dev) return cudaSuccess;
  if (shape.g_log2 < 0 || shape.g_log2 > 5 || shape.tile_rounds < 1 ||
      (int64_t)(32 >> shape.g_log2) * shape.tile_rounds > kGrpTileMaxBins)
    return cudaErrorInvalidValue;
  const bool ign = nan == TSDS_NAN_IGNORE;
  const bool multi = s_dev != nullptr;
#define TSDS_GRP(POL, NM)                                                                                     \
  (multi ? launch_grp_var<POL, NM, true>(s_dev, single, tile_series, total_tiles, work, shape, st, total_dev,  \
                                          sm_count)                                                           \
         : launch_grp_var<POL, NM, false>(s_dev, single, tile_series, total_tiles, work, shape, st, total_dev, \
                                           sm_count))
  switch (y_dtype) {
    case TSDS_I8: return TSDS_GRP(PolSmallInt<int8_t>, 0);
    case TSDS_U8: return TSDS_GRP(PolSmallInt<uint8_t>, 0);
    case TSDS_I16: return TSDS_GRP(PolSmallInt<int16_t>, 0);
    case TSDS_U16: return TSDS_GRP(PolSmallInt<uint16_t>, 0);
    case TSDS_I32: return TSDS_GRP(PolInt32<int32_t>, 0);
    case TSDS_U32: return TSDS_GRP(PolInt32<uint32_t>, 0);
    case TSDS_I64: return TSDS_GRP(PolI64, 0);
    case TSDS_U64: return TSDS_GRP(PolU64, 0);
    case TSDS_F16: return ign ? TSDS_GRP(PolF16<1>, 1) : TSDS_GRP(PolF16<0>, 0);
    case TSDS_F32: return ign ? TSDS_GRP(PolF32<1>, 1) : TSDS_GRP(PolF32<0>, 0);
    case TSDS_F64: return ign ? TSDS_GRP(PolF64Ign, 1) : TSDS_GRP(PolF64Prop, 0);
    default: return cudaErrorInvalidValue;
  }
#undef TSDS_GRP
}

cudaError_t launch_bins_multi(const SeriesDev* s_dev, const int32_t* cta_series, int64_t ctas, tsds_dtype y_dtype,
                              tsds_nan_mode nan, cudaStream_t st, const int64_t* ctas_dev) {
  if (ctas <= 0) return cudaSuccess;
  const bool ign = nan == TSDS_NAN_IGNORE;
#define TSDS_BINS(POL, NM) launch_bins_multi_pol<POL, NM>(s_dev, cta_series, ctas, ctas_dev, st)
  switch (y_dtype) {
    case TSDS_I8: return TSDS_BINS(PolSmallInt<int8_t>, 0);
    case TSDS_U8: return TSDS_BINS(PolSmallInt<uint8_t>, 0);
    case TSDS_I16: return TSDS_BINS(PolSmallInt<int16_t>, 0);
    case TSDS_U16: return TSDS_BINS(PolSmallInt<uint16_t>, 0);
    case TSDS_I32: return TSDS_BINS(PolInt32<int32_t>, 0);
    case TSDS_U32: return TSDS_BINS(PolInt32<uint32_t>, 0);
    case TSDS_I64: return TSDS_BINS(PolI64, 0);
    case TSDS_U64: return TSDS_BINS(PolU64, 0);
    case TSDS_F16: return ign ? TSDS_BINS(PolF16<1>, 1) : TSDS_BINS(PolF16<0>, 0);
    case TSDS_F32: return ign ? TSDS_BINS(PolF32<1>, 1) : TSDS_BINS(PolF32<0>, 0);
    case TSDS_F64: return ign ? TSDS_BINS(PolF64Ign, 1) : TSDS_BINS(PolF64Prop, 0);
    default: return cudaErrorInvalidValue;
  }
#undef TSDS_BINS
}

cudaError_t launch_small(const SeriesDev& S, tsds_dtype y_dtype, tsds_nan_mode nan, Algo algo, bool has_x,
                         unsigned* done, bool emit, cudaStream_t st) {
  const bool ign = nan == TSDS_NAN_IGNORE;
#define TSDS_SMALL(POL, NM) launch_small_pol<POL, NM>(S, algo, has_x, done, emit, st)
  switch (y_dtype) {
    case TSDS_I8: return TSDS_SMALL(PolSmallInt<int8_t>, 0);
    case TSDS_U8: return TSDS_SMALL(PolSmallInt<uint8_t>, 0);
    case TSDS_I16: return TSDS_SMALL(PolSmallInt<int16_t>, 0);
    case TSDS_U16: return TSDS_SMALL(PolSmallInt<uint16_t>, 0);
    case TSDS_I32: return TSDS_SMALL(PolInt32<int32_t>, 0);
    case TSDS_U32: return TSDS_SMALL(PolInt32<uint32_t>, 0);
    case TSDS_I64: return TSDS_SMALL(PolI64, 0);
    case TSDS_U64: return TSDS_SMALL(PolU64, 0);
    case TSDS_F16: return ign ? TSDS_SMALL(PolF16<1>, 1) : TSDS_SMALL(PolF16<0>, 0);
    case TSDS_F32: return ign ? TSDS_SMALL(PolF32<1>, 1) : TSDS_SMALL(PolF32<0>, 0);
    case TSDS_F64: return ign ? TSDS_SMALL(PolF64Ign, 1) : TSDS_SMALL(PolF64Prop, 0);
    default: return cudaErrorInvalidValue;
  }
#undef TSDS_SMALL
}

}  // namespace tsds

extern "C" int tsds_stream_variant(int variant) {
  if (variant < tsds::STREAM_AUTO || variant > tsds::STREAM_GRP) return -1;
  const int prev = tsds::variant_override();
  tsds::g_variant.store(variant, std::memory_order_relaxed);
  return prev;
}
