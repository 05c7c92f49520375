// device.cuh -- device helpers shared by the kernels: ordered keys for the
// (value, index) comparisons, candidate combines and warp searches.
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

#include "internal.h"

namespace tsds {

constexpr uint64_t kKeyMax = ~0ull;
constexpr int64_t kIdxNone = INT64_MAX;
constexpr uint64_t kSign64 = 1ull << 63;

// ---------------------------------------------------------------------------
// Ordered 64-bit keys.  Every element maps to an unsigned key whose order is
// the order the selections use (Section 2.1: smallest / largest value, the
// earliest index on ties), so partial results of any dtype combine with one
// unsigned comparison plus an index tie-break.
//
//   signed ints : sign-extend, flip the top bit (two's complement order).
//   unsigned    : the value.
//   floats      : the value widened exactly to binary64; non-negative values
//                 get the top bit set, negative values are negated as
//                 integers, which maps -0 and +0 to the same key and keeps
//                 every finite value and both infinities strictly inside
//                 (0, 2^64-1).  NaN takes an end key chosen by the NaN mode:
//                 propagate puts it below everything for argmin and above
//                 everything for argmax (the first NaN wins both); ignore does
//                 the opposite (it never wins unless the bin is all NaN).
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint64_t f64_bits_key(uint64_t b) {
  return (b & kSign64) ? (0ull - b) : (b | kSign64);
}
// Keys of +inf and -inf: raw keys beyond them are NaNs.
constexpr uint64_t kKeyPosInf = 0xFFF0000000000000ull;
constexpr uint64_t kKeyNegInf = 0x0010000000000000ull;

__device__ __forceinline__ bool raw_key_is_nan(uint64_t k) { return k > kKeyPosInf || k < kKeyNegInf; }

template <int NAN_MODE>
__device__ __forceinline__ uint64_t nan_key_min() { return NAN_MODE == TSDS_NAN_PROPAGATE ? 0ull : kKeyMax; }
template <int NAN_MODE>
__device__ __forceinline__ uint64_t nan_key_max() { return NAN_MODE == TSDS_NAN_PROPAGATE ? kKeyMax : 0ull; }

// The bits of a binary64 value as an integer.  The move goes through inline
// PTX so that the integer operations applied to the bits afterwards stay
// integer operations: when the compiler saw the sign-bit OR of a
// reinterpreted double it could carry it out as a floating-point sign
// operation, which leaves a NaN untouched and broke the NaN keys.
__device__ __forceinline__ uint64_t f64_bits(double d) {
  uint64_t b;
  asm("mov.b64 %0, %1;" : "=l"(b) : "d"(d));
  return b;
}

template <int NAN_MODE>
__device__ __forceinline__ uint64_t fkey_min(double d) {
  if (isnan(d)) return nan_key_min<NAN_MODE>();
  return f64_bits_key(f64_bits(d));
}
template <int NAN_MODE>
__device__ __forceinline__ uint64_t fkey_max(double d) {
  if (isnan(d)) return nan_key_max<NAN_MODE>();
  return f64_bits_key(f64_bits(d));
}

// The same order for float32 (and float16 widened to float32) straight from
// its bits, with integer operations only: -0 as +0, negative values below
// positive ones, NaN as in fkey_*.  Finite keys lie strictly between 0 and
// kKeyMax, like the binary64 ones.
__device__ __forceinline__ uint64_t f32_bits_key(uint32_t b) {
  if (b == 0x80000000u) b = 0u;
  return (b & 0x80000000u) ? (uint64_t)(~b) : (uint64_t)(b | 0x80000000u);
}
template <int NAN_MODE>
__device__ __forceinline__ uint64_t f32key_min(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x7fffffffu) > 0x7f800000u ? nan_key_min<NAN_MODE>() : f32_bits_key(b);
}
template <int NAN_MODE>
__device__ __forceinline__ uint64_t f32key_max(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x7fffffffu) > 0x7f800000u ? nan_key_max<NAN_MODE>() : f32_bits_key(b);
}

__device__ __forceinline__ uint64_t skey(int64_t v) { return (uint64_t)v ^ kSign64; }
__device__ __forceinline__ uint64_t ukey(uint64_t v) { return v; }

// ---------------------------------------------------------------------------
// Candidates: (key, index) for the minimum and the maximum.  The identity
// element is (max key, no index) for the minimum and (0, no index) for the
// maximum, so an empty lane never wins.
// ---------------------------------------------------------------------------
struct Cand {
  uint64_t kmin;
  int64_t imin;
  uint64_t kmax;
  int64_t imax;
};

__device__ __forceinline__ void cand_init(Cand& c) {
  c.kmin = kKeyMax; c.imin = kIdxNone; c.kmax = 0; c.imax = kIdxNone;
}
__device__ __forceinline__ void cand_merge_min(Cand& c, uint64_t k, int64_t i) {
  if (k < c.kmin || (k == c.kmin && i < c.imin)) { c.kmin = k; c.imin = i; }
}
__device__ __forceinline__ void cand_merge_max(Cand& c, uint64_t k, int64_t i) {
  if (k > c.kmax || (k == c.kmax && i < c.imax)) { c.kmax = k; c.imax = i; }
}
__device__ __forceinline__ void cand_merge(Cand& c, const Cand& o) {
  cand_merge_min(c, o.kmin, o.imin);
  cand_merge_max(c, o.kmax, o.imax);
}
__device__ __forceinline__ void cand_warp_reduce(Cand& c) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    Cand t;
    t.kmin = __shfl_xor_sync(0xffffffffu, c.kmin, o);
    t.imin = __shfl_xor_sync(0xffffffffu, c.imin, o);
    t.kmax = __shfl_xor_sync(0xffffffffu, c.kmax, o);
    t.imax = __shfl_xor_sync(0xffffffffu, c.imax, o);
    cand_merge(c, t);
  }
}

// ---------------------------------------------------------------------------
// Warp-cooperative search: the first j in [lo, hi) with pred(j) true, for a
// predicate that is false then true along j; hi when none.  Each round the
// 32 lanes probe 32 evenly spaced positions, so a range of n shrinks to one
// in about log32(n) dependent rounds.  All lanes return the same value.
// ---------------------------------------------------------------------------
template <class Pred>
__device__ __forceinline__ int64_t warp_lower_bound(int64_t lo, int64_t hi, Pred pred) {
  const int lane = threadIdx.x & 31;
  while (lo < hi) {
    int64_t len = hi - lo;
    int64_t step = (len + 31) / 32;      // probes lo, lo+step, ... cover [lo, hi)
    int64_t q = lo + (int64_t)lane * step;
    bool valid = q < hi;
    bool p = valid && pred(q);
    unsigned m = __ballot_sync(0xffffffffu, p);
    unsigned vm = __ballot_sync(0xffffffffu, valid);
    if (m == 0) {
      // everything probed is false: answer is after the last probe
      int last = 31 - __clz(vm);
      lo = lo + (int64_t)last * step + 1;
    } else {
      int f = __ffs(m) - 1;
      int64_t qf = lo + (int64_t)f * step;
      if (f == 0) return qf;             // pred(lo) holds
      // answer in (q_{f-1}, q_f]
      lo = lo + (int64_t)(f - 1) * step + 1;
      hi = qf;
      if (step == 1) return qf;
      // pred(hi) is known true: search [lo, hi) and fall back to hi
    }
  }
  return hi;
}

// The same search with GL lanes per query (a warp serves 32/GL searches at
// once), whose first round probes the window [a, b) around a guess instead of
// all of [lo, hi).  Every lane of the warp calls it; lanes of groups without a
// search pass act = false.  Rounds go on until every group is done, so the
// warp stays converged and the probes of all groups of a round are in flight
// together.  Invariant: pred is false on [.., lo), the answer lies in
// [lo, hi], and pred(hi) is true or hi is the end.  Returns the answer on
// every lane of the group (hi for a group that has no search).
template <int GL, class Pred>
__device__ __forceinline__ int64_t group_lower_bound(int64_t lo, int64_t hi, int64_t a, int64_t b, bool act,
                                                     Pred pred) {
  static_assert(GL >= 2 && GL <= 32 && (GL & (GL - 1)) == 0, "a power-of-two group");
  const int lane = threadIdx.x & 31, sl = lane & (GL - 1);
  const unsigned shift = (unsigned)(lane / GL * GL);
  const unsigned gm = GL == 32 ? 0xffffffffu : ((1u << GL) - 1u);
  a = a < lo ? lo : a;
  b = b > hi ? hi : b;
  bool first = a < b;
  bool done = !act || lo >= hi;
  while (__any_sync(0xffffffffu, !done)) {
    const int64_t s = first ? a : lo, e = first ? b : hi;
    const int64_t step = (e - s + GL - 1) / GL;
    const int64_t q = s + (int64_t)sl * step;
    const bool valid = !done && q < e;
    const bool p = valid && pred(q);
    const unsigned m = (__ballot_sync(0xffffffffu, p) >> shift) & gm;
    const unsigned vm = (__ballot_sync(0xffffffffu, valid) >> shift) & gm;
    if (!done) {
      if (m == 0) {
        // every probe false: so is everything up to the last one
        lo = s + (int64_t)(31 - __clz(vm)) * step + 1;
      } else {
        const int f = __ffs(m) - 1;
        const int64_t qf = s + (int64_t)f * step;
        if (f == 0) {
          if (s == lo) { lo = qf; hi = qf; }   // pred(lo) holds: lo is the answer
          else hi = qf;                        // the window started past the answer
        } else {
          lo = s + (int64_t)(f - 1) * step + 1;
          hi = qf;
        }
      }
      if (lo >= hi) done = true;
    }
    first = false;
  }
  return hi;
}

// floor(a*b/c) and ceil(a*b/c) for non-negative a, b and positive c with a*b
// below 2^127: one 64-bit division when a and b are below 2^32 (the product
// then fits 64 bits), the 128-bit one otherwise.
__device__ __forceinline__ uint64_t muldiv_floor(uint64_t a, uint64_t b, uint64_t c) {
  if (((a | b) >> 32) == 0) return (a * b) / c;
  return (uint64_t)(((unsigned __int128)a * b) / c);
}
__device__ __forceinline__ uint64_t muldiv_ceil(uint64_t a, uint64_t b, uint64_t c) {
  if (((a | b) >> 32) == 0) {
    const uint64_t p = a * b;
    return p / c + (p % c != 0 ? 1 : 0);
  }
  return (uint64_t)(((unsigned __int128)a * b + c - 1) / c);
}

// Fused value gather -------------------------------------------------------
// dst[pos] = src[idx] for raw elements of `size` bytes (1, 2, 4 or 8).
__device__ __forceinline__ void gather_elem(void* dst, int64_t pos, const void* src, int64_t idx, int size) {
  switch (size) {
    case 1: static_cast<uint8_t*>(dst)[pos] = static_cast<const uint8_t*>(src)[idx]; break;
    case 2: static_cast<uint16_t*>(dst)[pos] = static_cast<const uint16_t*>(src)[idx]; break;
    case 4: static_cast<uint32_t*>(dst)[pos] = static_cast<const uint32_t*>(src)[idx]; break;
    default: static_cast<uint64_t*>(dst)[pos] = static_cast<const uint64_t*>(src)[idx]; break;
  }
}

__device__ __forceinline__ void gather_point(const Gather& g, int64_t pos, const void* y, const void* x, int64_t idx) {
  if (g.y_out) gather_elem(g.y_out, pos, y, idx, g.y_size);
  if (g.x_out) gather_elem(g.x_out, pos, x, idx, g.x_size);
}

// out[pos] = v + bias, with the values of point v of the series beside it.
__device__ __forceinline__ void emit_point(const SeriesDev& S, int64_t pos, int64_t v) {
  S.out[pos] = v + S.idx_bias;
  gather_point(S.g, pos, S.y, S.x, v);
}

// Load helpers -------------------------------------------------------------
template <class T>
__device__ __forceinline__ T ldg_elem(const T* p) { return __ldg(p); }
template <>
__device__ __forceinline__ __half ldg_elem<__half>(const __half* p) {
  unsigned short s = __ldg(reinterpret_cast<const unsigned short*>(p));
  return __ushort_as_half(s);
}

__device__ __forceinline__ uint4 ldg_vec(const uint4* p) { return __ldg(p); }

}  // namespace tsds
