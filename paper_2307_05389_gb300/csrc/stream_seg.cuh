// stream_seg.cuh -- the segmented variant of the per-bin argmin/argmax pass
// (included by argminmax.cu after the policies and bin_result), for bins of a
// few bytes to about a KB.
//
// The other variants give every bin to the whole warp: a bin costs a warp
// reduction and a few dependent memory round trips, which dominate once bins
// are small.  Here the warp streams its window in sub-steps of 512 bytes, one
// 16-byte vector per lane, and the bins are handled by the lanes that hold
// them:
//  * every element becomes an (ordered key, offset in the window) pair for the
//    minimum and (key, complemented offset) for the maximum, so the smallest /
//    largest value with the earliest index wins; with 32-bit keys the pair is
//    one packed 64-bit word and one unsigned min/max decides;
//  * a sub-step without a bin boundary costs one packed group min/max per
//    lane (value space, as in the other variants); a lane looks up the
//    element index only when its extremum strictly improves, and the lanes
//    are joined when the next boundary comes;
//  * in a sub-step with boundaries, the bin starts that fall in it (from 64
//    prefetched bin starts in registers) become per-lane bit masks in shared
//    memory; each lane walks its elements, writing the bins that open and
//    close inside it directly, and a segmented warp scan joins the bins that
//    cross lanes, so no bin costs a memory round trip of its own.
// NaN rules live in the keys: NaN-propagate gives a NaN the smallest minimum
// key and the largest maximum key (the first NaN wins both), NaN-ignore the
// opposite, so an all-NaN bin selects its first index.
#pragma once

constexpr int kSegThreads = 256;   // 8 warps per CTA
constexpr int kSegWarps = kSegThreads / 32;
constexpr int kSegDepth = 8;       // sub-steps in flight per warp (4 KB)

// Per-lane asynchronous 16-byte copies global -> shared (each lane reads back
// only what it copied itself, so the lane's own group wait is the only
// synchronisation).
__device__ __forceinline__ void seg_cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void seg_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void seg_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Ordered keys of one element (minimum side, maximum side): 32-bit for
// dtypes of up to 32 bits, 64-bit for the 64-bit dtypes.
template <class T, int NM, class K>
__device__ __forceinline__ void seg_keys(T v, K& kmn, K& kmx) {
  if constexpr (std::is_same<T, double>::value) {
    const uint64_t k = f64_bits_key(f64_bits(v));
    const bool nan = raw_key_is_nan(k);
    kmn = nan ? nan_key_min<NM>() : k;
    kmx = nan ? nan_key_max<NM>() : k;
  } else if constexpr (sizeof(T) == 8) {
    kmn = kmx = std::is_signed<T>::value ? ((uint64_t)v ^ kSign64) : (uint64_t)v;
  } else if constexpr (std::is_same<T, float>::value || std::is_same<T, __half>::value) {
    float f;
    if constexpr (std::is_same<T, __half>::value) f = __half2float(v);
    else f = v;
    uint32_t b = __float_as_uint(f);
    if (b == 0x80000000u) b = 0u;   // -0 orders as +0
    const uint32_t k = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    const bool nan = (b & 0x7fffffffu) > 0x7f800000u;
    kmn = nan ? (NM == TSDS_NAN_PROPAGATE ? 0u : 0xffffffffu) : k;
    kmx = nan ? (NM == TSDS_NAN_PROPAGATE ? 0xffffffffu : 0u) : k;
  } else if constexpr (std::is_signed<T>::value) {
    kmn = kmx = (uint32_t)(int32_t)v ^ 0x80000000u;
  } else {
    kmn = kmx = (uint32_t)v;
  }
}

// A running selection (smallest key, earliest offset; largest key, earliest
// offset).  With 32-bit keys it is two packed words, mn = (key << 32 |
// offset) and mx = (key << 32 | ~offset), so one unsigned min/max decides;
// with 64-bit keys the offsets ride beside the keys.
template <int KB>
struct SegRun;

template <>
struct SegRun<4> {
  using Key = uint32_t;
  uint64_t mn, mx;
};

template <>
struct SegRun<8> {
  using Key = uint64_t;
  uint64_t kmn, kmx;
  uint32_t omn, omx;   // offset of the minimum; complemented offset of the maximum
};

__device__ __forceinline__ void seg_empty(SegRun<4>& r) {
  r.mn = ~0ull;
  r.mx = 0ull;
}
__device__ __forceinline__ void seg_empty(SegRun<8>& r) {
  r.kmn = ~0ull;
  r.omn = 0xffffffffu;
  r.kmx = 0ull;
  r.omx = 0u;
}
__device__ __forceinline__ void seg_add(SegRun<4>& r, uint32_t kmn, uint32_t kmx, uint32_t rel) {
  const uint64_t a = ((uint64_t)kmn << 32) | rel;
  const uint64_t b = ((uint64_t)kmx << 32) | (0xffffffffu - rel);
  r.mn = a < r.mn ? a : r.mn;
  r.mx = b > r.mx ? b : r.mx;
}
__device__ __forceinline__ void seg_add(SegRun<8>& r, uint64_t kmn, uint64_t kmx, uint32_t rel) {
  if (kmn < r.kmn || (kmn == r.kmn && rel < r.omn)) { r.kmn = kmn; r.omn = rel; }
  const uint32_t nrel = 0xffffffffu - rel;
  if (kmx > r.kmx || (kmx == r.kmx && nrel > r.omx)) { r.kmx = kmx; r.omx = nrel; }
}
__device__ __forceinline__ void seg_join(SegRun<4>& r, const SegRun<4>& o) {
  r.mn = o.mn < r.mn ? o.mn : r.mn;
  r.mx = o.mx > r.mx ? o.mx : r.mx;
}
__device__ __forceinline__ void seg_join(SegRun<8>& r, const SegRun<8>& o) {
  if (o.kmn < r.kmn || (o.kmn == r.kmn && o.omn < r.omn)) { r.kmn = o.kmn; r.omn = o.omn; }
  if (o.kmx > r.kmx || (o.kmx == r.kmx && o.omx > r.omx)) { r.kmx = o.kmx; r.omx = o.omx; }
}
// Shuffles of a whole run.
__device__ __forceinline__ SegRun<4> seg_shfl_xor(const SegRun<4>& r, int o) {
  SegRun<4> t;
  t.mn = __shfl_xor_sync(0xffffffffu, r.mn, o);
  t.mx = __shfl_xor_sync(0xffffffffu, r.mx, o);
  return t;
}
__device__ __forceinline__ SegRun<8> seg_shfl_xor(const SegRun<8>& r, int o) {
  SegRun<8> t;
  t.kmn = __shfl_xor_sync(0xffffffffu, r.kmn, o);
  t.kmx = __shfl_xor_sync(0xffffffffu, r.kmx, o);
  t.omn = __shfl_xor_sync(0xffffffffu, r.omn, o);
  t.omx = __shfl_xor_sync(0xffffffffu, r.omx, o);
  return t;
}
__device__ __forceinline__ SegRun<4> seg_shfl_up(const SegRun<4>& r, int d) {
  SegRun<4> t;
  t.mn = __shfl_up_sync(0xffffffffu, r.mn, d);
  t.mx = __shfl_up_sync(0xffffffffu, r.mx, d);
  return t;
}
__device__ __forceinline__ SegRun<8> seg_shfl_up(const SegRun<8>& r, int d) {
  SegRun<8> t;
  t.kmn = __shfl_up_sync(0xffffffffu, r.kmn, d);
  t.kmx = __shfl_up_sync(0xffffffffu, r.kmx, d);
  t.omn = __shfl_up_sync(0xffffffffu, r.omn, d);
  t.omx = __shfl_up_sync(0xffffffffu, r.omx, d);
  return t;
}
__device__ __forceinline__ SegRun<4> seg_shfl(const SegRun<4>& r, int src) {
  SegRun<4> t;
  t.mn = __shfl_sync(0xffffffffu, r.mn, src);
  t.mx = __shfl_sync(0xffffffffu, r.mx, src);
  return t;
}
__device__ __forceinline__ SegRun<8> seg_shfl(const SegRun<8>& r, int src) {
  SegRun<8> t;
  t.kmn = __shfl_sync(0xffffffffu, r.kmn, src);
  t.kmx = __shfl_sync(0xffffffffu, r.kmx, src);
  t.omn = __shfl_sync(0xffffffffu, r.omn, src);
  t.omx = __shfl_sync(0xffffffffu, r.omx, src);
  return t;
}
template <int KB>
__device__ __forceinline__ void seg_warp_join(SegRun<KB>& r) {
#pragma unroll
  for (int o = 16; o; o >>= 1) seg_join(r, seg_shfl_xor(r, o));
}
// As an ordered-key candidate with series indices (offsets from ws).
__device__ __forceinline__ Cand seg_cand(const SegRun<4>& r, int64_t ws) {
  Cand c;
  c.kmin = r.mn >> 32;
  c.imin = ws + (int64_t)(uint32_t)r.mn;
  c.kmax = r.mx >> 32;
  c.imax = ws + (int64_t)(0xffffffffu - (uint32_t)r.mx);
  return c;
}
__device__ __forceinline__ Cand seg_cand(const SegRun<8>& r, int64_t ws) {
  Cand c;
  c.kmin = r.kmn;
  c.imin = ws + (int64_t)r.omn;
  c.kmax = r.kmx;
  c.imax = ws + (int64_t)(0xffffffffu - r.omx);
  return c;
}
template <int KB>
__device__ __forceinline__ void seg_write(const SeriesDev& S, int64_t b, const SegRun<KB>& r, int64_t ws) {
  const Cand c = seg_cand(r, ws);
  S.res[2 * b] = c.imin;
  S.res[2 * b + 1] = c.imax;
}

// The keys of a policy's running value (the value of one element).
template <class P, int NM, class K>
__device__ __forceinline__ void seg_acc_keys(typename P::Acc a, K& kmn, K& kmx) {
  if constexpr (sizeof(typename P::T) == 8) kmn = kmx = a;   // the 64-bit policies keep ordered keys
  else if constexpr (P::kFloat) seg_keys<float, NM>((float)a, kmn, kmx);
  else seg_keys<typename P::T, NM>((typename P::T)a, kmn, kmx);
}

template <class T>
using SegRunFor = SegRun<sizeof(T) == 8 ? 8 : 4>;

// Per-lane running extremum of the full sub-steps without a bin start, kept
// in value space: one packed group reduction per vector, and the element
// index only when the lane's extremum strictly improves (the earliest
// occurrence survives).
template <class P>
struct SegLane {
  typename P::Acc vmin, vmax;
  uint32_t rmin, rmax;   // window offsets
  bool valid;
};

template <class P>
__device__ __forceinline__ void seg_lane_group(SegLane<P>& L, const uint4& v, uint32_t rel) {
  using T = typename P::T;
  constexpr int E = 16 / sizeof(T);
  typename P::Acc gmin, gmax;
  P::group1(v, gmin, gmax);
  const bool bmin = !L.valid || P::better_min(gmin, L.vmin);
  const bool bmax = !L.valid || P::better_max(gmax, L.vmax);
  if (bmin || bmax) {
    T el[E];
    memcpy(el, &v, 16);
    if (bmin) {
      int f = E - 1;
#pragma unroll
      for (int e = E - 2; e >= 0; --e)
        if (P::match_min(el[e], gmin)) f = e;
      L.vmin = gmin;
      L.rmin = rel + (uint32_t)f;
    }
    if (bmax) {
      int f = E - 1;
#pragma unroll
      for (int e = E - 2; e >= 0; --e)
        if (P::match_max(el[e], gmax)) f = e;
      L.vmax = gmax;
      L.rmax = rel + (uint32_t)f;
    }
  }
  L.valid = true;
}

// The same over four consecutive full sub-steps (v[u] is sub-step u; rel is
// the window offset of the lane's first element in sub-step 0).
template <class P>
__device__ __forceinline__ void seg_lane_group4(SegLane<P>& L, const uint4 (&v)[4], uint32_t rel) {
  using T = typename P::T;
  constexpr int E = 16 / sizeof(T);
  constexpr int SUB = 32 * E;
  typename P::Acc gmin, gmax;
  P::group(v, gmin, gmax);
  const bool bmin = !L.valid || P::better_min(gmin, L.vmin);
  const bool bmax = !L.valid || P::better_max(gmax, L.vmax);
  if (bmin || bmax) {
    int fmin = 0, fmax = 0;
#pragma unroll
    for (int u = 3; u >= 0; --u) {
      T el[E];
      memcpy(el, &v[u], 16);
#pragma unroll
      for (int e = E - 1; e >= 0; --e) {
        if (P::match_min(el[e], gmin)) fmin = u * SUB + e;
        if (P::match_max(el[e], gmax)) fmax = u * SUB + e;
      }
    }
    if (bmin) {
      L.vmin = gmin;
      L.rmin = rel + (uint32_t)fmin;
    }
    if (bmax) {
      L.vmax = gmax;
      L.rmax = rel + (uint32_t)fmax;
    }
  }
  L.valid = true;
}

__device__ __forceinline__ SegRun<4> seg_pair(uint32_t kmn, uint32_t omn, uint32_t kmx, uint32_t omx) {
  SegRun<4> r;
  r.mn = ((uint64_t)kmn << 32) | omn;
  r.mx = ((uint64_t)kmx << 32) | (0xffffffffu - omx);
  return r;
}
__device__ __forceinline__ SegRun<8> seg_pair(uint64_t kmn, uint32_t omn, uint64_t kmx, uint32_t omx) {
  SegRun<8> r;
  r.kmn = kmn;
  r.omn = omn;
  r.kmx = kmx;
  r.omx = 0xffffffffu - omx;
  return r;
}

template <class P, int NM, int KB>
__device__ __forceinline__ void seg_lane_flush(SegLane<P>& L, SegRun<KB>& acc) {
  if (L.valid) {
    typename SegRun<KB>::Key kmn, kmx, t;
    seg_acc_keys<P, NM>(L.vmin, kmn, t);
    seg_acc_keys<P, NM>(L.vmax, t, kmx);
    seg_join(acc, seg_pair(kmn, L.rmin, kmx, L.rmax));
    L.valid = false;
  }
}

// Where the window's sub-step grid lies: the 16-byte aligned start gbase
// (element position q0), the number of sub-steps, and the range [mlo, mhi)
// of sub-steps that lie wholly inside [ws, we).
struct SegGrid {
  uintptr_t gbase;
  int64_t q0, nsub, mlo, mhi, ws, we;
};

// Starts the copy of sub-step m into the lane's slot: lane `lane` takes the
// 16-byte vector (m*32 + lane) of the grid.  A vector that reaches outside
// [ws, we) (only in the window's first and last sub-steps) is assembled from
// the elements inside it with plain loads.  Commits one copy group per call,
// also past the last sub-step.
template <class T>
__device__ __forceinline__ void seg_issue(uint4* slot, const T* __restrict__ y, const SegGrid& g, int64_t m,
                                          int lane) {
  constexpr int E = 16 / sizeof(T);
  const uint4* src = reinterpret_cast<const uint4*>(g.gbase) + m * 32 + lane;
  if (m >= g.mlo && m < g.mhi) {
    seg_cp16(slot, src);
  } else if (m < g.nsub) {
    const int64_t p = g.q0 + (m * 32 + lane) * E;
    if (p >= g.ws && p + E <= g.we) {
      seg_cp16(slot, src);
    } else {
      T a[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int64_t i = p + e;
        a[e] = (i >= g.ws && i < g.we) ? ldg_elem<T>(y + i) : T();
      }
      uint4 v;
      memcpy(&v, a, 16);
      *slot = v;
    }
  }
  seg_commit();
}

// A partial sub-step (the window's first or last) with no bin start: each
// lane adds its elements in [o_lo, o_hi).
template <class T, int NM, int KB>
__device__ __forceinline__ void seg_lane_add(SegRun<KB>& acc, const uint4& v, int lane, int o_lo, int o_hi,
                                             uint32_t rel0) {
  constexpr int E = 16 / sizeof(T);
  T el[E];
  memcpy(el, &v, 16);
  const int ob = lane * E;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (ob + e >= o_lo && ob + e < o_hi) {
      typename SegRun<KB>::Key kmn, kmx;
      seg_keys<T, NM>(el[e], kmn, kmx);
      seg_add(acc, kmn, kmx, rel0 + (uint32_t)(ob + e));
    }
  }
}

template <class P, int NM, bool MULTI>
__global__ void __launch_bounds__(kSegThreads)
k_argminmax_seg(const SeriesDev* __restrict__ sd, SeriesDev single, const int32_t* __restrict__ win_series,
                int64_t total_windows, Piece* __restrict__ first_piece, Piece* __restrict__ last_piece,
                WorkCounters* __restrict__ work, int64_t welems, const int64_t* __restrict__ total_dev,
            int64_t w_first, const int64_t* __restrict__ first_dev) {
  using T = typename P::T;
  using Run = SegRunFor<T>;
  using Key = typename Run::Key;
  constexpr int E = 16 / sizeof(T);   // elements per lane per sub-step
  constexpr int SUB = 32 * E;         // elements per sub-step
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ __align__(16) uint4 s_stage[kSegWarps][kSegDepth][32];
  __shared__ uint32_t s_mask[kSegWarps][32];
  __shared__ uint8_t s_tab[kSegWarps][SUB];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* mask = s_mask[warp];
  uint8_t* tab = s_tab[warp];
  uint4* stage = &s_stage[warp][0][lane];   // slot d of this lane: stage[d * 32]
  if (total_dev) total_windows = *total_dev;
  if (first_dev) w_first = *first_dev;
  for (;;) {
    unsigned long long wu = 0;
    if (lane == 0) wu = atomicAdd(&work->next_window, 1ull);
    const int64_t w = w_first + (int64_t)__shfl_sync(FULL, wu, 0);
    if (w >= total_windows) break;
    const SeriesDev S = MULTI ? sd[win_series[w]] : single;
    const T* __restrict__ y = static_cast<const T*>(S.y);
    const int64_t* __restrict__ edges = S.edges;
    const int64_t nb = S.nb;
    const int64_t k = w - S.win_base;
    const int64_t ws = k * welems;
    const int64_t we = min(ws + welems, S.n);
    // the sub-step grid: 16-byte aligned, starting at or before ws
    const uintptr_t a_ws = reinterpret_cast<uintptr_t>(y + ws);
    SegGrid g;
    g.gbase = a_ws & ~(uintptr_t)15;
    const int64_t q0 = ws - (int64_t)((a_ws - g.gbase) / sizeof(T));
    const int64_t nsub = (we - q0 + SUB - 1) / SUB;
    g.q0 = q0;
    g.nsub = nsub;
    g.mlo = (ws - q0 + SUB - 1) / SUB;
    g.mhi = (we - q0) / SUB;
    g.ws = ws;
    g.we = we;
    // kSegDepth - 1 sub-steps in flight ahead of the one being reduced
#pragma unroll
    for (int d = 0; d < kSegDepth - 1; ++d) seg_issue<T>(stage + d * 32, y, g, d, lane);

    // the bin holding ws, and the next 64 bin starts (cur: eb..eb+31, nxt: eb+32..eb+63)
    const int64_t b0 = warp_lower_bound(1, nb + 1, [&](int64_t j) { return __ldg(edges + j) > ws; }) - 1;
    const int64_t lo0 = __ldg(edges + b0);
    int64_t eb = b0 + 1;
    int64_t cur = (eb + lane <= nb) ? __ldg(edges + eb + lane) : INT64_MAX;
    int64_t nxt = (eb + 32 + lane <= nb) ? __ldg(edges + eb + 32 + lane) : INT64_MAX;
    int ep = 0;                          // cur[ep..31] not yet passed
    int64_t cb = b0;                     // the open bin
    Run carry, acc, fpart;               // open bin before the sub-step (uniform); lanes' open-bin
    seg_empty(carry);                    // pairs since the last boundary; b0's part when it began
    seg_empty(acc);                      // before ws and closes in this window (uniform)
    seg_empty(fpart);
    SegLane<P> lane_run;
    lane_run.valid = false;
    bool adirty = false, fset = false;
    const bool b0_piece = lo0 < ws;

    // at the top of each iteration, sub-steps up to m + kSegDepth - 2 are issued
#pragma unroll 1
    for (int64_t m = 0; m < nsub; ++m) {
      {
        const int64_t qs = q0 + m * SUB;
        const int64_t ne = __shfl_sync(FULL, cur, ep);
        if (m >= g.mlo && m + 4 <= g.mhi && ne >= qs + 4 * SUB) {
          // four full sub-steps inside the open bin: one packed group reduction
          seg_wait<kSegDepth - 5>();
          uint4 v4[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) v4[u] = stage[(int)((m + u) % kSegDepth) * 32];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            seg_issue<T>(stage + (int)((m + kSegDepth - 1 + u) % kSegDepth) * 32, y, g, m + kSegDepth - 1 + u, lane);
          seg_lane_group4<P>(lane_run, v4, (uint32_t)(qs - ws) + (uint32_t)(lane * E));
          adirty = true;
          m += 3;
          continue;
        }
        seg_wait<kSegDepth - 2>();
        const uint4 cv = stage[(int)(m % kSegDepth) * 32];
        seg_issue<T>(stage + (int)((m + kSegDepth - 1) % kSegDepth) * 32, y, g, m + kSegDepth - 1, lane);
        const int64_t s_hi = min(qs + SUB, we);
        const int o_lo = (int)(max(qs, ws) - qs), o_hi = (int)(s_hi - qs);
        const uint32_t rel0 = (uint32_t)(qs - ws);   // offsets wrap back into range for valid elements
        if (ne >= s_hi) {
          if (o_lo == 0 && o_hi == SUB) seg_lane_group<P>(lane_run, cv, rel0 + (uint32_t)(lane * E));
          else seg_lane_add<T, NM>(acc, cv, lane, o_lo, o_hi, rel0);
          adirty = true;
          continue;
        }
        if (adirty) {
          seg_lane_flush<P, NM>(lane_run, acc);
          seg_warp_join(acc);
          seg_join(carry, acc);
          seg_empty(acc);
          adirty = false;
        }
        T el[E];
        memcpy(el, &cv, 16);
        int r_lo = o_lo;
        for (;;) {
          // this pass of the loop: positions [r_lo, r_hi) and the bin starts cur[j] < qs + r_hi
          const int64_t n0 = __shfl_sync(FULL, nxt, 0);
          const int r_hi = n0 < s_hi ? (int)(n0 - qs) : o_hi;
          const bool in = lane >= ep && cur < qs + r_hi;
          const int64_t cdn = __shfl_down_sync(FULL, cur, 1);
          // of equal starts (empty bins) only the last opens a bin
          const bool last = in && (lane == 31 || cdn != cur);
          const unsigned inb = __ballot_sync(FULL, in);
          __syncwarp();
          mask[lane] = 0u;
          __syncwarp();
          // (the range check only matters for bin starts that are out of
          // order, which an unsorted x can produce)
          if (last && cur >= qs + r_lo) {
            const int pos = (int)(cur - qs);
            tab[pos] = (uint8_t)lane;
            atomicOr(&mask[pos / E], 1u << (pos % E));
          }
          __syncwarp();
          const uint32_t my = mask[lane];

          Run run, head;
          seg_empty(run);
          seg_empty(head);
          bool hv = false, ropen = false;
          int64_t rb = cb;
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int o = lane * E + e;
            if ((my >> e) & 1u) {
              if (ropen) seg_write(S, rb, run, ws);   // opened and closed in this lane
              else { head = run; hv = true; }         // closes the bin open at the lane's start
              rb = eb + tab[o];
              ropen = true;
              seg_empty(run);
            }
            if (o >= r_lo && o < r_hi) {
              Key kmn, kmx;
              seg_keys<T, NM>(el[e], kmn, kmx);
              seg_add(run, kmn, kmx, rel0 + (uint32_t)o);
            }
          }

          // segmented inclusive scan of the lanes' open runs (a lane that
          // opened a bin starts a segment; lane 0 continues the carry)
          Run sc = run;
          int64_t sb = ropen ? rb : cb;
          bool f = ropen;
          if (lane == 0 && !f) {
            seg_join(sc, carry);
            f = true;
          }
#pragma unroll
          for (int d = 1; d < 32; d <<= 1) {
            const Run o = seg_shfl_up(sc, d);
            const int64_t ob = __shfl_up_sync(FULL, sb, d);
            const int of = __shfl_up_sync(FULL, (int)f, d);
            if (lane >= d) {
              if (!f) {
                seg_join(sc, o);
                sb = ob;
              }
              f = f || of;
            }
          }
          // a lane's head joins everything before it in its bin
          Run pv = seg_shfl_up(sc, 1);
          int64_t pb = __shfl_up_sync(FULL, sb, 1);
          if (lane == 0) {
            pv = carry;
            pb = cb;
          }
          bool is_first = false;
          if (hv) {
            seg_join(head, pv);
            if (pb == b0 && b0_piece) is_first = true;
            else seg_write(S, pb, head, ws);
          }
          const unsigned fb = __ballot_sync(FULL, is_first);
          if (fb) {
            const int src = __ffs(fb) - 1;
            fpart = seg_shfl(head, src);
            fset = true;
          }
          carry = seg_shfl(sc, 31);
          cb = __shfl_sync(FULL, sb, 31);

          if (r_hi < o_hi) {
            // every start in cur is passed (those equal to nxt[0] open empty bins)
            cur = nxt;
            eb += 32;
            nxt = (eb + 32 + lane <= nb) ? __ldg(edges + eb + 32 + lane) : INT64_MAX;
            ep = 0;
            r_lo = r_hi;
            continue;
          }
          ep += __popc(inb);
          if (ep >= 32) {
            cur = nxt;
            eb += 32;
            nxt = (eb + 32 + lane <= nb) ? __ldg(edges + eb + 32 + lane) : INT64_MAX;
            ep = 0;
          }
          break;
        }
      }
    }
    if (adirty) {
      seg_lane_flush<P, NM>(lane_run, acc);
      seg_warp_join(acc);
      seg_join(carry, acc);
    }
    // the bin open at the window's end, then b0 if it began before ws and closed here
    bin_result<P, NM>(S, cb, __ldg(edges + cb), __ldg(edges + cb + 1), k, welems, seg_cand(carry, ws), first_piece,
                      last_piece, lane);
    if (fset)
      bin_result<P, NM>(S, b0, lo0, __ldg(edges + b0 + 1), k, welems, seg_cand(fpart, ws), first_piece, last_piece,
                        lane);
  }
}
