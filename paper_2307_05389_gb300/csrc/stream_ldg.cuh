// stream_ldg.cuh -- the register-streaming variant of the per-bin
// argmin/argmax pass (included by argminmax.cu after the policies).
//
// Each lane loads 4 vectors of 16 bytes per step straight into registers
// (coalesced across the warp, 2 KB per warp-step) and resolves indices every
// 8 steps from a cached re-read.  Its per-byte overhead is the smallest, so it
// is the faster variant when bins are large (tens of KB and more); the ring
// variant in argminmax.cu wins when bins are small, since there every bin
// costs one shared-memory round trip instead of one DRAM round trip.
#pragma once

constexpr int kStreamThreadsLdg = 256;   // 8 warps per CTA
constexpr int kCH = 8;                   // steps between index resolutions
constexpr int kPrefetchAhead = 8192;     // bytes of the window requested into L2 ahead of the loads
// Prefetch pays when pieces are short (each costs a few round trips of its
// own) and costs when they are long (steps already stream at the copy rate):
// on for launches whose bytes-weighted mean bin is below this.
constexpr int64_t kPrefetchMaxBinBytes = 128 * 1024;

// Requests the 2 KB of y that start kPrefetchAhead bytes past base + off into
// L2 (lane l the 64 bytes at 64 l), never at or past base + room; a hint with
// no register cost, so the loads of the next bins and steps find their lines
// in L2.
__device__ __forceinline__ void prefetch_ahead(const char* base, int off, int room, int lane) {
  const int q = off + kPrefetchAhead + 64 * lane;
  if (q < room) asm volatile("prefetch.global.L2 [%0];" ::"l"(base + q));
}

// ---------------------------------------------------------------------------
// One bin piece [a, b) of a series, reduced by one warp.
// ---------------------------------------------------------------------------
// Element offset (from the first body element) of the first element of the
// vectors v of step t that matches `target`, or -1.
template <class P, bool MIN>
__device__ __forceinline__ int find_in_step(const uint4 (&v)[kU], int nvec, int t, int lane,
                                            typename P::Acc target) {
  using T = typename P::T;
  const int vb = t * (32 * kU) + lane;
#pragma unroll
  for (int u = 0; u < kU; ++u) {
    const int vi = vb + u * 32;
    if (vi < nvec) {
#pragma unroll
      for (int e = 0; e < P::E; ++e) {
        const T val = vec_elem<T, P::E>(v[u], e);
        if (MIN ? P::match_min(val, target) : P::match_max(val, target)) return vi * P::E + e;
      }
    }
  }
  return -1;
}

// The same after re-reading step t (all of its vectors are requested before
// any is searched, so the re-read costs one round trip).
template <class P, bool MIN>
__device__ __noinline__ int find_first_g(const uint4* __restrict__ vp, int nvec, int t, int lane,
                                         typename P::Acc target) {
  const int vb = t * (32 * kU) + lane;
  uint4 v[kU];
#pragma unroll
  for (int u = 0; u < kU; ++u) v[u] = vb + u * 32 < nvec ? ldg_vec(vp + vb + u * 32) : make_uint4(0u, 0u, 0u, 0u);
  return find_in_step<P, MIN>(v, nvec, t, lane, target);
}

// A piece whose body is a single step: the head, tail and body loads are all
// issued before any is used, and the body's indices come straight from the
// registers (no re-read).  Kept out of line so that the main loop's register
// allocation does not carry it.
template <class P>
__device__ __noinline__ Cand one_step(const typename P::T* __restrict__ y, int64_t a, int64_t ia, int64_t ib,
                                      int64_t b, int lane) {
  using T = typename P::T;
  using Acc = typename P::Acc;
  const uint4* __restrict__ vp = reinterpret_cast<const uint4*>(y + ia);
  const int nv = (int)((ib - ia) / P::E);
  const bool has_h = a + lane < ia, has_t = ib + lane < b;   // fewer than 16 bytes each side
  T he{}, te{};
  if (has_h) he = ldg_elem<T>(y + a + lane);
  if (has_t) te = ldg_elem<T>(y + ib + lane);
  uint4 v[kU];
#pragma unroll
  for (int u = 0; u < kU; ++u) v[u] = lane + u * 32 < nv ? ldg_vec(vp + lane + u * 32) : make_uint4(0u, 0u, 0u, 0u);
  Cand c;
  cand_init(c);
  if (lane < nv) {
#pragma unroll
    for (int u = 1; u < kU; ++u)
      if (lane + u * 32 >= nv) v[u] = v[0];
    Acc mn, mx;
    P::group(v, mn, mx);
    cand_merge_min(c, P::key_min(mn), ia + find_in_step<P, true>(v, nv, 0, lane, mn));
    cand_merge_max(c, P::key_max(mx), ia + find_in_step<P, false>(v, nv, 0, lane, mx));
  }
  if (has_h) {
    cand_merge_min(c, P::elem_key_min(he), a + lane);
    cand_merge_max(c, P::elem_key_max(he), a + lane);
  }
  if (has_t) {
    cand_merge_min(c, P::elem_key_min(te), ib + lane);
    cand_merge_max(c, P::elem_key_max(te), ib + lane);
  }
  return c;
}

// room (optional): bytes from y + a to the end of the window holding the
// piece, which is prefetched ahead within that window (0: no prefetch)
template <class P>
__device__ __forceinline__ Cand piece_ldg(const typename P::T* __restrict__ y, int64_t a, int64_t b, int room = 0) {
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
  if (room > 0) {
    // the bytes kPrefetchAhead past this piece (the following pieces of the
    // window), at most 16 KB, requested before the piece's own loads
    const char* pbase = reinterpret_cast<const char*>(y + a);
    const int pbytes = (int)min((int64_t)16384, (b - a) * (int64_t)sizeof(T));
    for (int off = 0; off < pbytes; off += 2048) prefetch_ahead(pbase, off, room, lane);
  }
  if (nvec <= 32 * kU) {
    c = one_step<P>(y, a, ia, ib, b, lane);
    cand_warp_reduce(c);
    return c;
  }
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

  {
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
          rimin = find_first_g<P, true>(vp, nv, tmin, lane, cmin);
        }
        if (!rvalid || P::better_max(cmax, rmax)) {
          rmax = cmax;
          rimax = find_first_g<P, false>(vp, nv, tmax, lane, cmax);
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

template <class P, int NM, bool MULTI>
__global__ void __launch_bounds__(kStreamThreadsLdg, MULTI ? 3 : 4)
k_argminmax_ldg(const SeriesDev* __restrict__ sd, SeriesDev single, const int32_t* __restrict__ win_series,
            int64_t total_windows, Piece* __restrict__ first_piece, Piece* __restrict__ last_piece,
            WorkCounters* __restrict__ work, int64_t welems, const int64_t* __restrict__ total_dev,
            int64_t w_first, const int64_t* __restrict__ first_dev, int prefetch, int64_t min_bin,
            const unsigned long long* __restrict__ large_dev) {
  using T = typename P::T;
  const int lane = threadIdx.x & 31;
  // min_bin > 0: only bins of more than min_bin points (the lane-group pass
  // did the others); nothing to do when it found none
  if (large_dev && *large_dev == 0) return;
  if (total_dev) total_windows = *total_dev;
  if (first_dev) w_first = *first_dev;
  // a warp claims its next window as soon as it starts on one, so the claim's
  // round trip overlaps the work
  unsigned long long wu = 0;
  if (lane == 0) wu = atomicAdd(&work->next_window, 1ull);
  for (;;) {
    const int64_t w = w_first + (int64_t)__shfl_sync(0xffffffffu, wu, 0);
    if (w >= total_windows) break;
    if (lane == 0) wu = atomicAdd(&work->next_window, 1ull);
    SeriesDev S = MULTI ? sd[win_series[w]] : single;
    const T* __restrict__ y = static_cast<const T*>(S.y);
    const int64_t* __restrict__ edges = S.edges;
    const int64_t nb = S.nb;
    const int64_t k = w - S.win_base;
    const int64_t ws = k * welems;
    const int64_t we = min(ws + welems, S.n);
    // with prefetch (launches of small and mid-size bins): the window's first
    // lines into L2 while its first bin is searched
    if (prefetch) {
      const int wroom = (int)((we - ws) * (int64_t)sizeof(T));
#pragma unroll
      for (int q = 0; q < kPrefetchAhead / 2048; ++q)
        prefetch_ahead(reinterpret_cast<const char*>(y + ws), 2048 * q - kPrefetchAhead, wroom, lane);
    }
    // the bin holding ws: the last b with edges[b] <= ws
    int64_t b = warp_lower_bound(1, nb + 1, [&](int64_t j) { return __ldg(edges + j) > ws; }) - 1;
    int64_t lo = __ldg(edges + b);
    while (b < nb && lo < we) {
      // the ends of the next 32 bins, one per lane
      const int64_t my_hi = (b + lane < nb) ? __ldg(edges + b + 1 + lane) : INT64_MAX;
      for (int q = 0; q < 32 && b < nb && lo < we; ++q, ++b) {
        const int64_t hi = __shfl_sync(0xffffffffu, my_hi, q);
        if (hi - lo > min_bin) {
          const int64_t pa = max(lo, ws), pb = min(hi, we);
          Cand c = piece_ldg<P>(y, pa, pb, prefetch ? (int)((we - pa) * (int64_t)sizeof(T)) : 0);
          bin_result<P, NM>(S, b, lo, hi, k, welems, c, first_piece, last_piece, lane);
        }
        lo = hi;
      }
    }
  }
}
