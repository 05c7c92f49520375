// stream_grp.cuh -- the lane-group variant of the per-bin argmin/argmax pass
// (included by argminmax.cu after the policies and stream_seg.cuh, whose
// packed (key, offset) runs it reuses), for bins of a few bytes to tens of KB.
//
// The windowed variants give a bin to a whole warp, or walk bin boundaries
// inside a warp-wide stream; both pay a fixed cost per bin that dominates when
// bins are small.  Here a warp claims a tile of up to kGrpTileMaxBins
// consecutive whole bins, stages their starts in shared memory with one
// coalesced load, asks L2 for the tile's bytes when its bins are small, and
// splits into 32/G groups of G lanes (G a power of two chosen from the mean
// bin size), each group reducing one whole bin at a time:
//  * a bin's first and last 16-byte vector may hold elements of the
//    neighbouring bins; those are replaced by one inside the bin (which
//    changes neither extremum).  Every lane of the group starts from the
//    first vector (one broadcast load), so its running extremum is defined
//    from the start; the last vector goes to one lane;
//  * the interior vectors are dealt to the group's lanes round-robin, so every
//    load instruction reads G*16 contiguous bytes per group, and each lane
//    issues grp_unroll loads (16, or 8 for 8-byte elements) before it uses
//    any of them; the first vector is loaded together with the first round;
//  * a vector reduces to one group minimum and maximum with the policy's
//    packed instructions (value space, as in the other variants); a lane keeps
//    its running extremum and the number of the vector it came from, replacing
//    them only on a strict improvement, so the earliest occurrence survives;
//  * at the end a lane reads its winning vector again (an L1 hit) to find the
//    first matching slot inside the bin, the lanes join packed (ordered key,
//    offset) runs with log2(G) shuffle rounds, and the group's first lane
//    writes the bin's selections.
// No bin is cut, so nothing is published or merged across warps.
#pragma once

constexpr int kGrpThreads = 256;   // 8 warps per CTA
// A tile holds at most kGrpTileMaxBins bins (their starts are staged in
// shared memory) and its first kGrpPrefetchBytes are requested into L2 when
// it starts.
constexpr int64_t kGrpPrefetchBytes = 64 * 1024;
// Only tiles whose bins average less than this are requested into L2: larger
// bins give each lane enough loads in flight on their own, and there the
// requests measured 2-6 % slower.
constexpr int64_t kGrpPrefetchMaxBin = 4 * 1024;

// Replaces the elements of v outside positions [e_lo, e_hi) by element e_lo
// (which lies inside).
template <class T>
__device__ __forceinline__ uint4 grp_mask(uint4 v, int e_lo, int e_hi) {
  constexpr int E = 16 / sizeof(T);
  T el[E];
  memcpy(el, &v, 16);
  T ref = el[0];
#pragma unroll
  for (int e = 1; e < E; ++e)
    if (e == e_lo) ref = el[e];
#pragma unroll
  for (int e = 0; e < E; ++e)
    if (e < e_lo || e >= e_hi) el[e] = ref;
  memcpy(&v, el, 16);
  return v;
}

// Vector vi of the aligned grid (element i sits in vector (i + d) / E): a
// plain 16-byte load when the vector lies inside the array [0, n), else its
// in-array elements one at a time (only the array's first and last vector).
template <class T>
__device__ __forceinline__ uint4 grp_load(const uint4* __restrict__ gbase, const T* __restrict__ y, int64_t vi,
                                          int64_t d, int64_t n) {
  constexpr int E = 16 / sizeof(T);
  const int64_t p = vi * E - d;   // element index of the vector's first slot
  if (p >= 0 && p + E <= n) return ldg_vec(gbase + vi);
  T a[E];
#pragma unroll
  for (int e = 0; e < E; ++e) a[e] = (p + e >= 0 && p + e < n) ? ldg_elem<T>(y + p + e) : T();
  uint4 v;
  memcpy(&v, a, 16);
  return v;
}

// First position e in [e_lo, e_hi) of vector v whose element matches the
// running extremum t (MIN: minimum side).
template <class P, bool MIN>
__device__ __forceinline__ int grp_find(const uint4& v, int e_lo, int e_hi, typename P::Acc t) {
  using T = typename P::T;
  constexpr int E = 16 / sizeof(T);
  T el[E];
  memcpy(el, &v, 16);
  int f = e_hi - 1;
#pragma unroll
  for (int e = E - 1; e >= 0; --e)
    if (e >= e_lo && e < e_hi && (MIN ? P::match_min(el[e], t) : P::match_max(el[e], t))) f = e;
  return f;
}

// A lane's running extremum over the vectors it has taken so far (in
// increasing order) and the vector each came from; a later vector replaces it
// only when strictly better, so the earliest occurrence survives.
template <class P>
struct GrpLane {
  typename P::Acc rmin, rmax;
  uint32_t pmin, pmax;
  bool valid;
};

template <class P>
__device__ __forceinline__ void grp_take(GrpLane<P>& L, const uint4& w, uint32_t r) {
  typename P::Acc gmin, gmax;
  P::group1(w, gmin, gmax);
  if (P::better_min(gmin, L.rmin)) {
    L.rmin = gmin;
    L.pmin = r;
  }
  if (P::better_max(gmax, L.rmax)) {
    L.rmax = gmax;
    L.pmax = r;
  }
}

template <class P, int NM, bool MULTI>
__global__ void __launch_bounds__(kGrpThreads, 2)
k_argminmax_grp(const SeriesDev* __restrict__ sd, SeriesDev single, const int32_t* __restrict__ tile_series,
                int64_t total_tiles, WorkCounters* __restrict__ work, int g_log2, int tile_rounds,
                int64_t max_bin, const int64_t* __restrict__ total_dev) {
  using T = typename P::T;
  using Acc = typename P::Acc;
  using Run = SegRunFor<T>;
  using Key = typename Run::Key;
  constexpr int E = 16 / sizeof(T);
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  __shared__ int64_t s_tile[kGrpThreads / 32][kGrpTileMaxBins + 1];
  int64_t* ts = s_tile[threadIdx.x >> 5];
  if (total_dev) total_tiles = *total_dev;
  unsigned long long tu = 0;
  if (lane == 0) tu = atomicAdd(&work->next_window, 1ull);
  for (;;) {
    const int64_t t = (int64_t)__shfl_sync(FULL, tu, 0);
    if (t >= total_tiles) break;
    if (lane == 0) tu = atomicAdd(&work->next_window, 1ull);   // the next claim overlaps this tile
    const SeriesDev S = MULTI ? sd[tile_series[t]] : single;
    // the group shape: one per launch, or per series in a batch (S.grp)
    const int lg = MULTI ? (S.grp & 0xff) : g_log2;
    const int G = 1 << lg;
    const int groups = 32 >> lg;
    const int gi = lane >> lg, gj = lane & (G - 1);
    const int64_t tile_bins = (int64_t)groups * (MULTI ? (S.grp >> 8) : tile_rounds);
    const T* __restrict__ y = static_cast<const T*>(S.y);
    const uintptr_t ya = reinterpret_cast<uintptr_t>(y);
    const uint4* __restrict__ gbase = reinterpret_cast<const uint4*>(ya & ~(uintptr_t)15);
    const int64_t d = (int64_t)((ya & 15) / sizeof(T));   // elements between the grid base and y
    const int64_t b_first = (t - S.tile_base) * tile_bins;
    const int64_t b_end = min(b_first + tile_bins, S.nb);
    // the tile's bin starts, one coalesced load into this warp's shared slots,
    // then the tile's bytes requested into L2 so that every round after the
    // first finds its lines there
    const int nts = (int)(b_end - b_first);
    __syncwarp();
    for (int j = lane; j <= nts; j += 32) ts[j] = __ldg(S.edges + b_first + j);
    __syncwarp();
    {
      const int64_t e0 = ts[0], e1 = ts[nts];
      const char* pa = reinterpret_cast<const char*>(y + e0);
      const int64_t tb = (e1 - e0) * (int64_t)sizeof(T);
      const int64_t bytes = tb < kGrpPrefetchMaxBin * nts ? min(tb, kGrpPrefetchBytes) : 0;
      for (int64_t q = 128 * (int64_t)lane; q < bytes; q += 32 * 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(pa + q));
    }
    for (int64_t bb = b_first; bb < b_end; bb += groups) {
      const int64_t b = bb + gi;
      const bool active = b < b_end;
      int64_t lo = 0, hi = 0;
      if (active) {
        lo = ts[b - b_first];
        hi = ts[b - b_first + 1];
        if (max_bin > 0 && hi - lo > max_bin) {
          // left to the windowed pass, which splits it across warps
          if (gj == 0) atomicAdd(&work->large, 1ull);
          hi = lo;
        }
      }
      // the bin's vectors on the aligned grid, numbered from its first one
      const int64_t v_lo = (lo + d) / E;
      const uint32_t nv = hi > lo ? (uint32_t)((hi - 1 + d) / E + 1 - v_lo) : 0u;
      const int e_first = (int)((lo + d) % E);           // first bin slot of vector 0
      const int e_last = (int)((hi - 1 + d) % E) + 1;    // one past the last bin slot of vector nv-1
      // a vector of the bin reaches outside the array only at the array's two ends
      const bool at_ends = v_lo * E - d < 0 || (v_lo + (int64_t)nv) * E - d > S.n;
      const uint4* __restrict__ bp = gbase + v_lo;
      // vector r of the bin (the array-end form only when a vector of the bin can reach outside)
      auto vec = [&](uint32_t r) { return at_ends ? grp_load<T>(gbase, y, v_lo + r, d, S.n) : ldg_vec(bp + r); };
      // interior vectors 1 .. nv-2 (inside the bin, so inside the array) are
      // dealt round-robin: lane gj takes 1 + gj, 1 + gj + G, ...  Every lane
      // of the group also takes vector 0 (one broadcast load; partly outside
      // the bin unless the bin starts on a vector), so no vector needs a
      // first-take test.  Vector 0 and the first round's loads are issued
      // before any of them is used; then the rounds of G*U vectors that
      // lie wholly inside the bin run without a test per load, and one
      // partial round ends the bin (the same split for every lane of the
      // group, so the group stays converged).
      const uint32_t ni = nv >= 2 ? nv - 2 : 0u;
      const uint4* __restrict__ ip = bp + 1;
      const uint32_t step = (uint32_t)G;
      constexpr int U = grp_unroll(sizeof(T));
      const uint32_t round = step * U;
      GrpLane<P> L;
      L.valid = nv > 0;
      {
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        if (L.valid) w = vec(0);
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const uint32_t q = (uint32_t)gj + step * u;
          v[u] = q < ni ? ldg_vec(ip + q) : make_uint4(0u, 0u, 0u, 0u);
        }
        if (L.valid) {
          const int e_hi = nv == 1 ? e_last : E;
          if (e_first > 0 || e_hi < E) w = grp_mask<T>(w, e_first, e_hi);
          P::group1(w, L.rmin, L.rmax);
          L.pmin = L.pmax = 0u;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const uint32_t q = (uint32_t)gj + step * u;
          if (q < ni) grp_take(L, v[u], 1u + q);
        }
      }
      uint32_t r0 = round;
      for (; r0 + round <= ni; r0 += round) {
        const uint32_t q0 = r0 + (uint32_t)gj;
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = ldg_vec(ip + q0 + step * u);
#pragma unroll
        for (int u = 0; u < U; ++u) grp_take(L, v[u], 1u + q0 + step * u);
      }
      if (r0 < ni) {
        const uint32_t q0 = r0 + (uint32_t)gj;
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const uint32_t q = q0 + step * u;
          v[u] = q < ni ? ldg_vec(ip + q) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const uint32_t q = q0 + step * u;
          if (q < ni) grp_take(L, v[u], 1u + q);
        }
      }
      // the last vector, after the interior ones of the lane it falls to
      if (nv >= 2 && (uint32_t)gj == ((nv - 2) & (uint32_t)(G - 1))) {
        uint4 w = vec(nv - 1);
        if (e_last < E) w = grp_mask<T>(w, 0, e_last);
        grp_take(L, w, nv - 1);
      }
      Run run;
      seg_empty(run);
      if (L.valid) {
        // the first bin slot of the winning vector (read again) that holds the
        // extremum; bin offset of slot e of vector r: r*E + e - e_first
        const uint4 wmin = vec(L.pmin), wmax = vec(L.pmax);
        const int fmin = grp_find<P, true>(wmin, L.pmin == 0 ? e_first : 0, L.pmin + 1 == nv ? e_last : E, L.rmin);
        const int fmax = grp_find<P, false>(wmax, L.pmax == 0 ? e_first : 0, L.pmax + 1 == nv ? e_last : E, L.rmax);
        const Acc rmin = L.rmin, rmax = L.rmax;
        const uint32_t pmin = L.pmin, pmax = L.pmax;
        Key kmn, kmx, tk;
        seg_acc_keys<P, NM>(rmin, kmn, tk);
        seg_acc_keys<P, NM>(rmax, tk, kmx);
        run = seg_pair(kmn, pmin * (uint32_t)E + (uint32_t)fmin - (uint32_t)e_first, kmx,
                       pmax * (uint32_t)E + (uint32_t)fmax - (uint32_t)e_first);
      }
      for (int o = 1; o < G; o <<= 1) seg_join(run, seg_shfl_xor(run, o));
      if (active && gj == 0 && hi > lo) {   // (hi == lo also for a bin left to the windowed pass)
        const Cand c = seg_cand(run, lo);
        S.res[2 * b] = c.imin;
        S.res[2 * b + 1] = c.imax;
      }
    }
  }
}
