// lttb.h -- host entry points of the LTTB and MinMaxLTTB pipelines, and the
// job descriptors the batched server reuses.
#pragma once
#include "internal.h"

namespace tsds {

tsds_status fail(tsds_status s, const char* fmt, ...);

tsds_status run_binned_series(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                              int64_t n, int64_t nb, tsds_nan_mode nan, Algo algo, int64_t* out,
                              int64_t* out_count, int64_t idx_bias, cudaStream_t st, const Gather* g = nullptr);

// means_out (optional, device): the averages of buckets 1..B-1 as (x, y) pairs
// g (optional): values written beside the indices
tsds_status run_lttb(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype, int64_t n,
                     int64_t n_out, tsds_nan_mode nan, int64_t* out, int64_t* out_count, cudaStream_t st,
                     double* means_out = nullptr, const Gather* g = nullptr);

tsds_status run_minmaxlttb(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                           int64_t n, int64_t n_out, int64_t minmax_ratio, tsds_nan_mode nan,
                           int64_t* out, int64_t* out_count, cudaStream_t st, const Gather* g = nullptr);

// One LTTB problem over m binary64 points (see lttb.cu).
struct LttbJob {
  const double* px;      // m x values
  const double* py;      // m y values
  const int64_t* m_dev;  // number of points on the device, or null (m_host)
  int64_t m_host;
  int64_t B;             // n_out - 2
  int64_t K;             // bound on any bucket's size: ceil((m_max - 2) / B)
  int nan;
  int mode;              // 0: transition table over whole buckets (K <= kLttbTableMaxK),
                         // 2: transition table over each bucket's hull candidates
  int x_index;           // 1: px[k] == k (no x, every point kept)
  const int64_t* R;      // point -> output index (null: index + bias)
  int64_t bias;
  double2* means;        // B+1 entries
  int32_t* table;        // mode 0: B*K picks; mode 2: B*kLttbCandMax picks (relative to the bucket start)
  float2* p32;           // mode 2: m points relative to their bucket's first point, in FP32
  int32_t* cand;         // mode 2: B*kLttbCandMax candidate picks per bucket (relative, -1: none)
  int32_t* fslot;        // slot of the pick among the next step's inputs (mode 0: the table itself)
  uint8_t* chain;        // mode 2: per bucket, 1 when its mean needs the sequential sum (k_sums_wide)
  float4* box;           // mode 2: per bucket, the FP32 bounding box of each of its 32 slices
  int32_t* comp;         // per segment of 32 steps and input slot: the slot after the segment (-1: leaves the table)
  int32_t* seg_start;    // per segment: its input slot, or -1 when the chain was replayed there directly
  int64_t* out;
  int64_t* out_count;
  const void* ysrc;      // with g: the series the output indices point into
  const void* xsrc;
  Gather g;              // values written beside the indices (null pointers: none)
};

// Gathers points as binary64: px[k] = x[i] or i, py[k] = y[i], i = R[k] or k.
struct PointsJob {
  const void* x;
  int x_dtype;
  const void* y;
  int y_dtype;
  const int64_t* R;
  const int64_t* m_dev;
  int64_t m_host;
  double* px;
  double* py;
};

constexpr int kLttbTableMaxK = 32;
constexpr int kLttbCandMax = 32;

inline int lttb_mode(int64_t K) { return K <= kLttbTableMaxK ? 0 : 2; }

// Scratch bytes a job needs besides its points (means, tables, candidates),
// and the binding of those pointers into `p` (J.B, J.K set; sets J.mode).
size_t lttb_job_scratch(int64_t m_max, int64_t B, int64_t K);
void lttb_job_bind(LttbJob& J, char* p, int64_t m_max);

// Runs the LTTB kernels for jobs already filled in (device memory for their
// points and scratch in place); jobs_dev must hold a copy of jobs_host.
tsds_status run_lttb_jobs(const LttbJob* jobs_host, const LttbJob* jobs_dev, int count, int64_t max_B,
                          int64_t max_m, cudaStream_t st);

// k_points over `count` jobs in device memory.
tsds_status launch_points_jobs(const PointsJob* jobs_dev, int count, int64_t max_m, cudaStream_t st);

}  // namespace tsds
