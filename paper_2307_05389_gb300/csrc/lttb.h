// lttb.h -- host entry points of the LTTB and MinMaxLTTB pipelines.
#pragma once
#include "internal.h"

namespace tsds {

tsds_status fail(tsds_status s, const char* fmt, ...);

tsds_status run_binned_series(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                              int64_t n, int64_t nb, tsds_nan_mode nan, Algo algo, int64_t* out,
                              int64_t* out_count, int64_t idx_bias, cudaStream_t st);

tsds_status run_lttb(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype, int64_t n,
                     int64_t n_out, tsds_nan_mode nan, int64_t* out, int64_t* out_count, cudaStream_t st);

tsds_status run_minmaxlttb(const void* x, tsds_dtype x_dtype, const void* y, tsds_dtype y_dtype,
                           int64_t n, int64_t n_out, int64_t minmax_ratio, tsds_nan_mode nan,
                           int64_t* out, int64_t* out_count, cudaStream_t st);

}  // namespace tsds
