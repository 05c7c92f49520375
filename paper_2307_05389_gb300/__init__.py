"""GB300-native downsampling for line-chart visualisation: MinMax, M4, LTTB,
MinMaxLTTB and EveryNth (the algorithms of tsdownsample, arXiv 2307.05389) as hand-written
sm_103a CUDA kernels behind a C ABI (include/tsds.h).

``binding`` holds the ctypes entry points (same names as the C ABI) and the
torch-facing ``downsample`` / ``*Downsampler`` helpers; ``inputs`` draws the
seeded synthetic series used by the tests and the benchmark.
"""
from .binding import (  # noqa: F401
    DTYPES,
    EveryNthDownsampler,
    M4Downsampler,
    LTTBDownsampler,
    MinMaxDownsampler,
    MinMaxLTTBDownsampler,
    NAN_MODES,
    TsdsError,
    Plan,
    downsample,
    downsample_values,
    downsample_batched,
    downsample_host,
    tsds_batched,
    tsds_minmax_noalloc,
    tsds_plan_create,
    tsds_plan_destroy,
    tsds_plan_execute,
    tsds_plan_info,
    last_error,
    load,
    tsds_everynth,
    tsds_everynth_values,
    tsds_lttb,
    tsds_lttb_means,
    tsds_lttb_values,
    tsds_m4_values,
    tsds_minmax_values,
    tsds_minmaxlttb_values,
    tsds_m4,
    tsds_minmax,
    tsds_minmaxlttb,
    tsds_shutdown,
    tsds_version,
    tsds_kernel_launches,
    tsds_timing_enable,
    tsds_timing_read,
    tsds_read_stream,
    read_stream,
)
