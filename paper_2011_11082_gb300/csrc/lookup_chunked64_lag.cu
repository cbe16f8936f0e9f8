// lookup_multi64_lag.cu -- the time-delay form of the chunked lookup for 64-byte tile rows (16 FP32 / 32 FP16 targets per row), for series too long for 128-byte rows.
#define EDM_RB 64
#define EDM_LAG true
#define EDM_MULTI_NAME lookup_multi64_lag_kernel
#define EDM_MULTI_LAUNCH launch_lookup_multi64_lag
#define EDM_MULTI_TIMEOUTS lookup_multi64_lag_wait_timeouts
#include "lookup_multi_impl.cuh"
