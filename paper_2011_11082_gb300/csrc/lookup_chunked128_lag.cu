// lookup_multi128_lag.cu -- the time-delay form of the chunked lookup for 128-byte tile rows (32 FP32 / 64 FP16 targets per row).
#define EDM_RB 128
#define EDM_LAG true
#define EDM_MULTI_NAME lookup_multi128_lag_kernel
#define EDM_MULTI_LAUNCH launch_lookup_multi128_lag
#define EDM_MULTI_TIMEOUTS lookup_multi128_lag_wait_timeouts
#include "lookup_multi_impl.cuh"
