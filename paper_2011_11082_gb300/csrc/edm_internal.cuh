// edm_internal.cuh -- shared device helpers of the sm_103a CCM kernels.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <math_constants.h>
#include <stdint.h>

#include "edm.h"

namespace edm {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;
// Neighbour lists keep E+1 entries plus this many guard entries, so an
// uncertain order at the k-th place can be settled in FP64 without a rescan.
constexpr int kGuard = 2;
constexpr int kKmax = EDM_MAX_E + 1 + kGuard;
// Per-warp compaction buffer (candidates at or below the running threshold).
constexpr int kCandCap = 64;
// FP32 squared distances below this go through FP64 (near-duplicate points).
constexpr float kNearDup = 1e-30f;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Ascending bitonic sort of one value per lane across the warp.
__device__ __forceinline__ float warp_sort_asc(float v)
{
    const int lane = lane_id();
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            float o = __shfl_xor_sync(kFull, v, stride);
            bool up = (lane & size) == 0;
            bool lower = (lane & stride) == 0;
            v = (lower == up) ? fminf(v, o) : fmaxf(v, o);
        }
    }
    return v;
}

// Lexicographic key of a (non-negative float distance, candidate index)
// pair: the bit pattern of a non-negative float orders like the value.
__device__ __forceinline__ unsigned long long dkey(float d, int s)
{
    return ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)s;
}

// Bound on |fl32(d2) - d2| for a sum of E squared differences accumulated
// with fused multiply-adds from float inputs: (E+2) units of 2^-24 relative
// (one rounding per difference, its square is exact in the FMA, one rounding
// per accumulation), widened to E+3 for margin.
__device__ __forceinline__ float d2_err(float d, int E) { return d * (float)(E + 3) * 5.9604645e-8f; }

// Pearson rho of one (library, target) pair (Algorithm 1/2, corrcoef) from
// FP32 moment sums over its n query rows: sd = sum(p - K), sdd =
// sum((p - K)^2), sdo = sum((p - K) o) for any shift K of the predictions p
// (it cancels), so_ = sum(o), dvo = n sum(o^2) - so_^2.  The centred
// numerator n sdo - sd so_ and variance n sdd - sd^2 are single fused
// operations (the callers guarantee a well-conditioned variance: mean^2 at
// most 7x the variance, else shifted sums); the variance product and its
// normalisation of the numerator are FP64.  A side of zero variance gives
// NaN.
__device__ __forceinline__ float rho_final(float sd, float sdd, float sdo, float so_, float dvo, int nrows)
{
    const float n = (float)nrows;
    const float den_p = fmaf(n, sdd, -sd * sd);
    if (!(den_p > 0.f) || !(dvo > 0.f))
        return CUDART_NAN_F;
    const float num = fmaf(n, sdo, -sd * so_);
    return (float)((double)num * rsqrt((double)den_p * (double)dvo));
}

// Conditioning test of unshifted prediction sums (sp = sum p, spp = sum p^2):
// true when the mean is large against the spread (n spp / (n spp - sp^2)
// above 8), where n spp - sp^2 from FP32 sums loses digits; the caller then
// sums again with the predictions shifted by one row's prediction.
__device__ __forceinline__ bool moments_ill_conditioned(float sp, float spp, int nrows)
{
    const float n = (float)nrows;
    const float den_p = fmaf(n, spp, -sp * sp);
    return !(8.f * den_p > n * spp);
}

}  // namespace edm
