// bulk_copy.cuh -- 1-D bulk copies (TMA, cp.async.bulk) from this GPU's
// global memory into the issuing CTA's shared memory, completed on an
// mbarrier (no cluster multicast).  One thread issues the copy; every
// thread waits on the barrier phase with a bounded number of polls.
//
// Rules the callers keep: source and destination 16-byte aligned, size a
// multiple of 16 bytes and below 2^20 per barrier phase (the transaction
// count limit).
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace edm {

// Waits that gave up (a completed copy never takes this long).  Each
// translation unit has its own counter; EDM_WAIT_TIMEOUT_READER(fn) defines
// the host function fn(&count, reset) that reads (and optionally clears)
// that unit's counter, and edm_wait_timeouts() sums them.
static __device__ unsigned long long g_wait_timeouts;

#define EDM_WAIT_TIMEOUT_READER(fn)                                                                                    \
    cudaError_t fn(unsigned long long *count, bool reset)                                                              \
    {                                                                                                                  \
        cudaError_t e = cudaMemcpyFromSymbol(count, g_wait_timeouts, sizeof *count);                                    \
        if (e == cudaSuccess && reset) {                                                                               \
            const unsigned long long z = 0ull;                                                                         \
            e = cudaMemcpyToSymbol(g_wait_timeouts, &z, sizeof z);                                                     \
        }                                                                                                              \
        return e;                                                                                                      \
    }

constexpr int kWaitPolls = 1 << 22;  // each try_wait may itself sleep a while

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// Copy `bytes` from global `src` to shared `dst`; completes on mbar.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

// Bring `bytes` of global memory at src into L2 (no destination, no
// completion to wait for); src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Generic-proxy accesses to shared memory before a later bulk copy into it.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(mbar), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of mbar.  On timeout the wait is counted
// and retried once more (bounded too) so that no copy into this CTA's shared
// memory is left in flight when it returns; false = the data is not there.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (int i = 0; i < kWaitPolls; ++i)
        if (mbar_try_wait(mbar, parity))
            return true;
    atomicAdd(&g_wait_timeouts, 1ull);
    for (int i = 0; i < kWaitPolls; ++i)
        if (mbar_try_wait(mbar, parity))
            return false;
    return false;
}

}  // namespace edm

namespace edm {

// Stage series src (T floats) into xs_base[front .. front + T) and +inf
// everywhere else in [0, total) (lags before the series start, the tail of
// the last candidate chunk).  The 16-byte aligned body goes by one bulk copy
// when src and the destination are 16-byte aligned; the rest (and every
// unaligned series) by the threads.  Call with every thread of the CTA;
// returns with the series in place after a __syncthreads, with the same
// value in every thread (false: the copy timed out and the CTA should skip
// its work).
__device__ __forceinline__ bool stage_series_bulk(float *xs_base, const float *__restrict__ src, int T, int front,
                                                  int total)
{
    __shared__ __align__(8) unsigned long long series_bar;
    const uint32_t xb = (uint32_t)__cvta_generic_to_shared(xs_base);
    const uint32_t dst = xb + (uint32_t)front * 4u;
    const bool aligned = ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) && ((dst & 15u) == 0);
    const int body = aligned ? (T & ~3) : 0;  // floats moved by the bulk copy
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&series_bar);
    if (body > 0 && threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_expect_tx(bar, (uint32_t)body * 4u);
        bulk_g2s(dst, src, (uint32_t)body * 4u, bar);
    }
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int t = i - front;
        if (t < 0 || t >= body)
            xs_base[i] = (t >= 0 && t < T) ? src[t] : CUDART_INF_F;
    }
    __syncthreads();
    const bool ok = body > 0 ? mbar_wait(bar, 0) : true;
    return __syncthreads_and(ok) != 0;
}

}  // namespace edm
