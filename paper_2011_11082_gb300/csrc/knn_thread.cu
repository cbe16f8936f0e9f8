// knn_thread.cu -- thread-per-query exact kNN tables for one E <= 6 (tau = 1).
//
// The warp-per-query kernel of knn_core.cuh grows distances for every E in
// one sweep and pays a warp-wide selection per (query, E).  For the common
// small E (phase-2 target blocks hold one or a few E) it is cheaper to give
// each thread one query point t and let it sweep all candidates itself:
// all threads of a warp read the same candidate window (broadcast shared
// loads, four candidates per group of 16-byte loads), compute the FP32
// squared distance in the same operation order as the warp kernel (zero
// start, one fma per lag, lags 0..E-1 -- Sec. II-B's embedding, Algorithm
// 3's distances), and keep the K = E+3 smallest (d2, s) keys in a sorted
// register list (insertion is rare after the first few hundred candidates).
// Certification, FP64 fallback and weights follow the warp kernel's rules
// exactly, so the neighbour indices are identical; tables are written one
// row per thread, i.e. coalesced.  Measured against the warp kernel on
// 1,024 libraries of T = 1,500 (one E per launch): 1.37 vs 2.30 ms at E = 1,
// 2.44 vs 3.21 ms at E = 4, equal at E = 7, slower above -- so it serves
// single-E table sets with E <= 6 (a multi-E set is cheaper in the warp
// kernel, whose distance sweep serves every E at once).
#include <cuda_fp16.h>

#include "bulk_copy.cuh"
#include "edm_internal.cuh"
#include "launchers.h"

namespace edm {

EDM_WAIT_TIMEOUT_READER(knn_thread_wait_timeouts)

namespace {

__device__ unsigned long long g_thread_counts[2];  // FP64 re-ranks, exhaustive scans

constexpr int kTqThreads = 256;

// Floats staged before x[0] (+inf) for E lags read in 16-byte groups.
__host__ __device__ constexpr int tq_front(int E) { return ((E - 1 + 3) / 4) * 4 + 4; }

__host__ __device__ inline size_t tq_smem_floats(int T, int E) { return (size_t)tq_front(E) + ((T + 3) & ~3) + 8; }

// FP64 squared distance in the reference's operation order.
__device__ __forceinline__ double dist64_t(const float *x, int t, int s, int E)
{
    double d = 0.0;
    for (int m = 0; m < E; ++m) {
        double diff = __dsub_rn((double)x[t - m], (double)x[s - m]);
        d = __dadd_rn(d, __dmul_rn(diff, diff));
    }
    return d;
}

template <int E, bool kPublic>
__global__ void __launch_bounds__(kTqThreads, (E <= 8 ? 4 : 2))
    knn_thread_kernel(const float *__restrict__ Y, int64_t ldY, int64_t lib0, int T, int Tp, int excl,
                      const __grid_constant__ TableLayout lay, uint8_t *__restrict__ tables,
                      int32_t *__restrict__ pub_idx, float *__restrict__ pub_w, const uint32_t *__restrict__ sel_dev,
                      int s_lo)
{
    if (sel_dev && !((*sel_dev >> (E - 1)) & 1u))
        return;  // E not in use (set planned on the device)
    constexpr int k = E + 1;
    constexpr int KL = E + 1 + kGuard;  // kept entries (k + guard)
    constexpr int F = tq_front(E);
    constexpr int NV = (E - 1 + 3) / 4 + 1;  // float4 groups per candidate group
    extern __shared__ __align__(16) float xs_base[];
    float *xs = xs_base + F;
    const int lib = blockIdx.y;
    const float *src = Y + (lib0 + lib) * ldY;
    const int total = (int)tq_smem_floats(T, E);
    if (!stage_series_bulk(xs_base, src, T, F, total))
        return;

    const int Tq = T - Tp - (E - 1);
    const int r = blockIdx.x * kTqThreads + threadIdx.x;
    if (blockIdx.x * kTqThreads >= Tq)
        return;
    const bool active = r < Tq && (E - 1) + r >= s_lo;
    const int t = (E - 1) + (active ? r : 0);
    const int s_last = T - 1 - Tp;
    float xq[E];
#pragma unroll
    for (int m = 0; m < E; ++m)
        xq[m] = xs[t - m];
    // sorted list of the KL smallest (d2, s); the sweep visits s in
    // increasing order, so a candidate whose d2 equals a kept one ranks after
    // it and the strict float comparison reproduces the (d2, s) order
    float D[KL];
    int S[KL];
#pragma unroll
    for (int i = 0; i < KL; ++i) {
        D[i] = CUDART_INF_F;
        S[i] = 0x7fffffff;
    }
    // exclusion window |s - t| <= excl as one unsigned range test
    const int ex_lo = excl >= 0 ? t - excl : s_last + 8;
    const unsigned ex_span = excl >= 0 ? (unsigned)(2 * excl) : 0u;

    const float4 *x4 = reinterpret_cast<const float4 *>(xs_base);
    // candidates below E-1 read the +inf padding (d2 = +inf, never kept);
    // full groups need no bound test, the last partial group does
    const int s_start = max(E - 1, s_lo);
    for (int s0 = s_start & ~3; s0 <= s_last; s0 += 4) {
        // v[j] = x[s0 - 4(NV-1) + j], j < 4 NV
        float v[4 * NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const float4 f = x4[(F + s0) / 4 - (NV - 1) + i];
            v[4 * i] = f.x;
            v[4 * i + 1] = f.y;
            v[4 * i + 2] = f.z;
            v[4 * i + 3] = f.w;
        }
        const bool edge = s0 + 3 > s_last || s0 < s_start;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float d = 0.f;
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const float diff = xq[m] - v[4 * (NV - 1) + u - m];
                d = fmaf(diff, diff, d);
            }
            const int s = s0 + u;
            if ((unsigned)(s - ex_lo) <= ex_span || (edge && (s > s_last || s < s_start)))
                d = CUDART_INF_F;
            if (d < D[KL - 1]) {
                float cd = d;
                int cs = s;
#pragma unroll
                for (int i = 0; i < KL; ++i) {
                    const bool lt = cd < D[i];
                    const float td = D[i];
                    const int ts = S[i];
                    D[i] = lt ? cd : td;
                    S[i] = lt ? cs : ts;
                    cd = lt ? td : cd;
                    cs = lt ? ts : cs;
                }
            }
        }
    }
    if (!active)
        return;

    // certification (same rule as the warp kernel)
    int have = 0;
#pragma unroll
    for (int i = 0; i < KL; ++i)
        have += D[i] < CUDART_INF_F;
    bool full = have < k;
    bool ok = !full && D[0] >= kNearDup;
#pragma unroll
    for (int n = 0; n < k; ++n) {
        if (n + 1 < KL) {
            if (n + 1 < have)
                ok = ok && (D[n + 1] - D[n]) > d2_err(D[n], E) + d2_err(D[n + 1], E);
            else
                ok = ok && have < KL;
        }
    }
    int s_n[k];
    float w_n[k];
    if (ok) {
        const float inv_d1 = __frcp_rn(sqrtf(D[0]));
        float u[k], sum = 0.f;
#pragma unroll
        for (int n = 0; n < k; ++n) {
            u[n] = expf(-sqrtf(D[n]) * inv_d1);
            sum += u[n];
        }
        const float inv = __frcp_rn(sum);
#pragma unroll
        for (int n = 0; n < k; ++n) {
            w_n[n] = u[n] * inv;
            s_n[n] = S[n];
        }
    } else {
        // FP64 re-rank of the kept entries; exhaustive FP64 scan when the
        // k-th place cannot be separated from what was left out
        double d64[KL];
        int s64[KL];
        const int hv = have;
        for (int i = 0; i < KL; ++i) {
            s64[i] = S[i];
            d64[i] = i < hv ? dist64_t(xs, t, S[i], E) : CUDART_INF;
        }
        for (int i = 1; i < hv; ++i)  // insertion sort by (d64, s)
            for (int j = i; j > 0 && (d64[j] < d64[j - 1] || (d64[j] == d64[j - 1] && s64[j] < s64[j - 1])); --j) {
                const double td = d64[j];
                d64[j] = d64[j - 1];
                d64[j - 1] = td;
                const int ts = s64[j];
                s64[j] = s64[j - 1];
                s64[j - 1] = ts;
            }
        if (!full && hv >= KL) {
            const float Dlast = D[KL - 1];
            full = !(d64[k - 1] < (double)(Dlast - d2_err(Dlast, E)));
        }
        if (full) {
            double last_d = -1.0;
            int last_s = -1;
            for (int n = 0; n < k; ++n) {
                double bd = CUDART_INF;
                int bs = 0x7fffffff;
                for (int s = s_start; s <= s_last; ++s) {
                    if (excl >= 0 && abs(s - t) <= excl)
                        continue;
                    const double dd = dist64_t(xs, t, s, E);
                    const bool after = (dd > last_d) || (dd == last_d && s > last_s);
                    const bool better = (dd < bd) || (dd == bd && s < bs);
                    if (after && better) {
                        bd = dd;
                        bs = s;
                    }
                }
                d64[n] = bd;
                s64[n] = bs;
                last_d = bd;
                last_s = bs;
            }
        }
        atomicAdd(&g_thread_counts[full ? 1 : 0], 1ull);
        const double d1 = sqrt(d64[0]);
        double u[k], sum = 0.0;
        for (int n = 0; n < k; ++n) {
            const double dd = sqrt(d64[n]);
            u[n] = d1 > 0.0 ? exp(-dd / d1) : (dd == 0.0 ? 1.0 : 0.0);
        }
        for (int n = 0; n < k; ++n)
            sum += u[n];
        for (int n = 0; n < k; ++n) {
            w_n[n] = (float)(u[n] / sum);
            // (non-finite inputs can leave a sentinel; keep indices inside)
            s_n[n] = min(max(s64[n], s_start), s_last);
        }
    }
    if (kPublic) {
        int32_t *ip = pub_idx + ((size_t)lib * Tq + r) * k;
        float *wp = pub_w + ((size_t)lib * Tq + r) * k;
#pragma unroll
        for (int n = 0; n < k; ++n) {
            ip[n] = s_n[n];
            wp[n] = w_n[n];
        }
    } else {
        uint8_t *lb = tables + (size_t)lib * lay.lib_stride;
        float *wp = reinterpret_cast<float *>(lb + lay.off_w[E]);
        uint16_t *ip = reinterpret_cast<uint16_t *>(lb + lay.off_i[E]);
#pragma unroll
        for (int n = 0; n < k; ++n) {
            wp[(size_t)n * lay.Tq_pad + r] = w_n[n];
            ip[(size_t)n * lay.Tq_pad + r] = (uint16_t)(s_n[n] + Tp);
        }
    }
}

template <int E, bool kPublic>
cudaError_t launch_E(const float *Y, int64_t ldY, int64_t lib0, int n_lib, int T, int Tp, int excl,
                     const TableLayout &lay, uint8_t *tables, int32_t *pidx, float *pw, cudaStream_t st,
                     const uint32_t *sel_dev, int s_lo)
{
    const size_t smem = tq_smem_floats(T, E) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(knn_thread_kernel<E, kPublic>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    const int Tq = T - Tp - (E - 1);
    dim3 grid((unsigned)((Tq + kTqThreads - 1) / kTqThreads), (unsigned)n_lib);
    knn_thread_kernel<E, kPublic><<<grid, kTqThreads, smem, st>>>(Y, ldY, lib0, T, Tp, excl, lay, tables, pidx, pw,
                                                                   sel_dev, s_lo);
    return cudaGetLastError();
}

template <bool kPublic>
cudaError_t launch_any(int E, const float *Y, int64_t ldY, int64_t lib0, int n_lib, int T, int Tp, int excl,
                       const TableLayout &lay, uint8_t *tables, int32_t *pidx, float *pw, cudaStream_t st,
                       const uint32_t *sel_dev, int s_lo)
{
    switch (E) {
#define EDM_TQ(EE)                                                                                                     \
    case EE:                                                                                                           \
        return launch_E<EE, kPublic>(Y, ldY, lib0, n_lib, T, Tp, excl, lay, tables, pidx, pw, st, sel_dev, s_lo);
        EDM_TQ(1)
        EDM_TQ(2)
        EDM_TQ(3)
        EDM_TQ(4)
        EDM_TQ(5)
        EDM_TQ(6)
#undef EDM_TQ
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int knn_thread_max_E() { return 6; }

cudaError_t launch_knn_thread(const float *Y, int64_t ldY, int64_t lib0, int n_lib, int T, int Tp, int excl, int E,
                              const TableLayout &lay, uint8_t *tables, cudaStream_t st, const uint32_t *sel_dev,
                              int s_lo)
{
    return launch_any<false>(E, Y, ldY, lib0, n_lib, T, Tp, excl, lay, tables, nullptr, nullptr, st, sel_dev, s_lo);
}

cudaError_t launch_knn_thread_public(const float *Y, int64_t ldY, int n_lib, int T, int E, int Tp, int excl,
                                     int32_t *idx, float *w, cudaStream_t st)
{
    TableLayout lay{};
    return launch_any<true>(E, Y, ldY, 0, n_lib, T, Tp, excl, lay, nullptr, idx, w, st, nullptr, 0);
}

cudaError_t knn_thread_counters(unsigned long long out[2], bool reset)
{
    cudaError_t e = cudaMemcpyFromSymbol(out, g_thread_counts, sizeof(unsigned long long) * 2);
    if (e == cudaSuccess && reset) {
        const unsigned long long z[2] = {0ull, 0ull};
        e = cudaMemcpyToSymbol(g_thread_counts, z, sizeof z);
    }
    return e;
}

}  // namespace edm
