// backward.cu -- adjoint of the cross map: dL/dY for L = sum_ij g_ij rho_ij
// with every kNN index and every optimal E held fixed.
//
// The paper has no gradients; this differentiates its rho (simplex weights
// w = exp(-d/d_1)/sum, Algorithm 5 lookup, Pearson corrcoef).  For one pair
// (library x, target y, rows t of the table):
//   p_t = sum_n w_tn y(s_tn + Tp),  o_t = y(t + Tp),
//   d rho / d p_t = a_t = alpha (o_t - o_bar) - beta (p_t - p_bar),
//   d rho / d o_t = b_t = alpha (p_t - p_bar) - gamma (o_t - o_bar),
//   alpha = g / sqrt(Vp Vo), beta = g rho / Vp, gamma = g rho / Vo
// (g = dL/d rho folded in).  Target side: y(s_tn + Tp) += a_t w_tn,
// y(t + Tp) += b_t.  Library side, through the weights:
//   H_tn = sum_targets a_t (y(s_tn + Tp) - p_t),
//   dL/dd_tn = -(w_tn / d_t1) H_tn (n >= 2),
//   dL/dd_t1 = sum_{n>=2} (w_tn d_tn / d_t1^2) H_tn,
// then d_tn = sqrt(sum_m (x(t - m tau) - x(s_tn - m tau))^2) carries it to x.
// Where d = 0 (or d_t1 = 0, duplicate-only weights) the gradient is 0.
//
// Pass 1 (one CTA per target) also stores (alpha, beta, p_bar) per pair for
// pass 2 (one CTA per library).  Both accumulate in shared memory with
// atomic adds and then add their row of grad_Y once.  The per-pair sums
// are FP32 within a thread and a warp and FP64 across the warps (FP64 is a
// small fraction of the FP32 rate on this GPU), over predictions shifted by
// row 0's prediction K (d = p - K; equal predictions give exact zeros, so a
// constant prediction keeps its zero variance and zero gradient): sum d,
// then the centred sums of (d - d_bar)^2 and (d - d_bar)(o - o_bar).  The
// means, variances and coefficients are FP64.
#include <algorithm>

#include "bulk_copy.cuh"
#include "edm_internal.cuh"
#include "launchers.h"

namespace edm {

constexpr int kBwThreads = 256;
constexpr int kBwMaxRows = 12;  // rows per thread: T - Tp <= 12 * 256

__device__ __forceinline__ double block_sum_d(double v, double *sh)
{
    v = warp_sum_d(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0)
        sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (int)(blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        t = warp_sum_d(t);
        if (threadIdx.x == 0)
            sh[0] = t;
    }
    __syncthreads();
    return sh[0];
}

// Block sum of per-thread FP32 partials (two at once): FP32 within each
// warp, FP64 across the warps.  Thread 0 receives the sums; the others 0.
__device__ __forceinline__ void block_sum2_f(float v0, float v1, double *sh, double &s0, double &s1)
{
    v0 = warp_sum(v0);
    v1 = warp_sum(v1);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sh[2 * w] = (double)v0;
        sh[2 * w + 1] = (double)v1;
    }
    __syncthreads();
    s0 = s1 = 0.0;
    if (threadIdx.x < 32) {
        const bool in = threadIdx.x < (int)(blockDim.x >> 5);
        s0 = warp_sum_d(in ? sh[2 * threadIdx.x] : 0.0);
        s1 = warp_sum_d(in ? sh[2 * threadIdx.x + 1] : 0.0);
    }
}

// Per-pair scalars of pass 1, formed once by thread 0 and shared.
struct BwPairScalars {
    float dbf, fa, fb, fg, fpb;
};

// Pass 1 for one target of k neighbours: every library of the block in turn.
__device__ __forceinline__ void bw_target_libs(const BwArgs &a, const float *y, float *gy, int j, int E, int k, int L,
                                               int Tq, double ob, double vo, double *sh, BwPairScalars &ps)
{
    const double n = (double)Tq;
    const double inv_n = 1.0 / n;
    const float obf = (float)ob;
    const size_t tq = (size_t)a.lay.Tq_pad;
    for (int li = 0; li < a.n_lib; ++li) {
        const int64_t i = a.lib0 + li;
        const uint8_t *lb = a.tables + (size_t)li * a.lay.lib_stride;
        const float *Wt = reinterpret_cast<const float *>(lb + a.lay.off_w[E]);
        const uint16_t *It = reinterpret_cast<const uint16_t *>(lb + a.lay.off_i[E]);
        float p[kBwMaxRows];
#pragma unroll
        for (int q = 0; q < kBwMaxRows; ++q) {
            const int r = threadIdx.x + q * kBwThreads;
            p[q] = 0.f;
            if (r < Tq) {
                float acc = 0.f;
                for (int nn = 0; nn < k; ++nn)
                    acc = fmaf(__ldg(Wt + nn * tq + r), y[__ldg(It + nn * tq + r)], acc);
                p[q] = acc;
            }
        }
        // shift: row 0's prediction (Tq >= 1)
        if (threadIdx.x == 0)
            ps.fpb = p[0];
        __syncthreads();
        const float K0 = ps.fpb;
        float sdf = 0.f;
#pragma unroll
        for (int q = 0; q < kBwMaxRows; ++q)
            if (threadIdx.x + q * kBwThreads < Tq)
                sdf += p[q] - K0;
        double S, unused;
        block_sum2_f(sdf, 0.f, sh, S, unused);
        if (threadIdx.x == 0)
            ps.dbf = (float)(S * inv_n);
        __syncthreads();
        const float dbf = ps.dbf;
        float vpf = 0.f, cf = 0.f;
#pragma unroll
        for (int q = 0; q < kBwMaxRows; ++q) {
            const int r = threadIdx.x + q * kBwThreads;
            if (r < Tq) {
                const float dp = (p[q] - K0) - dbf;
                vpf = fmaf(dp, dp, vpf);
                cf = fmaf(dp, y[L + r + a.Tp] - obf, cf);
            }
        }
        double vp, c;
        block_sum2_f(vpf, cf, sh, vp, c);
        if (threadIdx.x == 0) {
            const double pb = (double)K0 + S * inv_n;
            const double g = (double)a.grad_rho[(int64_t)j * a.ld_g + i];
            double alpha = 0.0, beta = 0.0, gam = 0.0;
            if (vp > 0.0 && vo > 0.0) {
                const double sq = sqrt(vp * vo);
                const double rho = c / sq;
                alpha = g / sq;
                beta = g * rho / vp;
                gam = g * rho / vo;
            }
            a.stats[i * a.N + j] = make_float4((float)alpha, (float)beta, (float)pb, 0.f);
            ps.fa = (float)alpha;
            ps.fb = (float)beta;
            ps.fg = (float)gam;
            ps.fpb = (float)pb;
        }
        __syncthreads();
        const float fa = ps.fa, fb = ps.fb, fg = ps.fg, fpb = ps.fpb;
#pragma unroll
        for (int q = 0; q < kBwMaxRows; ++q) {
            const int r = threadIdx.x + q * kBwThreads;
            if (r < Tq) {
                const float ov = y[L + r + a.Tp] - obf, pv = p[q] - fpb;
                const float at = fa * ov - fb * pv;
                const float bt = fa * pv - fg * ov;
                for (int nn = 0; nn < k; ++nn)
                    atomicAdd(&gy[__ldg(It + nn * tq + r)], at * __ldg(Wt + nn * tq + r));
                atomicAdd(&gy[L + r + a.Tp], bt);
            }
        }
        __syncthreads();
    }
}

// Pass 1: one CTA per target j, libraries lib0 .. lib0+n_lib-1.
__global__ void __launch_bounds__(kBwThreads) bw_target_kernel(BwArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float *y = reinterpret_cast<float *>(smem);
    float *gy = y + a.T;
    __shared__ double sh[32];
    __shared__ BwPairScalars ps;
    const int j = blockIdx.x;
    const float *src = a.Y + (int64_t)j * a.ldY;
    for (int t = threadIdx.x; t < a.T; t += blockDim.x) {
        y[t] = src[t];
        gy[t] = 0.f;
    }
    __syncthreads();
    const int E = a.optE[j], k = E + 1;
    const int L = (E - 1) * a.tau;
    const int Tq = a.T - a.Tp - L;
    // a target whose E is unusable (outside 1..EDM_MAX_E, or too few
    // candidates) has no rho and no gradient
    if (E < 1 || E > EDM_MAX_E || Tq - (a.excl >= 0 ? 2 * a.excl + 1 : 0) < k) {
        float *dst = a.grad_Y + (int64_t)j * a.ldY;
        for (int t = threadIdx.x; t < a.T; t += blockDim.x)
            dst[t] += gy[t];
        return;
    }
    const double n = (double)Tq;
    // observation window statistics (once per target)
    double so = 0.0;
    for (int r = threadIdx.x; r < Tq; r += blockDim.x)
        so += (double)y[L + r + a.Tp];
    so = block_sum_d(so, sh);
    const double ob = so / n;
    double vo = 0.0;
    for (int r = threadIdx.x; r < Tq; r += blockDim.x) {
        double d = (double)y[L + r + a.Tp] - ob;
        vo += d * d;
    }
    vo = block_sum_d(vo, sh);
    if (threadIdx.x == 0)
        a.obar[j] = (float)ob;
    bw_target_libs(a, y, gy, j, E, k, L, Tq, ob, vo, sh, ps);
    float *dst = a.grad_Y + (int64_t)j * a.ldY;
    for (int t = threadIdx.x; t < a.T; t += blockDim.x)
        dst[t] += gy[t];
}

// Pass 2: one CTA per library in the block.  For each E, in chunks of
// rows: the chunk's table entries (W and I) are staged in shared memory
// once, then every target of that E adds its terms to H [k][rows of the
// chunk] from shared memory only.  With dbl (rows 16-byte aligned, T a
// multiple of 4) the target series are double-buffered: while one target's
// terms are added, a bulk copy brings the next target's series into the
// other buffer.
__global__ void __launch_bounds__(kBwThreads) bw_library_kernel(BwArgs a, int buf_bytes, int dbl)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(8) unsigned long long ybar[2];
    float *x = reinterpret_cast<float *>(smem);
    float *gx = x + a.T;
    float *const yb0 = gx + a.T, *const yb1 = gx + 2 * a.T;  // yb1 only with dbl
    unsigned char *buf = reinterpret_cast<unsigned char *>(gx + (dbl ? 3 : 2) * a.T);
    const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&ybar[0]);
    const uint32_t bar1 = (uint32_t)__cvta_generic_to_shared(&ybar[1]);
    const uint32_t ybytes = (uint32_t)a.T * 4u;
    uint32_t par0 = 0u, par1 = 0u;  // phase of each buffer's next completion
    if (dbl && threadIdx.x == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar1, 1);
    }
    const int li = blockIdx.x;
    const int64_t i = a.lib0 + li;
    const float *src = a.Y + i * a.ldY;
    for (int t = threadIdx.x; t < a.T; t += blockDim.x) {
        x[t] = src[t];
        gx[t] = 0.f;
    }
    __syncthreads();
    const uint8_t *lb = a.tables + (size_t)li * a.lay.lib_stride;
    const size_t tq = (size_t)a.lay.Tq_pad;
    for (int E = 1; E <= EDM_MAX_E; ++E) {
        const int j0 = a.e_start[E], j1 = a.e_start[E + 1];
        if (j0 == j1)
            continue;
        const int k = E + 1;
        const int L = (E - 1) * a.tau;
        const int Tq = a.T - a.Tp - L;
        const float *Wt = reinterpret_cast<const float *>(lb + a.lay.off_w[E]);
        const uint16_t *It = reinterpret_cast<const uint16_t *>(lb + a.lay.off_i[E]);
        // rows per chunk: H and W (4 bytes each) and I (2 bytes) per entry,
        // a multiple of 4 rows so the arrays stay 16-byte aligned
        const int h_rows = max(4, min((Tq + 3) & ~3, (buf_bytes / (10 * k)) & ~3));
        for (int r0 = 0; r0 < Tq; r0 += h_rows) {
            const int rn = min(h_rows, Tq - r0);
            float *H = reinterpret_cast<float *>(buf);
            float *Ws = H + (size_t)k * h_rows;
            uint16_t *Is = reinterpret_cast<uint16_t *>(Ws + (size_t)k * h_rows);
            for (int q = threadIdx.x; q < k * rn; q += blockDim.x) {
                const int nn = q / rn, rr = q - nn * rn;
                H[nn * h_rows + rr] = 0.f;
                Ws[nn * h_rows + rr] = Wt[nn * tq + r0 + rr];
                Is[nn * h_rows + rr] = It[nn * tq + r0 + rr];
            }
            __syncthreads();
            if (dbl && threadIdx.x == 0) {
                fence_proxy_async_smem();
                mbar_expect_tx(bar0, ybytes);
                bulk_g2s((uint32_t)__cvta_generic_to_shared(yb0), a.Y + (int64_t)a.pi[j0] * a.ldY, ybytes, bar0);
            }
            for (int pj = j0; pj < j1; ++pj) {
                const int j = a.pi[pj];
                const float *ys = a.Y + (int64_t)j * a.ldY;
                const bool odd = dbl && ((pj - j0) & 1);
                float *yb = odd ? yb1 : yb0;
                if (dbl) {
                    // the other buffer was last read before the barrier that
                    // ended the previous target: refill it with the next one
                    if (threadIdx.x == 0 && pj + 1 < j1) {
                        fence_proxy_async_smem();
                        mbar_expect_tx(odd ? bar0 : bar1, ybytes);
                        bulk_g2s((uint32_t)__cvta_generic_to_shared(odd ? yb0 : yb1),
                                 a.Y + (int64_t)a.pi[pj + 1] * a.ldY, ybytes, odd ? bar0 : bar1);
                    }
                    const bool got = mbar_wait(odd ? bar1 : bar0, odd ? par1 : par0);
                    if (odd)
                        par1 ^= 1u;
                    else
                        par0 ^= 1u;
                    if (!__syncthreads_and(got)) {
                        // a copy that did not arrive in time (counted): load
                        // the row here (a late copy writes the same values)
                        for (int t = threadIdx.x; t < a.T; t += blockDim.x)
                            yb[t] = ys[t];
                        __syncthreads();
                    }
                } else {
                    for (int t = threadIdx.x; t < a.T; t += blockDim.x)
                        yb[t] = ys[t];
                    __syncthreads();
                }
                const float4 st = a.stats[i * a.N + j];
                const float ob = a.obar[j];
                for (int rr = threadIdx.x; rr < rn; rr += blockDim.x) {
                    const int r = r0 + rr;
                    float pv = 0.f;
                    for (int nn = 0; nn < k; ++nn)
                        pv = fmaf(Ws[nn * h_rows + rr], yb[Is[nn * h_rows + rr]], pv);
                    const float at = st.x * (yb[L + r + a.Tp] - ob) - st.y * (pv - st.z);
                    for (int nn = 0; nn < k; ++nn)
                        H[nn * h_rows + rr] += at * (yb[Is[nn * h_rows + rr]] - pv);
                }
                __syncthreads();
            }
            // chain H through the weights and distances into x
            for (int rr = threadIdx.x; rr < rn; rr += blockDim.x) {
                const int r = r0 + rr;
                const int t = L + r;
                float d[EDM_MAX_E + 1];
                for (int nn = 0; nn < k; ++nn) {
                    const int s = (int)Is[nn * h_rows + rr] - a.Tp;
                    float acc = 0.f;
                    for (int m = 0; m < E; ++m) {
                        float df = x[t - m * a.tau] - x[s - m * a.tau];
                        acc = fmaf(df, df, acc);
                    }
                    d[nn] = sqrtf(acc);
                }
                const float d1 = d[0];
                if (!(d1 > 0.f))
                    continue;  // duplicate-only weights: constant
                float g0 = 0.f;
                for (int nn = 1; nn < k; ++nn) {
                    const float wv = Ws[nn * h_rows + rr];
                    const float h = H[nn * h_rows + rr];
                    g0 += wv * d[nn] / (d1 * d1) * h;
                    const float gn = -(wv / d1) * h;
                    if (d[nn] > 0.f) {
                        const int s = (int)Is[nn * h_rows + rr] - a.Tp;
                        const float cf = gn / d[nn];
                        for (int m = 0; m < E; ++m) {
                            float df = x[t - m * a.tau] - x[s - m * a.tau];
                            atomicAdd(&gx[t - m * a.tau], cf * df);
                            atomicAdd(&gx[s - m * a.tau], -cf * df);
                        }
                    }
                }
                {
                    const int s = (int)Is[rr] - a.Tp;
                    const float cf = g0 / d1;
                    for (int m = 0; m < E; ++m) {
                        float df = x[t - m * a.tau] - x[s - m * a.tau];
                        atomicAdd(&gx[t - m * a.tau], cf * df);
                        atomicAdd(&gx[s - m * a.tau], -cf * df);
                    }
                }
            }
            __syncthreads();
        }
    }
    float *dst = a.grad_Y + i * a.ldY;
    for (int t = threadIdx.x; t < a.T; t += blockDim.x)
        dst[t] += gx[t];
}

int bw_max_T() { return kBwMaxRows * kBwThreads; }

EDM_WAIT_TIMEOUT_READER(backward_wait_timeouts)

// Library pass: x, gx and one or two target series (3T or 4T floats) and a
// buffer for a chunk's H, W and I (10 bytes per row and neighbour), sized
// for about 110 KB per CTA (two CTAs per SM) and at least 4 rows of the
// largest K.
static size_t bw_lib_smem(int T, int dbl, size_t buf_bytes) { return (size_t)(dbl ? 4 : 3) * T * 4 + buf_bytes; }

cudaError_t launch_backward(const BwArgs &a, int kmax, cudaStream_t st)
{
    size_t s1 = (size_t)2 * a.T * 4;
    cudaError_t e = cudaFuncSetAttribute(bw_target_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1);
    if (e != cudaSuccess)
        return e;
    bw_target_kernel<<<a.N, kBwThreads, s1, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    // double-buffered target series when every row is a 16-byte aligned bulk copy
    const int dbl = (a.T % 4 == 0 && a.ldY % 4 == 0 && (reinterpret_cast<uintptr_t>(a.Y) & 15) == 0 &&
                     (size_t)a.T * 4 < (1u << 20))
                        ? 1
                        : 0;
    const size_t fixed = (size_t)(dbl ? 4 : 3) * a.T * 4;
    const size_t target = 110 * 1024;
    const size_t floor_bytes = (size_t)10 * kmax * 8;
    size_t buf = target > fixed + floor_bytes ? target - fixed : floor_bytes;
    buf = std::min(buf, (size_t)10 * kmax * (size_t)(a.T + 3));
    buf &= ~(size_t)15;
    const size_t s2 = bw_lib_smem(a.T, dbl, buf);
    if (s2 > 227 * 1024)
        return cudaErrorInvalidValue;
    if ((e = cudaFuncSetAttribute(bw_library_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s2)) !=
        cudaSuccess)
        return e;
    bw_library_kernel<<<a.n_lib, kBwThreads, s2, st>>>(a, (int)buf, dbl);
    return cudaGetLastError();
}

}  // namespace edm
