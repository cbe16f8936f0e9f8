// lookup_chunked128.cu -- the chunked lookup for 128-byte tile rows
// (32 FP32 / 64 FP16 targets per row; series up to about 1,500 steps), the
// FP16 target staging and the dispatch over row widths and forms.
#define EDM_RB 128
#define EDM_LAG false
#define EDM_MULTI_NAME lookup_multi128_kernel
#define EDM_MULTI_LAUNCH launch_lookup_multi128
#define EDM_MULTI_TIMEOUTS lookup_multi128_wait_timeouts
#include "lookup_multi_impl.cuh"

namespace edm {

// alignment pad, the tile, the per-warp fold buffers, the tile's barrier word
size_t chunked_smem_bytes(int T, int RB) { return 128 + (size_t)T * RB + (size_t)kCkWarps * 32 * kCkRed * 4 + 16; }

// ---------------------------------------------------------------------------
// FP16 staging: 64 targets per tile, z-normalised in FP64 then rounded to
// FP16; the observation moments are taken over the rounded values (what the
// lookup reads).  Tiles without the FP16 flag are left to the FP32 stager.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) prep_targets_f16_kernel(const float *__restrict__ Y, int64_t ldY, int T, int tau,
                                                               int Tp, const int32_t *__restrict__ pi,
                                                               const TileMeta *__restrict__ meta, uint8_t *__restrict__ tiles,
                                                               float2 *__restrict__ omom, int words)
{
    __shared__ float mu_s[64], inv_s[64];
    const TileMeta m = meta[blockIdx.x];
    if (!(m.flags & kTileF16))
        return;
    const int lane = lane_id(), warp = warp_id();
    for (int slot = warp; slot < 64; slot += 8) {
        double mu = 0.0, inv = 0.0;
        if (slot < m.count) {
            const float *y = Y + (int64_t)pi[m.first + slot] * ldY;
            double acc = 0.0;
            for (int t = lane; t < T; t += 32)
                acc += (double)y[t];
            mu = warp_sum_d(acc) / (double)T;
            double v = 0.0;
            for (int t = lane; t < T; t += 32) {
                double d = (double)y[t] - mu;
                v += d * d;
            }
            v = warp_sum_d(v) / (double)T;
            inv = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
            const float muf = (float)mu, invf = (float)inv;
            const int L = (m.E - 1) * tau;
            double so = 0.0, soo = 0.0;
            for (int t = L + Tp + lane; t < T; t += 32) {
                float z = __half2float(__float2half_rn((y[t] - muf) * invf));
                so += (double)z;
                soo += (double)z * (double)z;
            }
            so = warp_sum_d(so);
            soo = warp_sum_d(soo);
            if (lane == 0) {
                double n = (double)(T - Tp - L);
                omom[m.first + slot] = make_float2((float)so, (float)(n * soo - so * so));
            }
        }
        if (lane == 0) {
            mu_s[slot] = (float)mu;
            inv_s[slot] = (float)inv;
        }
    }
    __syncthreads();
    // rows of `words` 32-bit words; word w holds targets w and w + words
    uint32_t *tile = reinterpret_cast<uint32_t *>(tiles + (size_t)blockIdx.x * T * words * 4);
    if (lane < words) {
        const float *ylo = lane < m.count ? Y + (int64_t)pi[m.first + lane] * ldY : nullptr;
        const float *yhi = lane + words < m.count ? Y + (int64_t)pi[m.first + lane + words] * ldY : nullptr;
        const float mlo = mu_s[lane], ilo = inv_s[lane], mhi = mu_s[lane + words], ihi = inv_s[lane + words];
        for (int t = warp; t < T; t += 8) {
            float zl = ylo ? (ylo[t] - mlo) * ilo : 0.f;
            float zh = yhi ? (yhi[t] - mhi) * ihi : 0.f;
            __half2 h = __floats2half2_rn(zl, zh);
            tile[(size_t)t * words + lane] = *reinterpret_cast<uint32_t *>(&h);
        }
    }
}

cudaError_t launch_prep_targets_f16(const float *Y, int64_t ldY, int T, int tau, int Tp, const int32_t *pi,
                                    const TileMeta *meta, int n_tiles, uint8_t *tiles, float2 *omom, cudaStream_t st,
                                    int RB)
{
    if (n_tiles <= 0)
        return cudaSuccess;
    prep_targets_f16_kernel<<<n_tiles, 256, 0, st>>>(Y, ldY, T, tau, Tp, pi, meta, tiles, omom, RB / 4);
    return cudaGetLastError();
}

cudaError_t launch_lookup_multi128_lag(const LookupArgs &a, cudaStream_t st);
cudaError_t launch_lookup_multi64(const LookupArgs &a, cudaStream_t st);
cudaError_t launch_lookup_multi64_lag(const LookupArgs &a, cudaStream_t st);

// The time-delay form is a separate instantiation, so the plain cross map
// keeps its register allocation.
cudaError_t launch_lookup_multi(const LookupArgs &a, int RB, cudaStream_t st)
{
    const bool lag = a.s_lo != 0 || a.lag != a.Tp;
    if (RB == 128)
        return lag ? launch_lookup_multi128_lag(a, st) : launch_lookup_multi128(a, st);
    return lag ? launch_lookup_multi64_lag(a, st) : launch_lookup_multi64(a, st);
}

int chunked_row_bytes(int T)
{
    if (chunked_smem_bytes(T, 128) <= 227u * 1024u)
        return 128;
    if (chunked_smem_bytes(T, 64) <= 227u * 1024u)
        return 64;
    return 0;
}

}  // namespace edm
