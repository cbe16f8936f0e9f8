// lookup_chunked.cu -- fused lookup + rho with 16-byte chunked gathers, for
// FP32 target tiles (32 targets per 128-byte row) and FP16 target tiles (64
// targets per row; 32-bit word w holds targets w and w+32).
//
// Each lane owns one query row t of the library's table (E+1 neighbour
// offsets and weights in registers, prefetched one row block ahead).  At
// step c = 0..7 the lane reads, from every neighbour row, the 16-byte chunk
// q = (lane & 7) ^ c of that row: within each quarter-warp the eight lanes
// read eight different chunks, i.e. all 32 banks once, whatever the rows --
// so the gathers run at full shared-memory bandwidth with one load and one
// address operation per 4 (FP32) or 8 (FP16) target values.  Accumulation
// is FP32 (Algorithm 5's weighted sum; then the rho moment sums); the FP16
// form converts each gathered value to FP32 before use.
#include "edm_internal.cuh"
#include "launchers.h"

namespace edm {

constexpr int kCkWarps = 8;
constexpr int kCkThreads = kCkWarps * 32;
constexpr int kCkRed = 33;

size_t chunked_smem_bytes(int T) { return 128 + (size_t)T * 128 + (size_t)kCkWarps * 32 * kCkRed * 4; }

__device__ __forceinline__ float4 lds_v4(uint32_t addr)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}

__device__ __forceinline__ uint4 lds_u4(uint32_t addr)
{
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
    return v;
}

__device__ __forceinline__ float2 h2f(uint32_t u)
{
    __half2 h = *reinterpret_cast<__half2 *>(&u);
    return __half22float2(h);
}

// slot s of lane k at step c holds target 4*((k & 7) ^ c) + (s & 3) of the
// set; target t of the set gathers slot ((t >> 2) ^ (k & 7)) * 4 + (t & 3)
// from every lane k.
__device__ __forceinline__ float gather_slot_sum(const float *red, int t)
{
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const int slot = ((((t >> 2) ^ (k & 7)) << 2) | (t & 3));
        s += red[slot * kCkRed + k];
    }
    return s;
}

template <int K, bool F16>
__global__ void __launch_bounds__(kCkThreads, 1) lookup_chunk_kernel(LookupArgs a)
{
    constexpr int NS = F16 ? 64 : 32;  // slots (targets) per lane
    // prefetching the next row block's entries costs 2K registers; the FP16
    // form (192 accumulators) affords it only for small K
    constexpr bool kPref = F16 ? (K <= 4) : (K <= 16);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const uint32_t raw = (uint32_t)__cvta_generic_to_shared(smem_raw);
    const uint32_t pad = (128u - (raw & 127u)) & 127u;
    unsigned char *smem = smem_raw + pad;
    float *red_all = reinterpret_cast<float *>(smem + (size_t)a.T * 128);
    const uint32_t base = raw + pad;

    const int tile = a.tile_begin + blockIdx.x;
    const TileMeta m = a.meta[tile];
    const int E = K - 1;
    const int L = (E - 1) * a.tau;
    const int Tq = a.T - a.Tp - L;
    const int nblk = (Tq + 31) / 32;

    {
        const float4 *src = reinterpret_cast<const float4 *>(
            reinterpret_cast<const unsigned char *>(a.tiles) + (size_t)tile * a.T * 128);
        float4 *dst = reinterpret_cast<float4 *>(smem);
        const int n4 = a.T * 8;
        for (int i = threadIdx.x; i < n4; i += blockDim.x)
            dst[i] = __ldg(src + i);
    }
    __syncthreads();

    const int lane = lane_id(), warp = warp_id();
    float *red = red_all + warp * 32 * kCkRed;
    const int per = (a.n_lib + a.lib_parts - 1) / a.lib_parts;
    const int lib_lo = blockIdx.y * per;
    const int lib_hi = min(a.n_lib, lib_lo + per);
    const uint32_t lane16 = (uint32_t)(lane & 7) * 16u;
    const size_t tq_pad = (size_t)a.lay.Tq_pad;

    for (int lib = lib_lo + warp; lib < lib_hi; lib += kCkWarps) {
        const uint8_t *lb = a.tables + (size_t)lib * a.lay.lib_stride;
        const float *Wt = reinterpret_cast<const float *>(lb + a.lay.off_w[E]);
        const uint16_t *It = reinterpret_cast<const uint16_t *>(lb + a.lay.off_i[E]);
        float Sp[NS], Spp[NS], Spo[NS];
#pragma unroll
        for (int r = 0; r < NS; ++r) {
            Sp[r] = 0.f;
            Spp[r] = 0.f;
            Spo[r] = 0.f;
        }
        float wq[kPref ? K : 1];
        uint32_t iq[kPref ? K : 1];
        if (kPref) {
            const bool v = lane < Tq;
#pragma unroll
            for (int n = 0; n < (kPref ? K : 1); ++n) {
                wq[n] = v ? __ldg(Wt + n * tq_pad + lane) : 0.f;
                iq[n] = v ? (uint32_t)__ldg(It + n * tq_pad + lane) : 0u;
            }
        }
        for (int b = 0; b < nblk; ++b) {
            const int row = b * 32 + lane;
            const bool valid = row < Tq;
            float wn[K];
            uint32_t Bn[K];
            if (kPref) {
#pragma unroll
                for (int n = 0; n < (kPref ? K : 1); ++n) {
                    wn[n] = wq[n];
                    Bn[n] = base + iq[n] * 128u + lane16;
                }
                const int nrow = row + 32;
                const bool v = nrow < Tq;
#pragma unroll
                for (int n = 0; n < (kPref ? K : 1); ++n) {
                    wq[n] = v ? __ldg(Wt + n * tq_pad + nrow) : 0.f;
                    iq[n] = v ? (uint32_t)__ldg(It + n * tq_pad + nrow) : 0u;
                }
            } else {
#pragma unroll
                for (int n = 0; n < K; ++n) {
                    wn[n] = valid ? __ldg(Wt + n * tq_pad + row) : 0.f;
                    Bn[n] = base + (valid ? (uint32_t)__ldg(It + n * tq_pad + row) : 0u) * 128u + lane16;
                }
            }
            const uint32_t orow = valid ? (uint32_t)(L + row + a.Tp) : 0u;
            const uint32_t Bo = base + orow * 128u + lane16;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const uint32_t x = (uint32_t)(c * 16);
                if (!F16) {
                    float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll
                    for (int n = 0; n < K; ++n) {
                        const float4 v = lds_v4(Bn[n] ^ x);
                        p0 = fmaf(wn[n], v.x, p0);
                        p1 = fmaf(wn[n], v.y, p1);
                        p2 = fmaf(wn[n], v.z, p2);
                        p3 = fmaf(wn[n], v.w, p3);
                    }
                    const float4 o = lds_v4(Bo ^ x);
                    const float pp[4] = {p0, p1, p2, p3};
                    const float oo[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int s = c * 4 + i;
                        Sp[s] += pp[i];
                        Spp[s] = fmaf(pp[i], pp[i], Spp[s]);
                        Spo[s] = fmaf(pp[i], oo[i], Spo[s]);
                    }
                } else {
                    float pl[4] = {0.f, 0.f, 0.f, 0.f}, ph[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int n = 0; n < K; ++n) {
                        const uint4 u = lds_u4(Bn[n] ^ x);
                        const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float2 f = h2f(uu[i]);
                            pl[i] = fmaf(wn[n], f.x, pl[i]);
                            ph[i] = fmaf(wn[n], f.y, ph[i]);
                        }
                    }
                    const uint4 ou = lds_u4(Bo ^ x);
                    const uint32_t oo[4] = {ou.x, ou.y, ou.z, ou.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float2 o = h2f(oo[i]);
                        const int s = c * 4 + i;
                        Sp[s] += pl[i];
                        Spp[s] = fmaf(pl[i], pl[i], Spp[s]);
                        Spo[s] = fmaf(pl[i], o.x, Spo[s]);
                        Sp[32 + s] += ph[i];
                        Spp[32 + s] = fmaf(ph[i], ph[i], Spp[32 + s]);
                        Spo[32 + s] = fmaf(ph[i], o.y, Spo[32 + s]);
                    }
                }
            }
        }
        // fold the per-(lane, slot) sums into per-target sums
#pragma unroll
        for (int set = 0; set < NS / 32; ++set) {
            float tot[3];
#pragma unroll
            for (int mm = 0; mm < 3; ++mm) {
                const float *S = mm == 0 ? Sp : (mm == 1 ? Spp : Spo);
#pragma unroll
                for (int r = 0; r < 32; ++r)
                    red[r * kCkRed + lane] = S[set * 32 + r];
                __syncwarp();
                tot[mm] = gather_slot_sum(red, lane);
                __syncwarp();
            }
            const int t = set * 32 + lane;
            if (t < m.count) {
                const int64_t j = a.pi[m.first + t];
                const float2 om = a.omom[m.first + t];
                const float n = (float)Tq;
                const float num = n * tot[2] - tot[0] * om.x;
                const float den_p = n * tot[1] - tot[0] * tot[0];
                const float rho = (den_p > 0.f && om.y > 0.f) ? num / sqrtf(den_p * om.y) : CUDART_NAN_F;
                a.rho[j * a.ld_rho + a.rho_col0 + lib] = rho;
            }
        }
    }
}

template <class Kern>
static cudaError_t launch_ck(Kern kern, const LookupArgs &a, cudaStream_t st)
{
    size_t smem = chunked_smem_bytes(a.T);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    dim3 grid((unsigned)a.n_tiles, (unsigned)a.lib_parts);
    kern<<<grid, kCkThreads, smem, st>>>(a);
    return cudaGetLastError();
}

int chunked_max_k(bool f16) { return f16 ? kF16MaxK : EDM_MAX_E + 1; }

#define EDM_CK_CASE(KK)                                                                                                \
    case KK:                                                                                                           \
        return f16 ? (KK <= kF16MaxK ? launch_ck(lookup_chunk_kernel<(KK <= kF16MaxK ? KK : 2), true>, a, st)          \
                                     : cudaErrorInvalidValue)                                                          \
                   : launch_ck(lookup_chunk_kernel<KK, false>, a, st);

cudaError_t launch_lookup_chunked(const LookupArgs &a, int E, bool f16, cudaStream_t st)
{
    if (a.n_tiles <= 0 || a.n_lib <= 0)
        return cudaSuccess;
    switch (E + 1) {
        EDM_CK_CASE(2)
        EDM_CK_CASE(3)
        EDM_CK_CASE(4)
        EDM_CK_CASE(5)
        EDM_CK_CASE(6)
        EDM_CK_CASE(7)
        EDM_CK_CASE(8)
        EDM_CK_CASE(9)
        EDM_CK_CASE(10)
        EDM_CK_CASE(11)
        EDM_CK_CASE(12)
        EDM_CK_CASE(13)
        EDM_CK_CASE(14)
        EDM_CK_CASE(15)
        EDM_CK_CASE(16)
        EDM_CK_CASE(17)
        EDM_CK_CASE(18)
        EDM_CK_CASE(19)
        EDM_CK_CASE(20)
        EDM_CK_CASE(21)
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// FP16 staging: 64 targets per tile, z-normalised in FP64 then rounded to
// FP16; the observation moments are taken over the rounded values (what the
// lookup reads).  Tiles without the FP16 flag are left to the FP32 stager.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) prep_targets_f16_kernel(const float *__restrict__ Y, int64_t ldY, int T, int tau,
                                                               int Tp, const int32_t *__restrict__ pi,
                                                               const TileMeta *__restrict__ meta, uint8_t *__restrict__ tiles,
                                                               float2 *__restrict__ omom)
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
    uint32_t *tile = reinterpret_cast<uint32_t *>(tiles + (size_t)blockIdx.x * T * 128);
    const float *ylo = lane < m.count ? Y + (int64_t)pi[m.first + lane] * ldY : nullptr;
    const float *yhi = lane + 32 < m.count ? Y + (int64_t)pi[m.first + lane + 32] * ldY : nullptr;
    const float mlo = mu_s[lane], ilo = inv_s[lane], mhi = mu_s[lane + 32], ihi = inv_s[lane + 32];
    for (int t = warp; t < T; t += 8) {
        float zl = ylo ? (ylo[t] - mlo) * ilo : 0.f;
        float zh = yhi ? (yhi[t] - mhi) * ihi : 0.f;
        __half2 h = __floats2half2_rn(zl, zh);
        tile[(size_t)t * 32 + lane] = *reinterpret_cast<uint32_t *>(&h);
    }
}

cudaError_t launch_prep_targets_f16(const float *Y, int64_t ldY, int T, int tau, int Tp, const int32_t *pi,
                                    const TileMeta *meta, int n_tiles, uint8_t *tiles, float2 *omom, cudaStream_t st)
{
    if (n_tiles <= 0)
        return cudaSuccess;
    prep_targets_f16_kernel<<<n_tiles, 256, 0, st>>>(Y, ldY, T, tau, Tp, pi, meta, tiles, omom);
    return cudaGetLastError();
}

}  // namespace edm
