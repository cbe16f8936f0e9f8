// lookup_kernels.cu -- target staging and the fused lookup + rho kernel.
//
// Lookup (Algorithm 5) and corrcoef for one E-homogeneous tile of 32
// targets and a block of libraries.  The tile ([T][32] floats, time-major,
// targets across the 32 banks) sits in shared memory.  A warp serves one
// library at a time: lane l owns query row t_l = 32b + l of the library's
// table (its E+1 neighbour offsets and weights stay in registers) and, at
// step r = 0..31, forms the prediction of target column l^r.  For a fixed
// r the 32 lanes read 32 different columns, so every gather hits 32
// distinct banks whatever the neighbour rows are.  Moment sums per
// (lane, r) are folded into per-target sums through a small shared
// transpose at the end of the library.  Every prediction enters the sums
// shifted by the prediction of the last table row of its (library, target)
// pair (kept per warp in shared memory, formed by the same operations), so
// nearly constant predictions keep their variance and equal ones give zero
// variance; rho is formed in FP64.
#include "edm_internal.cuh"
#include <cuda_fp16.h>

#include "launchers.h"

namespace edm {

constexpr int kLkWarps = 8;
constexpr int kLkThreads = kLkWarps * 32;
constexpr int kRedStride = 33;

// 128 spare bytes let the tile start on a 128-byte boundary of the shared
// window, which the XOR addressing of the gathers relies on.
size_t lookup_smem_bytes(int T)
{
    return 128 + (size_t)T * 32 * sizeof(float) + (size_t)kLkWarps * 32 * kRedStride * 4 + (size_t)kLkWarps * 32 * 4;
}

// Per-target shift of one library: the prediction of table row R for
// target column `lane` (same operation order as every other row), stored
// at sh[lane].
__device__ __forceinline__ void lookup_row_shift(const float *Wt, const uint16_t *It, size_t tq_pad, int k, int R,
                                                 uint32_t base, float *sh)
{
    const int lane = lane_id();
    float p = 0.f;
    for (int n = 0; n < k; ++n) {
        const float w = __ldg(Wt + (size_t)n * tq_pad + R);
        const uint32_t i = __ldg(It + (size_t)n * tq_pad + R);
        float v;
        asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(base + i * 128u + (uint32_t)lane * 4u));
        p = fmaf(w, v, p);
    }
    __syncwarp();
    sh[lane] = p;
    __syncwarp();
}

// Sum for target `lane` of the per-(lane, slot) sums S[r] of slot r =
// target lane ^ r in every lane (through red; four chains, then pairwise).
__device__ __forceinline__ float fold_xor(float *red, const float *S)
{
    const int lane = lane_id();
#pragma unroll
    for (int r = 0; r < 32; ++r)
        red[r * kRedStride + lane] = S[r];
    __syncwarp();
    float s[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int l2 = 0; l2 < 32; ++l2)
        s[l2 & 3] += red[(lane ^ l2) * kRedStride + l2];
    __syncwarp();
    return (s[0] + s[1]) + (s[2] + s[3]);
}

__device__ __forceinline__ float lds_f32(uint32_t addr)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}

// ---------------------------------------------------------------------------
// Target staging: z-normalise each target (mean/std over the whole series,
// FP64), store tiles [T][32], and the per-target observation moments over
// the window o(t) = z(t+Tp), t in [(E-1)tau, T-1-Tp].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) prep_targets_kernel(const float *__restrict__ Y, int64_t ldY, int T, int tau,
                                                           int Tp, const int32_t *__restrict__ pi,
                                                           const TileMeta *__restrict__ meta, float *__restrict__ tiles,
                                                           float2 *__restrict__ omom, int width)
{
    __shared__ float mu_s[32], inv_s[32];
    const TileMeta m = meta[blockIdx.x];
    if ((m.flags & kTileF16) || m.E == 0)
        return;  // staged by the FP16 kernel, or an unused (planned-empty) tile
    const int lane = lane_id(), warp = warp_id();
    for (int slot = warp; slot < 32; slot += 8) {
        double mu = 0.0, inv = 0.0;
        if (slot < m.count) {
            const float *y = Y + (int64_t)pi[m.first + slot] * ldY;
            double a = 0.0;
            for (int t = lane; t < T; t += 32)
                a += (double)y[t];
            mu = warp_sum_d(a) / (double)T;
            double v = 0.0;
            for (int t = lane; t < T; t += 32) {
                double d = (double)y[t] - mu;
                v += d * d;
            }
            v = warp_sum_d(v) / (double)T;
            inv = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
            // observation moments of the staged (float) values
            const float muf = (float)mu, invf = (float)inv;
            const int L = (m.E - 1) * tau;
            double so = 0.0, soo = 0.0;
            for (int t = L + Tp + lane; t < T; t += 32) {
                float z = (y[t] - muf) * invf;
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
    // rows of `width` targets (32 for 128-byte rows, 16 for 64-byte rows)
    float *tile = tiles + (size_t)blockIdx.x * T * width;
    const int slot = lane;
    if (slot < width) {
        const float *y = slot < m.count ? Y + (int64_t)pi[m.first + slot] * ldY : nullptr;
        const float muf = mu_s[slot], invf = inv_s[slot];
        for (int t = warp; t < T; t += 8) {
            float z = y ? (y[t] - muf) * invf : 0.f;
            tile[(size_t)t * width + slot] = z;
        }
    }
}

// Observation sums at one lag over a table's query window (time-delay form).
__global__ void __launch_bounds__(256) obs_moments_kernel(const float *__restrict__ tiles, int RB,
                                                          const TileMeta *__restrict__ meta, int T, int tau, int Tp,
                                                          int s_lo, int lag, float2 *__restrict__ omom)
{
    const TileMeta m = meta[blockIdx.x];
    if (m.E == 0)
        return;
    const bool f16 = (m.flags & kTileF16) != 0;
    const int words = RB / 4;  // 32-bit words per tile row
    const int L = (m.E - 1) * tau;
    const int t_lo = max(L, s_lo), t_hi = T - 1 - Tp;
    const int lane = lane_id(), warp = warp_id();
    const float *tile = tiles + (size_t)blockIdx.x * T * words;
    for (int slot = warp; slot < m.count; slot += blockDim.x / 32) {
        double so = 0.0, soo = 0.0;
        for (int t = t_lo + lane; t <= t_hi; t += 32) {
            const float *row = tile + (size_t)(t + lag) * words;
            float z;
            if (f16) {
                const uint32_t u = __float_as_uint(row[slot % words]);
                const unsigned short h = (unsigned short)(slot < words ? (u & 0xffffu) : (u >> 16));
                z = __half2float(__ushort_as_half(h));
            } else {
                z = row[slot];
            }
            so += (double)z;
            soo += (double)z * (double)z;
        }
        so = warp_sum_d(so);
        soo = warp_sum_d(soo);
        if (lane == 0) {
            const double n = (double)(t_hi - t_lo + 1);
            omom[m.first + slot] = make_float2((float)so, (float)(n * soo - so * so));
        }
    }
}

cudaError_t launch_obs_moments(const float *tiles, int RB, const TileMeta *meta, int n_tiles, int T, int tau, int Tp,
                               int s_lo, int lag, float2 *omom, cudaStream_t st)
{
    if (n_tiles <= 0)
        return cudaSuccess;
    obs_moments_kernel<<<n_tiles, 256, 0, st>>>(tiles, RB, meta, T, tau, Tp, s_lo, lag, omom);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Lookup + rho.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kLkThreads, 1) lookup_generic_kernel(LookupArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const uint32_t raw = (uint32_t)__cvta_generic_to_shared(smem_raw);
    const uint32_t pad = (128u - (raw & 127u)) & 127u;
    unsigned char *smem = smem_raw + pad;
    float *tile_s = reinterpret_cast<float *>(smem);
    float *red_all = reinterpret_cast<float *>(smem + (size_t)a.T * 32 * sizeof(float));
    float *sh_all = red_all + kLkWarps * 32 * kRedStride;
    const uint32_t base = raw + pad;

    const int tile = a.tile_begin + blockIdx.x;
    const TileMeta m = a.meta[tile];
    const int E = m.E, k = E + 1;
    const int L = (E - 1) * a.tau;
    const int Tq = a.T - a.Tp - L;
    const int nblk = (Tq + 31) / 32;

    {  // stage the tile
        const float4 *src = reinterpret_cast<const float4 *>(a.tiles + (size_t)tile * a.T * 32);
        float4 *dst = reinterpret_cast<float4 *>(tile_s);
        const int n4 = a.T * 8;
        for (int i = threadIdx.x; i < n4; i += blockDim.x)
            dst[i] = __ldg(src + i);
    }
    __syncthreads();

    const int lane = lane_id(), warp = warp_id();
    float *red = red_all + warp * 32 * kRedStride;
    float *sh = sh_all + warp * 32;
    const uint32_t sh_base = (uint32_t)__cvta_generic_to_shared(sh);
    const int per = (a.n_lib + a.lib_parts - 1) / a.lib_parts;
    const int lib_lo = blockIdx.y * per;
    const int lib_hi = min(a.n_lib, lib_lo + per);
    const uint32_t lane4 = (uint32_t)lane * 4u;

    for (int lib = lib_lo + warp; lib < lib_hi; lib += kLkWarps) {
        const uint8_t *lb = a.tables + (size_t)lib * a.lay.lib_stride;
        const float *Wt = reinterpret_cast<const float *>(lb + a.lay.off_w[E]);
        const uint16_t *It = reinterpret_cast<const uint16_t *>(lb + a.lay.off_i[E]);
        lookup_row_shift(Wt, It, (size_t)a.lay.Tq_pad, k, Tq - 1, base, sh);
        float Sp[32], Spp[32], Spo[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            Sp[r] = 0.f;
            Spp[r] = 0.f;
            Spo[r] = 0.f;
        }
        for (int b = 0; b < nblk; ++b) {
            const int row = b * 32 + lane;
            const bool valid = row < Tq;
            float p[32];
#pragma unroll
            for (int r = 0; r < 32; ++r)
                p[r] = 0.f;
            for (int n = 0; n < k; ++n) {
                float wv = 0.f;
                uint32_t iv = 0;
                if (valid) {
                    wv = __ldg(Wt + (size_t)n * a.lay.Tq_pad + row);
                    iv = __ldg(It + (size_t)n * a.lay.Tq_pad + row);
                }
                const uint32_t A = base + iv * 128u + lane4;
#pragma unroll
                for (int r = 0; r < 32; ++r)
                    p[r] = fmaf(wv, lds_f32(A ^ (uint32_t)(r * 4)), p[r]);
            }
            const uint32_t orow = valid ? (uint32_t)(L + row + a.Tp) : 0u;
            const uint32_t Ao = base + orow * 128u + lane4;
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                float o = lds_f32(Ao ^ (uint32_t)(r * 4));
                const float pr = valid ? p[r] - lds_f32(sh_base ^ (uint32_t)(r * 4) ^ lane4) : 0.f;
                Sp[r] += pr;
                Spp[r] = fmaf(pr, pr, Spp[r]);
                Spo[r] = fmaf(pr, o, Spo[r]);
            }
        }
        // per-target sums: target c collects slot c^l of every lane l
        const float t0 = fold_xor(red, Sp), t1 = fold_xor(red, Spp), t2 = fold_xor(red, Spo);
        if (lane < m.count) {
            const int64_t j = a.pi[m.first + lane];
            const float2 om = a.omom[m.first + lane];
            a.rho[j * a.ld_rho + a.rho_col0 + lib] = rho_final(t0, t1, t2, om.x, om.y, Tq);
        }
    }
}

// Fast path for k = E+1 <= kFastK: the row's k neighbour offsets and
// weights live in registers, loaded one t-block ahead so the L2 latency of
// the table overlaps the previous block's gathers; the neighbour loop is
// unrolled so each step r issues k independent gathers.
constexpr int kFastK = 12;

template <int K>
__global__ void __launch_bounds__(kLkThreads, 1) lookup_k_kernel(LookupArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const uint32_t raw = (uint32_t)__cvta_generic_to_shared(smem_raw);
    const uint32_t pad = (128u - (raw & 127u)) & 127u;
    unsigned char *smem = smem_raw + pad;
    float *tile_s = reinterpret_cast<float *>(smem);
    float *red_all = reinterpret_cast<float *>(smem + (size_t)a.T * 32 * sizeof(float));
    float *sh_all = red_all + kLkWarps * 32 * kRedStride;
    const uint32_t base = raw + pad;

    const int tile = a.tile_begin + blockIdx.x;
    const TileMeta m = a.meta[tile];
    const int E = K - 1;
    const int L = (E - 1) * a.tau;
    const int Tq = a.T - a.Tp - L;
    const int nblk = (Tq + 31) / 32;

    {
        const float4 *src = reinterpret_cast<const float4 *>(a.tiles + (size_t)tile * a.T * 32);
        float4 *dst = reinterpret_cast<float4 *>(tile_s);
        const int n4 = a.T * 8;
        for (int i = threadIdx.x; i < n4; i += blockDim.x)
            dst[i] = __ldg(src + i);
    }
    __syncthreads();

    const int lane = lane_id(), warp = warp_id();
    float *red = red_all + warp * 32 * kRedStride;
    float *sh = sh_all + warp * 32;
    const uint32_t sh_base = (uint32_t)__cvta_generic_to_shared(sh);
    const int per = (a.n_lib + a.lib_parts - 1) / a.lib_parts;
    const int lib_lo = blockIdx.y * per;
    const int lib_hi = min(a.n_lib, lib_lo + per);
    const uint32_t lane4 = (uint32_t)lane * 4u;
    const size_t tq_pad = (size_t)a.lay.Tq_pad;

    for (int lib = lib_lo + warp; lib < lib_hi; lib += kLkWarps) {
        const uint8_t *lb = a.tables + (size_t)lib * a.lay.lib_stride;
        const float *Wt = reinterpret_cast<const float *>(lb + a.lay.off_w[E]);
        const uint16_t *It = reinterpret_cast<const uint16_t *>(lb + a.lay.off_i[E]);
        lookup_row_shift(Wt, It, tq_pad, K, Tq - 1, base, sh);
        float Sp[32], Spp[32], Spo[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            Sp[r] = 0.f;
            Spp[r] = 0.f;
            Spo[r] = 0.f;
        }
        float wq[K];
        uint32_t iq[K];
        {
            const bool v = lane < Tq;
#pragma unroll
            for (int n = 0; n < K; ++n) {
                wq[n] = v ? __ldg(Wt + n * tq_pad + lane) : 0.f;
                iq[n] = v ? (uint32_t)__ldg(It + n * tq_pad + lane) : 0u;
            }
        }
        for (int b = 0; b < nblk; ++b) {
            const int row = b * 32 + lane;
            const bool valid = row < Tq;
            float wn[K];
            uint32_t An[K];
#pragma unroll
            for (int n = 0; n < K; ++n) {
                wn[n] = wq[n];
                An[n] = base + iq[n] * 128u + lane4;
            }
            {  // prefetch the next block's entries
                const int nrow = row + 32;
                const bool v = nrow < Tq;
#pragma unroll
                for (int n = 0; n < K; ++n) {
                    wq[n] = v ? __ldg(Wt + n * tq_pad + nrow) : 0.f;
                    iq[n] = v ? (uint32_t)__ldg(It + n * tq_pad + nrow) : 0u;
                }
            }
            const uint32_t orow = valid ? (uint32_t)(L + row + a.Tp) : 0u;
            const uint32_t Ao = base + orow * 128u + lane4;
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const uint32_t x = (uint32_t)(r * 4);
                float p = 0.f;
#pragma unroll
                for (int n = 0; n < K; ++n)
                    p = fmaf(wn[n], lds_f32(An[n] ^ x), p);
                const float o = lds_f32(Ao ^ x);
                p = valid ? p - lds_f32(sh_base ^ x ^ lane4) : 0.f;
                Sp[r] += p;
                Spp[r] = fmaf(p, p, Spp[r]);
                Spo[r] = fmaf(p, o, Spo[r]);
            }
        }
        const float t0 = fold_xor(red, Sp), t1 = fold_xor(red, Spp), t2 = fold_xor(red, Spo);
        if (lane < m.count) {
            const int64_t j = a.pi[m.first + lane];
            const float2 om = a.omom[m.first + lane];
            a.rho[j * a.ld_rho + a.rho_col0 + lib] = rho_final(t0, t1, t2, om.x, om.y, Tq);
        }
    }
}

cudaError_t launch_prep_targets(const float *Y, int64_t ldY, int T, int tau, int Tp, const int32_t *pi,
                                const TileMeta *meta, int n_tiles, float *tiles, float2 *omom, cudaStream_t st, int RB)
{
    if (n_tiles <= 0)
        return cudaSuccess;
    prep_targets_kernel<<<n_tiles, 256, 0, st>>>(Y, ldY, T, tau, Tp, pi, meta, tiles, omom, RB / 4);
    return cudaGetLastError();
}

template <class Kern>
static cudaError_t launch_one(Kern kern, const LookupArgs &a, cudaStream_t st)
{
    size_t smem = lookup_smem_bytes(a.T);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    dim3 grid((unsigned)a.n_tiles, (unsigned)a.lib_parts);
    kern<<<grid, kLkThreads, smem, st>>>(a);
    return cudaGetLastError();
}

int lookup_fast_k() { return kFastK; }

// All tiles of `a` must share one E (the caller splits blocks into runs).
cudaError_t launch_lookup(const LookupArgs &a, int E, cudaStream_t st)
{
    if (a.n_tiles <= 0 || a.n_lib <= 0)
        return cudaSuccess;
    switch (E + 1) {
    case 2: return launch_one(lookup_k_kernel<2>, a, st);
    case 3: return launch_one(lookup_k_kernel<3>, a, st);
    case 4: return launch_one(lookup_k_kernel<4>, a, st);
    case 5: return launch_one(lookup_k_kernel<5>, a, st);
    case 6: return launch_one(lookup_k_kernel<6>, a, st);
    case 7: return launch_one(lookup_k_kernel<7>, a, st);
    case 8: return launch_one(lookup_k_kernel<8>, a, st);
    case 9: return launch_one(lookup_k_kernel<9>, a, st);
    case 10: return launch_one(lookup_k_kernel<10>, a, st);
    case 11: return launch_one(lookup_k_kernel<11>, a, st);
    case 12: return launch_one(lookup_k_kernel<12>, a, st);
    default: return launch_one(lookup_generic_kernel, a, st);
    }
}

}  // namespace edm
