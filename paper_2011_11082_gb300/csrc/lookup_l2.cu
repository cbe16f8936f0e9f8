// lookup_l2.cu -- fused lookup + rho (Algorithm 5 and corrcoef) for series
// too long for a target tile to sit in shared memory (a tile of T rows above
// the 227 KB a CTA can hold even with 64-byte rows, i.e. T beyond about
// 3,100 steps).
//
// The FP32 tile ([T][32] z-normalised targets, 128-byte time rows) stays in
// global memory; the host cuts each E group of tiles into target blocks of
// about 64 MB, so the tiles of a block stay in L2 while every library block
// sweeps them.  The gathers
// are laid out for the L2 -> SM path rather than for shared-memory banks:
// the eight lanes of a lane group read the eight 16-byte chunks of ONE
// neighbour row, so every gather instruction of a warp fetches four whole
// 128-byte lines (no partly used sectors), and lane g of a group owns
// targets 4g .. 4g+3 of the tile.  A warp serves one library at a time; its
// four lane groups take four query rows per step.  Each lane loads the
// table entries (weight, neighbour time) of one query row per 32-row block,
// one block ahead, and the groups fetch the entries of their current row by
// warp shuffles.  Moment sums are two-level (per 32-row block, then over
// blocks) so the FP32 error stays small at T in the tens of thousands, of
// predictions shifted by the prediction of the last table row (so nearly
// constant predictions keep their variance and equal ones give zero
// variance); rho is formed in FP64.
#include <algorithm>

#include "edm_internal.cuh"
#include "launchers.h"

namespace edm {

constexpr int kL2Warps = 8;
constexpr int kL2Threads = kL2Warps * 32;

// Tiles whose rows do not fit shared memory (any row width) take this path.
bool lookup_needs_l2(int T) { return chunked_row_bytes(T) == 0; }

__device__ __forceinline__ float4 ldg_v4(const float4 *p)
{
    float4 v;
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

// kLag: the time-delay form (tables over t >= s_lo; gathers at the stored
// neighbour time shifted by lag - Tp, observations at t + lag).
template <int K, bool kLag>
__device__ __forceinline__ void lookup_l2_body(const LookupArgs &a, int tile, int part, int parts)
{
    const TileMeta m = a.meta[tile];
    const int E = K - 1;
    const int L = (E - 1) * a.tau;
    const int Tq = a.T - a.Tp - L;
    const int r_lo = kLag ? max(0, a.s_lo - L) : 0;
    const int nrows = Tq - r_lo;
    const int nblk = (nrows + 31) / 32;
    const int dshift = kLag ? a.lag - a.Tp : 0;
    const int lag = kLag ? a.lag : a.Tp;

    // 8 float4 chunks per 128-byte time row
    const float4 *tl = reinterpret_cast<const float4 *>(a.tiles) + (size_t)tile * a.T * 8;
    const int lane = lane_id(), warp = warp_id();
    const int grp = lane >> 3, sub = lane & 7;
    const int per = (a.n_lib + parts - 1) / parts;
    const int lib_lo = part * per;
    const int lib_hi = min(a.n_lib, lib_lo + per);
    const size_t tq_pad = (size_t)a.lay.Tq_pad;
    const float4 *tsub = tl + sub;

    for (int lib = lib_lo + warp; lib < lib_hi; lib += kL2Warps) {
        const uint8_t *lb = a.tables + (size_t)lib * a.lay.lib_stride;
        const float *Wt = reinterpret_cast<const float *>(lb + a.lay.off_w[E]);
        const uint16_t *It = reinterpret_cast<const uint16_t *>(lb + a.lay.off_i[E]);
        // moments of targets 4*sub + i over this group's rows
        float Sp[4], Spp[4], Spo[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            Sp[i] = 0.f;
            Spp[i] = 0.f;
            Spo[i] = 0.f;
        }
        // shift: the prediction of the last table row (same operations as
        // every other row), subtracted from every prediction
        float4 shn;
        {
            float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
            const int R = Tq - 1;
#pragma unroll
            for (int n = 0; n < K; ++n) {
                const float w = __ldg(Wt + n * tq_pad + R);
                const int off = ((int)__ldg(It + n * tq_pad + R) + dshift) * 8;
                const float4 v = ldg_v4(tsub + off);
                p.x = fmaf(w, v.x, p.x);
                p.y = fmaf(w, v.y, p.y);
                p.z = fmaf(w, v.z, p.z);
                p.w = fmaf(w, v.w, p.w);
            }
            shn = make_float4(-p.x, -p.y, -p.z, -p.w);
        }
        // table entries of row r_lo + 32 b + lane (row offsets in float4 units)
        float wq[K];
        int iq[K];
        {
            const int row = r_lo + lane;
            const bool v = row < Tq;
#pragma unroll
            for (int n = 0; n < K; ++n) {
                wq[n] = v ? __ldg(Wt + n * tq_pad + row) : 0.f;
                iq[n] = v ? ((int)__ldg(It + n * tq_pad + row) + dshift) * 8 : 0;
            }
        }
        for (int b = 0; b < nblk; ++b) {
            float wn[K];
            int in[K];
#pragma unroll
            for (int n = 0; n < K; ++n) {
                wn[n] = wq[n];
                in[n] = iq[n];
            }
            {
                const int row = r_lo + (b + 1) * 32 + lane;
                const bool v = row < Tq;
#pragma unroll
                for (int n = 0; n < K; ++n) {
                    wq[n] = v ? __ldg(Wt + n * tq_pad + row) : 0.f;
                    iq[n] = v ? ((int)__ldg(It + n * tq_pad + row) + dshift) * 8 : 0;
                }
            }
            float bp[4] = {0.f, 0.f, 0.f, 0.f}, bpp[4] = {0.f, 0.f, 0.f, 0.f}, bpo[4] = {0.f, 0.f, 0.f, 0.f};
            constexpr int kU = K <= 9 ? 2 : 1;  // register budget: large K unrolled once
#pragma unroll kU
            for (int q = 0; q < 8; ++q) {
                const int src = q * 4 + grp;  // lane holding this group's row
                const int row = r_lo + b * 32 + src;
                float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int n = 0; n < K; ++n) {
                    const float w = __shfl_sync(kFull, wn[n], src);
                    const int off = __shfl_sync(kFull, in[n], src);
                    const float4 v = ldg_v4(tsub + off);
                    p.x = fmaf(w, v.x, p.x);
                    p.y = fmaf(w, v.y, p.y);
                    p.z = fmaf(w, v.z, p.z);
                    p.w = fmaf(w, v.w, p.w);
                }
                if (row < Tq) {
                    const float4 o = ldg_v4(tsub + (size_t)(L + row + lag) * 8);
                    const float pp[4] = {p.x + shn.x, p.y + shn.y, p.z + shn.z, p.w + shn.w};
                    const float oo[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        bp[i] += pp[i];
                        bpp[i] = fmaf(pp[i], pp[i], bpp[i]);
                        bpo[i] = fmaf(pp[i], oo[i], bpo[i]);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                Sp[i] += bp[i];
                Spp[i] += bpp[i];
                Spo[i] += bpo[i];
            }
        }
        // fold the four lane groups (lanes sub, sub+8, sub+16, sub+24)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int o = 8; o <= 16; o <<= 1) {
                Sp[i] += __shfl_xor_sync(kFull, Sp[i], o);
                Spp[i] += __shfl_xor_sync(kFull, Spp[i], o);
                Spo[i] += __shfl_xor_sync(kFull, Spo[i], o);
            }
        }
        if (lane < 8) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int t = 4 * lane + i;
                if (t < m.count) {
                    const int64_t j = a.pi[m.first + t];
                    const float2 om = a.omom[m.first + t];
                    a.rho[j * a.ld_rho + a.rho_col0 + lib] = rho_final(Sp[i], Spp[i], Spo[i], om.x, om.y, nrows);
                }
            }
        }
    }
}

// One launch per register class over that class's tiles (mixed E within
// the class): each CTA runs the variant of its own tile; a tile of the other
// class (never launched here by launch_lookup_l2) would return at once.
// Small K = E + 1 (<= kL2SplitK) keeps two CTAs per SM within 128
// registers; larger K gets the registers of one CTA.
template <bool kLag, bool kLarge>
__global__ void __launch_bounds__(kL2Threads, kLarge ? 1 : 2) lookup_l2_kernel(LookupArgs a)
{
    int tile, part, parts;
    if (!lookup_item(a, tile, part, parts))
        return;
    const TileMeta m = a.meta[tile];
    const int K = m.E + 1;
    if (K < 2 || (K > kL2SplitK) != kLarge)
        return;
#define EDM_L2(KK)                                                                                                     \
    case KK: lookup_l2_body<KK, kLag>(a, tile, part, parts); break;
    if (!kLarge) {
        switch (K) {
            EDM_L2(2)
            EDM_L2(3)
            EDM_L2(4)
            EDM_L2(5)
            EDM_L2(6)
            EDM_L2(7)
            EDM_L2(8)
            EDM_L2(9)
        default: break;
        }
    } else {
        switch (K) {
            EDM_L2(10)
            EDM_L2(11)
            EDM_L2(12)
            EDM_L2(13)
            EDM_L2(14)
            EDM_L2(15)
            EDM_L2(16)
            EDM_L2(17)
            EDM_L2(18)
            EDM_L2(19)
            EDM_L2(20)
            EDM_L2(21)
        default: break;
        }
    }
#undef EDM_L2
}

cudaError_t launch_lookup_l2(const LookupArgs &a, int n_small, int sms, cudaStream_t st)
{
    if (a.n_tiles <= 0 || a.n_lib <= 0)
        return cudaSuccess;
    const bool lag = a.s_lo != 0 || a.lag != a.Tp;
    // each class gets its own library split, sized so that its tiles alone
    // fill the GPU (two resident CTAs per SM for small K, one for large K);
    // device-planned slots: both launches span the slot's tiles (a CTA of
    // the other class returns), the split sized for the slot
    for (int large = 0; large < 2; ++large) {
        LookupArgs b = a;
        dim3 grid;
        if (a.slot) {
            grid = dim3((unsigned)a.n_tiles);
            b.want = a.want * (large ? 1 : 2);
        } else {
            b.tile_begin = a.tile_begin + (large ? n_small : 0);
            b.n_tiles = large ? a.n_tiles - n_small : n_small;
            if (b.n_tiles <= 0)
                continue;
            const int want = 4 * sms * (large ? 1 : 2);
            b.lib_parts = std::max(1, std::min((want + b.n_tiles - 1) / b.n_tiles, (a.n_lib + 7) / 8));
            grid = dim3((unsigned)b.n_tiles, (unsigned)b.lib_parts);
        }
        if (lag) {
            if (large)
                lookup_l2_kernel<true, true><<<grid, kL2Threads, 0, st>>>(b);
            else
                lookup_l2_kernel<true, false><<<grid, kL2Threads, 0, st>>>(b);
        } else {
            if (large)
                lookup_l2_kernel<false, true><<<grid, kL2Threads, 0, st>>>(b);
            else
                lookup_l2_kernel<false, false><<<grid, kL2Threads, 0, st>>>(b);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

}  // namespace edm
