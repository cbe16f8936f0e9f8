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
// is FP32 (Algorithm 5's weighted sum; then the rho moment sums).  The FP16
// form feeds the FP16 values straight into mixed-precision FMAs (FP16
// operands, exact FP32 product, FP32 accumulator) with an FP16 copy of each
// weight (the tables stay FP32), so no separate conversion is issued: one
// FMA per gathered value, as in the FP32 form, at half the shared bytes.
#pragma once

#include "bulk_copy.cuh"
#include "edm_internal.cuh"
#include "launchers.h"

namespace edm {

constexpr int kCkWarps = 8;
constexpr int kCkThreads = kCkWarps * 32;
constexpr int kCkRed = 33;

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

// pl += w * lo(u), ph += w * hi(u): FP16 operands, exact FP32 product,
// FP32 accumulation (mixed-precision fma), no separate conversion.
__device__ __forceinline__ void fma_h2(float &pl, float &ph, uint32_t u, uint16_t w)
{
    asm("{.reg .f16 l, h; mov.b32 {l, h}, %2; fma.rn.f32.f16 %0, l, %3, %0; fma.rn.f32.f16 %1, h, %3, %1;}"
        : "+f"(pl), "+f"(ph)
        : "r"(u), "h"(w));
}

// Packed FP32 pairs (two IEEE single operations per instruction; each lane
// of the pair rounds exactly like the scalar operation).
__device__ __forceinline__ unsigned long long pk2(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ void unpk2(unsigned long long r, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}

// (p0, p1) += w * (v0, v1)
__device__ __forceinline__ void fma2(unsigned long long &p, unsigned long long ww, unsigned long long v)
{
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(p) : "l"(ww), "l"(v));
}

// (p0, p1) += (s0, s1)
__device__ __forceinline__ void add2(unsigned long long &p, unsigned long long s)
{
    asm("add.rn.f32x2 %0, %0, %1;" : "+l"(p) : "l"(s));
}

// Pearson moment sums of two slots: S_p += p, S_pp += p*p, S_po += p*o.
__device__ __forceinline__ void mom2(float &sp0, float &sp1, float &spp0, float &spp1, float &spo0, float &spo1,
                                     float p0, float p1, float o0, float o1)
{
    asm("{\n\t.reg .b64 P, O, A;\n\t"
        "mov.b64 P, {%6, %7};\n\tmov.b64 O, {%8, %9};\n\t"
        "mov.b64 A, {%0, %1};\n\tadd.rn.f32x2 A, A, P;\n\tmov.b64 {%0, %1}, A;\n\t"
        "mov.b64 A, {%2, %3};\n\tfma.rn.f32x2 A, P, P, A;\n\tmov.b64 {%2, %3}, A;\n\t"
        "mov.b64 A, {%4, %5};\n\tfma.rn.f32x2 A, P, O, A;\n\tmov.b64 {%4, %5}, A;\n\t}"
        : "+f"(sp0), "+f"(sp1), "+f"(spp0), "+f"(spp1), "+f"(spo0), "+f"(spo1)
        : "f"(p0), "f"(p1), "f"(o0), "f"(o1));
}

// FP16 copy of a weight (round to nearest) as an FMA operand.
__device__ __forceinline__ uint16_t w_f16(float w) { return __half_as_ushort(__float2half_rn(w)); }

// Chunk position a lane starts from: with 128-byte rows the eight lanes of
// a quarter-warp take positions 0..7; with 64-byte rows lanes pair up
// (2l, 2l+1) on position l, so the observation loads (consecutive rows, of
// alternating bank halves) stay conflict-free.
template <int RB>
__device__ __forceinline__ int lane_sub(int lane)
{
    return RB == 128 ? (lane & 7) : ((lane >> 1) & 3);
}

// Slot s of lane k at chunk step c holds target 4*(lane_sub(k) ^ c) + (s & 3)
// of the set; target t of the set gathers slot ((t >> 2) ^ lane_sub(k)) * 4
// + (t & 3) from every lane k.  The 32 lane sums (each over at most a few
// dozen rows) are added as four interleaved chains of eight, then pairwise.
template <int RB>
__device__ __forceinline__ float gather_slot_sum(const float *red, int t)
{
    float s[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const int slot = ((((t >> 2) ^ lane_sub<RB>(k)) << 2) | (t & 3));
        s[k & 3] += red[slot * kCkRed + k];
    }
    return (s[0] + s[1]) + (s[2] + s[3]);
}

// The same for an FP16 pass over half of the chunk positions (128-byte rows,
// chunk steps 4p .. 4p+3): only the 16 lanes k with ((k & 7) >> 2) == p ^
// (t >> 4) hold target t in that pass.
__device__ __forceinline__ float gather_slot_sum_half(const float *red, int t, int p)
{
    const int q = p ^ (t >> 4);
    float s[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k = 8 * j + 4 * q + i;
            const int slot = ((((t >> 2) ^ (k & 7)) << 2) | (t & 3));
            s[i] += red[slot * kCkRed + k];
        }
    return (s[0] + s[1]) + (s[2] + s[3]);
}

// Per-launch constants of the chunked lookup of one tile.
struct CkRows {
    uint32_t base;    // shared address of the tile
    uint32_t lane16;  // this lane's chunk position x 16
    size_t tq_pad;
    int Tq, r_lo, nblk, dshift, lag, L;
};

// Every row block of one library's table for the chunk steps c0 .. c0+NC-1:
// per (lane, slot) FP32 sums of p, p^2 and p*o into Sp/Spp/Spo (NS = 4*NC
// slots; FP16 tiles: lo-set slots 0..NS-1, hi-set slots NS..2NS-1).  kShift:
// every prediction enters the sums as p - K_slot (shn holds -K_slot), the
// shifted sums of an ill-conditioned pair.
template <int K, bool F16, int RB, int NC, bool kShift>
__device__ __forceinline__ void chunk_rows(const CkRows &cx, const float *Wt, const uint16_t *It, int c0,
                                           const float *shn, float *Sp, float *Spp, float *Spo)
{
    constexpr int NS = NC * 4;
    constexpr bool kPref = K <= 16;
    constexpr bool kPref2 = F16 && K <= 5;
    const int lane = lane_id();
    const size_t tq_pad = cx.tq_pad;
    const int Tq = cx.Tq, r_lo = cx.r_lo, dshift = cx.dshift;
    const uint32_t base = cx.base, lane16 = cx.lane16;
#pragma unroll
    for (int r = 0; r < NS * (F16 ? 2 : 1); ++r) {
        Sp[r] = 0.f;
        Spp[r] = 0.f;
        Spo[r] = 0.f;
    }
    // table entries prefetched one row block ahead (two for FP16 with small
    // K: its row blocks are half as long)
    float wq[kPref ? K : 1], wq2[kPref2 ? K : 1];
    uint32_t iq[kPref ? K : 1], iq2[kPref2 ? K : 1];
    if (kPref) {
        const bool v = r_lo + lane < Tq;
#pragma unroll
        for (int n = 0; n < (kPref ? K : 1); ++n) {
            wq[n] = v ? __ldg(Wt + n * tq_pad + r_lo + lane) : 0.f;
            iq[n] = v ? (uint32_t)((int)__ldg(It + n * tq_pad + r_lo + lane) + dshift) : 0u;
        }
    }
    if (kPref2) {
        const bool v = r_lo + lane + 32 < Tq;
#pragma unroll
        for (int n = 0; n < (kPref2 ? K : 1); ++n) {
            wq2[n] = v ? __ldg(Wt + n * tq_pad + r_lo + lane + 32) : 0.f;
            iq2[n] = v ? (uint32_t)((int)__ldg(It + n * tq_pad + r_lo + lane + 32) + dshift) : 0u;
        }
    }
    for (int b = 0; b < cx.nblk; ++b) {
        const int row = r_lo + b * 32 + lane;
        const bool valid = row < Tq;
        float wn[K];
        uint32_t Bn[K];
        if (kPref) {
#pragma unroll
            for (int n = 0; n < (kPref ? K : 1); ++n) {
                wn[n] = wq[n];
                Bn[n] = base + iq[n] * (uint32_t)RB + lane16;
            }
            if (kPref2) {
                const int nrow = row + 64;
                const bool v = nrow < Tq;
#pragma unroll
                for (int n = 0; n < (kPref2 ? K : 1); ++n) {
                    wq[n] = wq2[n];
                    iq[n] = iq2[n];
                    wq2[n] = v ? __ldg(Wt + n * tq_pad + nrow) : 0.f;
                    iq2[n] = v ? (uint32_t)((int)__ldg(It + n * tq_pad + nrow) + dshift) : 0u;
                }
            } else {
                const int nrow = row + 32;
                const bool v = nrow < Tq;
#pragma unroll
                for (int n = 0; n < (kPref ? K : 1); ++n) {
                    wq[n] = v ? __ldg(Wt + n * tq_pad + nrow) : 0.f;
                    iq[n] = v ? (uint32_t)((int)__ldg(It + n * tq_pad + nrow) + dshift) : 0u;
                }
            }
        } else {
#pragma unroll
            for (int n = 0; n < K; ++n) {
                wn[n] = valid ? __ldg(Wt + n * tq_pad + row) : 0.f;
                Bn[n] = base + (valid ? (uint32_t)((int)__ldg(It + n * tq_pad + row) + dshift) : 0u) *
                                   (uint32_t)RB + lane16;
            }
        }
        // an invalid row (past the table) has zero weights and reads row 0 as
        // its observation; its terms are masked below
        const uint32_t orow = valid ? (uint32_t)(cx.L + row + cx.lag) : 0u;
        const uint32_t Bo = base + orow * (uint32_t)RB + lane16;
        uint16_t wh[F16 ? K : 1];
        // packed weight pairs for the FP32 gathers (register budget: small K only)
        constexpr bool kPair = !F16 && K <= 12;
        unsigned long long ww[kPair ? K : 1];
        if (F16) {
#pragma unroll
            for (int n = 0; n < (F16 ? K : 1); ++n)
                wh[n] = w_f16(wn[n]);
        } else if (kPair) {
#pragma unroll
            for (int n = 0; n < (kPair ? K : 1); ++n)
                ww[n] = pk2(wn[n], wn[n]);
        }
#pragma unroll
        for (int cl = 0; cl < NC; ++cl) {
            const uint32_t x = (uint32_t)((c0 + cl) * 16);
            const int sl = cl * 4;
            if (!F16) {
                float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
                if (kPair) {
                    unsigned long long p01 = 0ull, p23 = 0ull;  // (+0.0f, +0.0f)
#pragma unroll
                    for (int n = 0; n < (kPair ? K : 1); ++n) {
                        const float4 v = lds_v4(Bn[n] ^ x);
                        fma2(p01, ww[n], pk2(v.x, v.y));
                        fma2(p23, ww[n], pk2(v.z, v.w));
                    }
                    if (kShift) {
                        add2(p01, pk2(shn[sl], shn[sl + 1]));
                        add2(p23, pk2(shn[sl + 2], shn[sl + 3]));
                    }
                    unpk2(p01, p0, p1);
                    unpk2(p23, p2, p3);
                } else {
#pragma unroll
                    for (int n = 0; n < K; ++n) {
                        const float4 v = lds_v4(Bn[n] ^ x);
                        p0 = fmaf(wn[n], v.x, p0);
                        p1 = fmaf(wn[n], v.y, p1);
                        p2 = fmaf(wn[n], v.z, p2);
                        p3 = fmaf(wn[n], v.w, p3);
                    }
                    if (kShift) {
                        p0 += shn[sl];
                        p1 += shn[sl + 1];
                        p2 += shn[sl + 2];
                        p3 += shn[sl + 3];
                    }
                }
                if (kShift && !valid)
                    p0 = p1 = p2 = p3 = 0.f;
                const float4 o = lds_v4(Bo ^ x);
                mom2(Sp[sl], Sp[sl + 1], Spp[sl], Spp[sl + 1], Spo[sl], Spo[sl + 1], p0, p1, o.x, o.y);
                mom2(Sp[sl + 2], Sp[sl + 3], Spp[sl + 2], Spp[sl + 3], Spo[sl + 2], Spo[sl + 3], p2, p3, o.z, o.w);
            } else {
                float pl[4] = {0.f, 0.f, 0.f, 0.f}, ph[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int n = 0; n < K; ++n) {
                    const uint4 u = lds_u4(Bn[n] ^ x);
                    const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        fma_h2(pl[i], ph[i], uu[i], wh[n]);
                }
                if (kShift) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        pl[i] = valid ? pl[i] + shn[sl + i] : 0.f;
                        ph[i] = valid ? ph[i] + shn[NS + sl + i] : 0.f;
                    }
                }
                const uint4 ou = lds_u4(Bo ^ x);
                const uint32_t oo[4] = {ou.x, ou.y, ou.z, ou.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float2 o = h2f(oo[i]);
                    // lo target (slot sl+i) and hi target (slot NS+sl+i) as one packed pair
                    mom2(Sp[sl + i], Sp[NS + sl + i], Spp[sl + i], Spp[NS + sl + i], Spo[sl + i], Spo[NS + sl + i],
                         pl[i], ph[i], o.x, o.y);
                }
            }
        }
    }
}

// Prediction of table row R for the targets of word `lane` of the tile row
// (FP32: target lane; FP16: targets lane and lane + SET), formed by exactly
// the operations chunk_rows applies to every row, into red[lane] and
// red[32 + lane].  Lanes past the row's words do nothing.
template <int K, bool F16, int RB>
__device__ __forceinline__ void row_prediction(const CkRows &cx, const float *Wt, const uint16_t *It, int R, float *red)
{
    const int lane = lane_id();
    if (lane >= RB / 4)
        return;
    float pl = 0.f, ph = 0.f;
#pragma unroll
    for (int n = 0; n < K; ++n) {
        const float w = __ldg(Wt + n * cx.tq_pad + R);
        const uint32_t g = (uint32_t)((int)__ldg(It + n * cx.tq_pad + R) + cx.dshift);
        uint32_t u;
        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(u) : "r"(cx.base + g * (uint32_t)RB + (uint32_t)lane * 4u));
        if (F16)
            fma_h2(pl, ph, u, w_f16(w));
        else
            pl = fmaf(w, __uint_as_float(u), pl);
    }
    red[lane] = pl;
    red[32 + lane] = ph;
}

// Fold the per-(lane, slot) sums of chunk steps c0 .. c0+NC-1 into
// per-target sums: tot[m][st] (moment m, set st) of target st*SET+lane.
template <bool F16, int RB, int NC>
__device__ __forceinline__ void chunk_fold(float *red, int c0, const float *Sp, const float *Spp, const float *Spo,
                                           float (*tot)[2])
{
    constexpr int CR = RB / 16;
    constexpr int SET = CR * 4;
    constexpr int NS = NC * 4;
    // an FP16 pass over half of a 128-byte row writes and folds only its
    // own chunk positions
    constexpr bool kHalf = RB == 128 && NC == CR / 2;
    const int lane = lane_id();
#pragma unroll
    for (int st = 0; st < (F16 ? 2 : 1); ++st) {
#pragma unroll
        for (int mm = 0; mm < 3; ++mm) {
            const float *S = mm == 0 ? Sp : (mm == 1 ? Spp : Spo);
#pragma unroll
            for (int c = 0; c < CR; ++c)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const bool mine = c >= c0 && c < c0 + NC;
                    const int sl = (F16 ? st * NS : 0) + ((c - c0) & (NC - 1)) * 4 + i;
                    if (mine || !kHalf)
                        red[(c * 4 + i) * kCkRed + lane] = mine ? S[sl] : 0.f;
                }
            __syncwarp();
            if (lane < SET)
                tot[mm][st] += kHalf ? gather_slot_sum_half(red, lane, c0 / NC) : gather_slot_sum<RB>(red, lane);
            __syncwarp();
        }
    }
}

// Negated per-slot shifts -K for chunk steps c0 .. c0+NC-1 from the
// per-target shifts in red[0..63] (FP32 tiles: red[t]; FP16 tiles: lo target
// w at red[w], hi target w+SET at red[32+w]).  Each quarter-warp reads eight
// different 16-byte chunks (no bank conflicts).
template <bool F16, int RB, int NC>
__device__ __forceinline__ void chunk_shifts(const float *red, int c0, float *shn)
{
    constexpr int NS = NC * 4;
    const int ls = lane_sub<RB>(lane_id());
#pragma unroll
    for (int cl = 0; cl < NC; ++cl) {
        const int q = ls ^ (c0 + cl);
        const float4 lo = *reinterpret_cast<const float4 *>(red + 4 * q);
        shn[cl * 4 + 0] = -lo.x;
        shn[cl * 4 + 1] = -lo.y;
        shn[cl * 4 + 2] = -lo.z;
        shn[cl * 4 + 3] = -lo.w;
        if (F16) {
            const float4 hi = *reinterpret_cast<const float4 *>(red + 32 + 4 * q);
            shn[NS + cl * 4 + 0] = -hi.x;
            shn[NS + cl * 4 + 1] = -hi.y;
            shn[NS + cl * 4 + 2] = -hi.z;
            shn[NS + cl * 4 + 3] = -hi.w;
        }
    }
}

// kLag: the time-delay form (tables over t >= s_lo, lag shift); the plain
// instantiation folds those terms away (s_lo = 0, lag = Tp).
template <int K, bool F16, int RB, bool kLag = false>
__device__ __forceinline__ void lookup_chunk_body(const LookupArgs &a, int tile, int part, int parts)
{
    // RB-byte rows hold RB/16 chunks; FP32 chunks are 4 targets, FP16 chunks
    // 4 words = 8 targets (word w = targets w and w + RB/4).  FP16 with
    // 128-byte rows makes two passes over the row blocks, each covering half
    // of the chunk positions (still 8 useful values per 16-byte load), so a
    // lane keeps at most 32 slots per pass.
    constexpr int CR = RB / 16;                    // chunks per row
    constexpr int PASSES = (F16 && RB == 128) ? 2 : 1;
    constexpr int CPP = CR / PASSES;               // chunk steps per pass
    constexpr int SET = CR * 4;                    // targets per set (lo / hi)
    constexpr int HS = CPP * 4;                    // slots per set and pass
    constexpr int CPR = CPP / 2;                   // chunk steps per shifted re-pass
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const uint32_t raw = (uint32_t)__cvta_generic_to_shared(smem_raw);
    const uint32_t pad = (128u - (raw & 127u)) & 127u;
    unsigned char *smem = smem_raw + pad;
    float *red_all = reinterpret_cast<float *>(smem + (size_t)a.T * RB);

    const TileMeta m = a.meta[tile];
    const int E = K - 1;
    CkRows cx;
    cx.base = raw + pad;
    cx.L = (E - 1) * a.tau;
    // table rows [r_lo, Tq): queries t = L + r >= s_lo; gathers at the stored
    // neighbour time + Tp shifted by lag - Tp, observations at t + lag
    cx.Tq = a.T - a.Tp - cx.L;
    cx.r_lo = kLag ? max(0, a.s_lo - cx.L) : 0;
    const int nrows = cx.Tq - cx.r_lo;
    cx.nblk = (nrows + 31) / 32;
    cx.dshift = kLag ? a.lag - a.Tp : 0;
    cx.lag = kLag ? a.lag : a.Tp;
    cx.tq_pad = (size_t)a.lay.Tq_pad;

    {
        // the tile (T rows of RB bytes, 16-byte aligned, a multiple of 16
        // bytes) by one bulk copy into shared memory; the barrier word sits
        // behind the per-warp fold buffers
        const unsigned char *src = reinterpret_cast<const unsigned char *>(a.tiles) + (size_t)tile * a.T * RB;
        const uint32_t bytes = (uint32_t)a.T * (uint32_t)RB;
        const uint32_t bar = cx.base + bytes + (uint32_t)(kCkWarps * 32 * kCkRed * 4);
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            mbar_expect_tx(bar, bytes);
            bulk_g2s(cx.base, src, bytes, bar);
        }
        __syncthreads();
        const bool ok = mbar_wait(bar, 0);
        if (!__syncthreads_and(ok))
            return;
    }

    const int lane = lane_id(), warp = warp_id();
    float *red = red_all + warp * 32 * kCkRed;
    const int per = (a.n_lib + parts - 1) / parts;
    const int lib_lo = part * per;
    const int lib_hi = min(a.n_lib, lib_lo + per);
    cx.lane16 = (uint32_t)lane_sub<RB>(lane) * 16u;

    // table bytes of one (library, E): K weight rows and K index rows of
    // Tq_pad entries (both 16-byte multiples at 16-byte aligned offsets)
    const uint32_t w_bytes = (uint32_t)(K * a.lay.Tq_pad * 4), i_bytes = (uint32_t)(K * a.lay.Tq_pad * 2);
    for (int lib = lib_lo + warp; lib < lib_hi; lib += kCkWarps) {
        const uint8_t *lb = a.tables + (size_t)lib * a.lay.lib_stride;
        const float *Wt = reinterpret_cast<const float *>(lb + a.lay.off_w[E]);
        const uint16_t *It = reinterpret_cast<const uint16_t *>(lb + a.lay.off_i[E]);
        // the warp's next library: its table into L2 while this one runs
        // (tables of a large library block live in HBM)
        if (lane == 0 && lib + kCkWarps < lib_hi) {
            const uint8_t *nb = lb + (size_t)kCkWarps * a.lay.lib_stride;
            bulk_prefetch_l2(nb + a.lay.off_w[E], w_bytes);
            bulk_prefetch_l2(nb + a.lay.off_i[E], i_bytes);
        }
        float tot[3][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 1
        for (int pass = 0; pass < PASSES; ++pass) {
            float Sp[HS * (F16 ? 2 : 1)], Spp[HS * (F16 ? 2 : 1)], Spo[HS * (F16 ? 2 : 1)];
            chunk_rows<K, F16, RB, CPP, false>(cx, Wt, It, pass * CPP, nullptr, Sp, Spp, Spo);
            chunk_fold<F16, RB, CPP>(red, pass * CPP, Sp, Spp, Spo, tot);
        }
        // A pair whose predictions sit far from zero against their spread
        // (a constant or near-constant library gives almost equal
        // predictions) loses digits in n S_pp - S_p^2: sum that library again
        // with every prediction shifted by the prediction of the last table
        // row (formed by the same operations, so equal predictions give
        // exact zeros, and zero variance stays zero).
        bool ill = false;
        float2 om[2];
#pragma unroll
        for (int st = 0; st < (F16 ? 2 : 1); ++st) {
            const int t = st * SET + lane;
            om[st] = (lane < SET && t < m.count) ? a.omom[m.first + t] : make_float2(0.f, 0.f);
            if (om[st].y > 0.f)
                ill |= moments_ill_conditioned(tot[0][st], tot[1][st], nrows);
        }
        if (__any_sync(kFull, ill)) {
#pragma unroll
            for (int mm = 0; mm < 3; ++mm)
                tot[mm][0] = tot[mm][1] = 0.f;
#pragma unroll 1
            for (int c0 = 0; c0 < CR; c0 += CPR) {
                float shn[CPR * 4 * (F16 ? 2 : 1)];
                row_prediction<K, F16, RB>(cx, Wt, It, cx.Tq - 1, red);
                __syncwarp();
                chunk_shifts<F16, RB, CPR>(red, c0, shn);
                __syncwarp();
                float Sp[CPR * 4 * (F16 ? 2 : 1)], Spp[CPR * 4 * (F16 ? 2 : 1)], Spo[CPR * 4 * (F16 ? 2 : 1)];
                chunk_rows<K, F16, RB, CPR, true>(cx, Wt, It, c0, shn, Sp, Spp, Spo);
                chunk_fold<F16, RB, CPR>(red, c0, Sp, Spp, Spo, tot);
            }
        }
#pragma unroll
        for (int st = 0; st < (F16 ? 2 : 1); ++st) {
            const int t = st * SET + lane;
            if (lane < SET && t < m.count) {
                const int64_t j = a.pi[m.first + t];
                a.rho[j * a.ld_rho + a.rho_col0 + lib] =
                    rho_final(tot[0][st], tot[1][st], tot[2][st], om[st].x, om[st].y, nrows);
            }
        }
    }
}

}  // namespace edm
