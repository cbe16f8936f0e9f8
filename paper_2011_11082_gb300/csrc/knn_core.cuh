// knn_core.cuh -- warp-cooperative exact kNN over all embedding dimensions.
//
// One warp serves one query point t.  Lane l owns the candidate slots
// s = s_first + c0 + l + 32 j (j < J) of the current chunk and keeps their
// squared distances in registers.  The distance grows by one lag per E
// (d2_E = d2_{E-1} + (x_q(t-(E-1)tau) - x_c(s-(E-1)tau))^2), so one sweep
// over the candidates serves every E in 1..E_lim; a bit mask selects the E
// whose neighbour lists are wanted (Sec. III-B: one table per E, Algorithm 2).
//
// Selection per (query, E), K = E+1+kGuard: a threshold th that at least K
// real candidates meet -- the smaller of the previous E's list grown by one
// lag (recomputed in the lanes' FP32 order), this E's list of earlier
// chunks, and the K-th smallest of the 32 lane minima; if more candidates
// than the buffer holds fall under it, counting rounds on the registers
// lower it.  The distances go to a per-warp shared scratch, each lane marks
// its slots at or below th in a bit mask, the marked candidates are
// compacted (exclusive warp scan of per-lane counts), ranked by (d2, s) and
// kept as a sorted list carried to the next chunk.  The hot loop stays
// small: rare paths are out of line.
// The list stores K+1 entries: the first K are the exact K smallest; the
// extra one is a real candidate that lets the next E seed its threshold.
//
// Exactness (neighbours identical to the FP64 reference): the FP32 sum has a
// known error bound (d2_err).  When every gap among the first E+2 entries
// exceeds the bounds, the FP32 order is the FP64 order.  Otherwise the kept
// entries are re-ranked with FP64 distances computed in the reference's
// operation order; if even the guard entries cannot separate the k-th place
// from the rest, the query falls back to an exhaustive FP64 selection.
#pragma once

#include "edm_internal.cuh"

namespace edm {

// Queries that needed the FP64 re-rank ([0]) and the exhaustive FP64 scan
// ([1]) since the last read (edm_knn_counters); rare-path accounting only.
static __device__ unsigned long long g_knn_counts[2];

// list capacity for E is E + 2 + kGuard (= K + 1)
__host__ __device__ constexpr int list_off(int E) { return (E - 1) * E / 2 + (E - 1) * (2 + kGuard); }
constexpr int kListTotal = list_off(EDM_MAX_E + 1);

struct __align__(16) KnnWarpScratch {
    unsigned long long ck[kCandCap];  // buffered candidates as dkey(d2, s)
    float ld[kListTotal];
    int ls[kListTotal];
    double l64[kKmax];
    int ls64[kKmax];
    int lcount[EDM_MAX_E + 1];
    int ovf[EDM_MAX_E + 1];
    int cnt;
    int pad;
};

struct KnnQuery {
    const float *xq;  // query series (shared memory)
    const float *xc;  // candidate series (shared memory); readable from
                      // xc[-(E_lim-1)*tau] to xc[s_first + 32*J*chunks - 1];
                      // the padding holds +inf, so a candidate whose lag
                      // falls before the series start gets distance +inf
    int t;            // query time in xq
    int s_first;      // first candidate time (slot 0)
    int s_last;       // last candidate time
    int tau;
    int same;         // xq and xc are the same series (apply the exclusion radius)
    int excl;
    int E_lim;        // distances are grown for E = 1..E_lim
    uint32_t sel;     // bit E-1: produce the neighbour list for E
    float *d2s;       // this warp's distance scratch (shared): 32 * J floats,
                      // slot j of lane l at d2s[(j/4)*128 + l*4 + j%4]
    const uint32_t *mask;  // optional candidate subset (bit s of word s/32)
};

// Per-warp distance scratch bytes for J register slots per lane.
__host__ __device__ constexpr size_t knn_d2s_bytes(int J) { return (size_t)32 * J * sizeof(float); }

// FP64 squared distance in the reference's operation order.
__device__ __forceinline__ double dist64(const float *xq, int t, const float *xc, int s, int E, int tau)
{
    double d = 0.0;
    for (int m = 0; m < E; ++m) {
        double diff = __dsub_rn((double)xq[t - m * tau], (double)xc[s - m * tau]);
        d = __dadd_rn(d, __dmul_rn(diff, diff));
    }
    return d;
}

__device__ __forceinline__ bool cand_ok(const KnnQuery &q, int s, int E)
{
    if (s < q.s_first || s > q.s_last || s < (E - 1) * q.tau)
        return false;
    if (q.same && q.excl >= 0 && abs(s - q.t) <= q.excl)
        return false;
    if (q.mask && !((__ldg(q.mask + (s >> 5)) >> (s & 31)) & 1u))
        return false;
    return true;
}

// FP32 squared distance of candidate s at dimension E in the lanes'
// operation order (zero start, one fma per lag, lags 0..E-1): bitwise equal
// to the incrementally grown register value.
__device__ __forceinline__ float dist32(const KnnQuery &q, int s, int E)
{
    float d = 0.f;
    for (int m = 0; m < E; ++m) {
        float diff = q.xq[q.t - m * q.tau] - q.xc[s - m * q.tau];
        d = fmaf(diff, diff, d);
    }
    return d;
}

// K-th smallest of the 32 lane minima (every lane minimum is a real
// candidate).  Small K: K rounds of a warp minimum on the (order-preserving)
// bit patterns of the non-negative distances; large K: a bitonic sort.
__device__ __forceinline__ float kth_lane_min(float mn, int K)
{
    if (K <= 12) {
        unsigned v = __float_as_uint(mn);
        unsigned m = 0u;
        int got = 0;
        while (got < K) {  // warp-uniform
            m = __reduce_min_sync(kFull, v);
            const unsigned hit = __ballot_sync(kFull, v == m);
            got += __popc(hit);
            if (v == m)
                v = 0xffffffffu;
            if (m == 0x7f800000u)  // +inf: fewer than K finite lane minima
                break;
        }
        return __uint_as_float(m);
    }
    float srt = warp_sort_asc(mn);
    return __shfl_sync(kFull, srt, K - 1);
}

// Rank-select: the buffer holds c (<= kCandCap) keys; write the cap
// smallest in order into the list at lo.  Returns the count kept.  Each lane
// ranks its own one or two keys against all c, reading the buffer two keys
// (16 bytes, a broadcast) at a time.
__device__ __forceinline__ int buffer_to_list(KnnWarpScratch &sc, int c, int cap, int lo)
{
    const int lane = lane_id();
    if ((c & 1) && lane == 0)
        sc.ck[c] = ~0ull;  // pad to a pair: ranks below no key
    __syncwarp();
    const unsigned long long k0 = lane < c ? sc.ck[lane] : ~0ull;
    const unsigned long long k1 = lane + 32 < c ? sc.ck[lane + 32] : ~0ull;
    const ulonglong2 *kp = reinterpret_cast<const ulonglong2 *>(sc.ck);
    int r0 = 0, r1 = 0;
    if (c <= 32) {
        for (int f = 0; f < c; f += 2) {
            const ulonglong2 kk = kp[f >> 1];
            r0 += (int)(kk.x < k0) + (int)(kk.y < k0);
        }
    } else {
        for (int f = 0; f < c; f += 2) {
            const ulonglong2 kk = kp[f >> 1];
            r0 += (int)(kk.x < k0) + (int)(kk.y < k0);
            r1 += (int)(kk.x < k1) + (int)(kk.y < k1);
        }
    }
    __syncwarp();
    if (lane < c && r0 < cap) {
        sc.ld[lo + r0] = __uint_as_float((unsigned)(k0 >> 32));
        sc.ls[lo + r0] = (int)(unsigned)k0;
    }
    if (lane + 32 < c && r1 < cap) {
        sc.ld[lo + r1] = __uint_as_float((unsigned)(k1 >> 32));
        sc.ls[lo + r1] = (int)(unsigned)k1;
    }
    __syncwarp();
    return c < cap ? c : cap;
}

// K-th smallest key among the first c buffered entries (c > K).
__device__ __forceinline__ unsigned long long buffer_kth_key(KnnWarpScratch &sc, int c, int K)
{
    const int lane = lane_id();
    unsigned long long k0 = lane < c ? sc.ck[lane] : ~0ull;
    unsigned long long k1 = lane + 32 < c ? sc.ck[lane + 32] : ~0ull;
    int r0 = 0, r1 = 0;
    for (int f = 0; f < c; ++f) {
        unsigned long long kf = sc.ck[f];
        r0 += kf < k0;
        r1 += kf < k1;
    }
    unsigned long long mine = ~0ull;
    if (lane < c && r0 == K - 1)
        mine = k0;
    if (lane + 32 < c && r1 == K - 1)
        mine = k1;
    // exactly one lane holds it (keys are distinct); min-reduce
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long other = __shfl_xor_sync(kFull, mine, o);
        mine = other < mine ? other : mine;
    }
    return mine;
}

// Threshold bound for the K-th smallest distance at E from the previous
// selected E's list (its entries grown to dimension E), or +inf.
__device__ __forceinline__ float seed_threshold(const KnnQuery &q, KnnWarpScratch &sc, int E, int prevE)
{
    const int lane = lane_id();
    const int K = E + 1 + kGuard;
    float th = CUDART_INF_F;
    const int have = sc.lcount[E];
    if (have >= K)
        th = sc.ld[list_off(E) + K - 1];
    if (prevE > 0 && sc.lcount[prevE] >= K) {
        const int plo = list_off(prevE);
        float dv = 0.f;
        if (lane < K) {
            dv = sc.ld[plo + lane];
            const int sv = sc.ls[plo + lane];
            if (sv < (E - 1) * q.tau) {
                dv = CUDART_INF_F;  // not embeddable at E: not a candidate
            } else {
                for (int m = prevE; m < E; ++m) {
                    float diff = q.xq[q.t - m * q.tau] - q.xc[sv - m * q.tau];
                    dv = fmaf(diff, diff, dv);
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            dv = fmaxf(dv, __shfl_xor_sync(kFull, dv, o));
        th = fminf(th, dv);
    }
    return th;
}

// Exclusive warp prefix sum of v; `total` receives the warp sum.
__device__ __forceinline__ int warp_excl_scan(int v, int &total)
{
    const int lane = lane_id();
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(kFull, incl, o);
        if (lane >= o)
            incl += u;
    }
    total = __shfl_sync(kFull, incl, 31);
    return incl - v;
}

// Next marked slot of a lane (bit j of m0/m1 = slot j), clearing it.
__device__ __forceinline__ int pop_slot(unsigned &m0, unsigned &m1)
{
    if (m0) {
        const int j = __ffs(m0) - 1;
        m0 &= m0 - 1;
        return j;
    }
    const int j = 32 + __ffs(m1) - 1;
    m1 &= m1 - 1;
    return j;
}

// Distance of slot j of this lane as stored in the warp scratch (the
// register value of the current E).
__device__ __forceinline__ float stored_d2(const KnnQuery &q, int j)
{
    return q.d2s[(j >> 2) * 128 + lane_id() * 4 + (j & 3)];
}

// Write the marked candidates of this lane with key <= kth into the buffer
// from position pos on (positions >= kCandCap are dropped).  Two slots per
// round, so their scratch loads are in flight together.
__device__ __forceinline__ void store_marked(const KnnQuery &q, KnnWarpScratch &sc, unsigned m0, unsigned m1, int c0,
                                             int pos, unsigned long long kth)
{
    const int lane = lane_id();
    const int s_lane = q.s_first + c0 + lane;
    while (m0 | m1) {
        const int ja = pop_slot(m0, m1);
        const bool two = (m0 | m1) != 0u;
        const int jb = two ? pop_slot(m0, m1) : ja;
        const unsigned long long ka = dkey(stored_d2(q, ja), s_lane + 32 * ja);
        const unsigned long long kb = dkey(stored_d2(q, jb), s_lane + 32 * jb);
        if (ka <= kth) {
            if (pos < kCandCap)
                sc.ck[pos] = ka;
            ++pos;
        }
        if (two && kb <= kth) {
            if (pos < kCandCap)
                sc.ck[pos] = kb;
            ++pos;
        }
    }
}

// Marked candidates of this lane with key <= kth.
__device__ __forceinline__ int count_marked(const KnnQuery &q, unsigned m0, unsigned m1, int c0,
                                            unsigned long long kth)
{
    const int lane = lane_id();
    int n = 0;
    while (m0 | m1) {
        const int j = pop_slot(m0, m1);
        n += dkey(stored_d2(q, j), q.s_first + c0 + lane + 32 * j) <= kth;
    }
    return n;
}

// Rare path: the list plus the marked candidates exceed the buffer.  The
// K-th smallest key of a buffered subset bounds the true K-th smallest
// (the subset holds at least K real candidates), so keeping only keys at or
// below it loses nothing; repeat until the survivors fit.
__device__ __noinline__ int select_overflow(const KnnQuery q, KnnWarpScratch &sc, unsigned m0, unsigned m1, int c0,
                                            int E, int have)
{
    const int lane = lane_id();
    const int K = E + 1 + kGuard;
    const int lo = list_off(E);
    unsigned long long kth = ~0ull;
    int c = kCandCap + 1;
    for (int tries = 0; tries < 6 && c > kCandCap; ++tries) {
        // buffer := (list U marked) with key <= kth, truncated to kCandCap
        const bool keep_l = lane < have && dkey(sc.ld[lo + lane], sc.ls[lo + lane]) <= kth;
        int total;
        const int mine = count_marked(q, m0, m1, c0, kth);
        const int off = warp_excl_scan(mine, total);
        const unsigned bl = __ballot_sync(kFull, keep_l);
        const int nl = __popc(bl);
        const float dl = keep_l ? sc.ld[lo + lane] : 0.f;
        const int sl = keep_l ? sc.ls[lo + lane] : 0;
        __syncwarp();
        if (keep_l)
            sc.ck[__popc(bl & ((1u << lane) - 1u))] = dkey(dl, sl);
        store_marked(q, sc, m0, m1, c0, nl + off, kth);
        __syncwarp();
        c = nl + total;
        if (c > kCandCap) {
            kth = buffer_kth_key(sc, kCandCap, K);
            __syncwarp();
        }
    }
    if (c > kCandCap) {
        if (lane == 0)
            sc.ovf[E] = 1;
        c = kCandCap;
    }
    return c;
}

// Exhaustive FP64 selection of the k nearest (rare fallback).
__device__ __noinline__ void exhaustive64(const KnnQuery q, KnnWarpScratch &sc, int E, int k)
{
    const int lane = lane_id();
    double last_d = -1.0;
    int last_s = -1;
    for (int n = 0; n < k; ++n) {
        double bd = CUDART_INF;
        int bs = 0x7fffffff;
        for (int s = q.s_first + lane; s <= q.s_last; s += 32) {
            if (!cand_ok(q, s, E))
                continue;
            double d = dist64(q.xq, q.t, q.xc, s, E, q.tau);
            bool after = (d > last_d) || (d == last_d && s > last_s);
            bool better = (d < bd) || (d == bd && s < bs);
            if (after && better) {
                bd = d;
                bs = s;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double od = __shfl_xor_sync(kFull, bd, o);
            int os = __shfl_xor_sync(kFull, bs, o);
            if (od < bd || (od == bd && os < bs)) {
                bd = od;
                bs = os;
            }
        }
        if (lane == 0) {
            sc.l64[n] = bd;
            sc.ls64[n] = bs;
        }
        last_d = bd;
        last_s = bs;
    }
    __syncwarp();
}

// Rare path of the finalisation: FP64 re-rank of the kept entries (and an
// exhaustive FP64 scan when even the guard entries cannot separate the k-th
// place from the entries left out), FP64 weights.  Lanes n < k receive
// (s_n, w_n).
__device__ __noinline__ void finalize64(const KnnQuery q, KnnWarpScratch &sc, int E, bool full, int &s_out,
                                        float &w_out)
{
    const int lane = lane_id();
    const int k = E + 1;
    const int lo = list_off(E);
    const int K = E + 1 + kGuard;
    const int have = min(sc.lcount[E], K);
    if (!full) {
        double d64 = CUDART_INF;
        int s_me = 0;
        if (lane < have) {
            s_me = sc.ls[lo + lane];
            d64 = dist64(q.xq, q.t, q.xc, s_me, E, q.tau);
        }
        int r = 0;
        for (int f = 0; f < have; ++f) {
            double df = __shfl_sync(kFull, d64, f);
            int sf = __shfl_sync(kFull, s_me, f);
            r += (df < d64) || (df == d64 && sf < s_me);
        }
        if (lane < have) {
            sc.l64[r] = d64;
            sc.ls64[r] = s_me;
        }
        __syncwarp();
        // entries left out have FP32 distance >= the last kept one
        if (have >= K) {
            float Dlast = sc.ld[lo + have - 1];
            full = !(sc.l64[k - 1] < (double)(Dlast - d2_err(Dlast, E)));
        }
    }
    if (full)
        exhaustive64(q, sc, E, k);
    if (lane == 0)
        atomicAdd(&g_knn_counts[full ? 1 : 0], 1ull);
    double dd = lane < k ? sqrt(sc.l64[lane]) : 0.0;
    // (an exhaustive scan over non-finite distances finds no candidate and
    // leaves a sentinel; keep every emitted index inside the series)
    s_out = lane < k ? min(max(sc.ls64[lane], q.s_first), q.s_last) : 0;
    double d1 = __shfl_sync(kFull, dd, 0);
    double u = 0.0;
    if (lane < k)
        u = d1 > 0.0 ? exp(-dd / d1) : (dd == 0.0 ? 1.0 : 0.0);
    double sum = warp_sum_d(u);
    w_out = (float)(u / sum);
}

// Final neighbours of (query, E) with exact order; lanes n < k receive
// (s_n, w_n) and call emit(E, k, s_n, w_n, lane < k).  Common path inline:
// the FP32 order is certified (every gap among the first E+2 entries
// exceeds the summed error bounds, no near duplicate) and the weights are
// FP32; everything else goes to finalize64.
template <class Emit>
__device__ __forceinline__ void finalize_E(const KnnQuery &q, KnnWarpScratch &sc, int E, Emit &emit)
{
    const int lane = lane_id();
    const int k = E + 1;
    const int lo = list_off(E);
    const int K = E + 1 + kGuard;
    const int have = min(sc.lcount[E], K);
    const bool full = sc.ovf[E] != 0 || have < k;
    bool all_ok = false;
    float Dn = 0.f, D0 = 0.f;
    if (!full) {
        Dn = lane < have ? sc.ld[lo + lane] : CUDART_INF_F;
        const float Dn1 = lane + 1 < have ? sc.ld[lo + lane + 1] : CUDART_INF_F;
        D0 = sc.ld[lo];
        bool ok = true;
        if (lane < k) {
            if (lane + 1 < have)
                ok = (Dn1 - Dn) > d2_err(Dn, E) + d2_err(Dn1, E);
            else
                ok = have < K;  // nothing was left out beyond the list
        }
        all_ok = __all_sync(kFull, ok) && D0 >= kNearDup;
    }
    int s_n = 0;
    float w = 0.f;
    if (all_ok) {
        const float dd = lane < k ? sqrtf(Dn) : 0.f;
        s_n = lane < k ? sc.ls[lo + lane] : 0;
        const float inv_d1 = __frcp_rn(sqrtf(D0));
        const float u = lane < k ? expf(-dd * inv_d1) : 0.f;
        w = u * __frcp_rn(warp_sum(u));
    } else {
        finalize64(q, sc, E, full, s_n, w);
    }
    emit(E, k, s_n, w, lane < k);
}

// Minimum of a lane's slots as a balanced tree (no serial dependency chain).
template <int J>
__device__ __forceinline__ float lane_min_tree(const float (&d2)[J])
{
    float m[J / 2];
#pragma unroll
    for (int j = 0; j < J / 2; ++j)
        m[j] = fminf(d2[2 * j], d2[2 * j + 1]);
#pragma unroll
    for (int w = J / 2; w > 1; w = (w + 1) / 2) {
#pragma unroll
        for (int j = 0; j < w / 2; ++j)
            m[j] = fminf(m[2 * j], m[2 * j + 1]);
        if (w & 1)
            m[w / 2] = m[w - 1];
    }
    return m[0];
}

// Bit j of (m0, m1) = slot j has d2 <= th; the bits of each 8-slot group are
// formed independently and then merged (short dependency chains).
template <int J>
__device__ __forceinline__ void mark_le(const float (&d2)[J], float th, unsigned &m0, unsigned &m1)
{
    unsigned g[(J + 7) / 8];
#pragma unroll
    for (int b = 0; b < (J + 7) / 8; ++b) {
        unsigned v = 0u;
#pragma unroll
        for (int u = 0; u < 8 && 8 * b + u < J; ++u)
            v |= (d2[8 * b + u] <= th ? 1u : 0u) << u;
        g[b] = v;
    }
    m0 = 0u;
    m1 = 0u;
#pragma unroll
    for (int b = 0; b < (J + 7) / 8; ++b) {
        if (b < 4)
            m0 |= g[b] << (8 * b);
        else
            m1 |= g[b] << (8 * (b - 4));
    }
}

// Candidates of the warp with d2 <= th (registers only).
template <int J>
__device__ __forceinline__ int count_le(const float (&d2)[J], float th)
{
    unsigned m0, m1;
    mark_le(d2, th, m0, m1);
    return (int)__reduce_add_sync(kFull, (unsigned)(__popc(m0) + __popc(m1)));
}

// Selection of one chunk for E (inline: the distance registers stay live
// across it).  1) A threshold that at least K = E+3 real candidates meet:
// the grown previous list (or this E's list of earlier chunks) when that
// alone marks at most a buffer's worth, else its minimum with the K-th
// smallest lane minimum.  For K <= kLaneMinK (and no list of earlier chunks)
// the lane-minimum bound is taken at once: there the grown list marks too
// many candidates in most selections.  2) If more than the buffer holds are at or below it, tighten it
// by counting rounds on the registers (the count of points within squared
// radius th grows about linearly for points near a low-dimensional
// attractor), keeping the count >= K.  3) Store
// the distances to the warp scratch, compact the marked candidates behind
// the list kept from earlier chunks (exclusive warp scan of per-lane
// counts), and rank them into the list.
template <int J, int kLaneMinK>
__device__ __forceinline__ void select_E(const KnnQuery &q, KnnWarpScratch &sc, const float (&d2)[J], int c0, int E,
                                         int prevE)
{
    const int lane = lane_id();
    const int K = E + 1 + kGuard;
    const int lo_l = list_off(E);
    const int have = sc.lcount[E];
    // never mark a +inf slot (not a candidate): thresholds are clamped
    float th = fminf(seed_threshold(q, sc, E, prevE), 3.40282347e38f);
    if (K <= kLaneMinK && have < K)
        th = fminf(th, fminf(kth_lane_min(lane_min_tree(d2), K), 3.40282347e38f));
    unsigned m0 = 0u, m1 = 0u;
    int c = kCandCap + 1;
    if (th < 3.40282347e38f) {  // a seed exists: often tight enough alone
        mark_le(d2, th, m0, m1);
        const int marked = (int)__reduce_add_sync(kFull, (unsigned)(__popc(m0) + __popc(m1)));
        // later chunks of a long series: when no slot of this chunk is at or
        // below the K-th entry kept from earlier chunks, the list is final
        // for this chunk as it stands
        if (marked == 0 && have >= K)
            return;
        c = have + marked;
    }
    if (c > kCandCap) {
        th = fminf(th, fminf(kth_lane_min(lane_min_tree(d2), K), 3.40282347e38f));
        mark_le(d2, th, m0, m1);
        c = have + (int)__reduce_add_sync(kFull, (unsigned)(__popc(m0) + __popc(m1)));
    }
    if (c > kCandCap) {
        // counting rounds; invariant: at least K real candidates (list
        // entries of earlier chunks or this chunk's slots) are <= hi
        float hi = th, lo = 0.f;
        int c_hi = c - have;
        const float want = (float)(K + 8);
        for (int r = 0; r < 8 && have + c_hi > kCandCap; ++r) {
            // the embedded points lie near a low-dimensional attractor, so
            // the count grows about linearly in th (not like th^(E/2))
            float g = lo > 0.f ? sqrtf(lo * hi) : hi * (want / (float)c_hi);
            if (!(g < hi) || !(g > lo))
                g = 0.5f * (lo + hi);
            const int cg = count_le(d2, g);
            const int lg = __popc(__ballot_sync(kFull, lane < have && sc.ld[lo_l + lane] <= g));
            if (lg + cg >= K) {
                hi = g;
                c_hi = cg;
            } else {
                lo = g;
            }
        }
        th = hi;
        c = have + c_hi;
        mark_le(d2, th, m0, m1);
    }
    // distances of this E to the scratch (16-byte stores, conflict-free)
#pragma unroll
    for (int j4 = 0; j4 < J / 4; ++j4)
        reinterpret_cast<float4 *>(q.d2s)[j4 * 32 + lane] =
            make_float4(d2[4 * j4], d2[4 * j4 + 1], d2[4 * j4 + 2], d2[4 * j4 + 3]);
    __syncwarp();
    if (c <= kCandCap) {
        int total;
        const int off = warp_excl_scan(__popc(m0) + __popc(m1), total);
        if (lane < have)
            sc.ck[lane] = dkey(sc.ld[lo_l + lane], sc.ls[lo_l + lane]);
        store_marked(q, sc, m0, m1, c0, have + off, ~0ull);
        __syncwarp();
    } else {
        c = select_overflow(q, sc, m0, m1, c0, E, have);
    }
    const int kept = buffer_to_list(sc, c, K + 1, lo_l);
    if (lane == 0)
        sc.lcount[E] = kept;
    __syncwarp();
}

// Two slots of one lag: d += (xq - v)^2 per slot with packed FP32 pairs;
// (xq - v) is formed as fma(v, -1, xq) (one rounding, as the plain
// subtraction), so the sums are bitwise those of the scalar form.
__device__ __forceinline__ void dist_step2(float &d0, float &d1, float xq, float v0, float v1)
{
    asm("{\n\t.reg .b64 D, V, Q, M;\n\t"
        "mov.b64 D, {%0, %1};\n\tmov.b64 V, {%2, %3};\n\t"
        "mov.b64 Q, {%4, %4};\n\tmov.b64 M, {%5, %5};\n\t"
        "fma.rn.f32x2 Q, V, M, Q;\n\tfma.rn.f32x2 D, Q, Q, D;\n\t"
        "mov.b64 {%0, %1}, D;\n\t}"
        : "+f"(d0), "+f"(d1)
        : "f"(v0), "f"(v1), "f"(xq), "f"(-1.0f));
}

// Full query: sweep all candidate chunks, then emit every selected E.
template <int J, class Emit>
__device__ void knn_query(const KnnQuery &q, KnnWarpScratch &sc, Emit &emit)
{
    const int lane = lane_id();
    for (int E = lane + 1; E <= q.E_lim; E += 32) {
        sc.lcount[E] = 0;
        sc.ovf[E] = 0;
    }
    __syncwarp();
    const int n_slots = q.s_last - q.s_first + 1;
    for (int c0 = 0; c0 < n_slots; c0 += 32 * J) {
        float d2[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
            int s = q.s_first + c0 + lane + 32 * j;
            d2[j] = cand_ok(q, s, 1) ? 0.f : CUDART_INF_F;
        }
        int prevE = 0;
        for (int E = 1; E <= q.E_lim; ++E) {
            const int off = (E - 1) * q.tau;
            const float xqv = q.xq[q.t - off];
            // lags before the series start read the +inf padding
            const float *xcj = q.xc + (q.s_first + c0 + lane - off);
#pragma unroll
            for (int j = 0; j < J; j += 2)
                dist_step2(d2[j], d2[j + 1], xqv, xcj[32 * j], xcj[32 * j + 32]);
            if ((q.sel >> (E - 1)) & 1u) {
                select_E<J, Emit::kLaneMinK>(q, sc, d2, c0, E, prevE);
                prevE = E;
            }
        }
    }
    for (int E = 1; E <= q.E_lim; ++E)
        if ((q.sel >> (E - 1)) & 1u)
            finalize_E(q, sc, E, emit);
}

}  // namespace edm
