// ccm_plan.cu -- the E grouping of the cross-map phase planned on the device
// (Algorithm 2 runs every target with its own E = optE[j]; Sec. III-B:
// tables are built once per library and E and reused for every target of
// that E), so the cross-map entry points never read optE back to the host.
//
// One CTA: count the targets of each E, sort the target indices by E
// (stable), cut each E's targets into tiles (E-sorted), zero the unused tile
// slots, and describe every launch slot of the host's fixed group structure
// -- its tile range and the bit mask of the E it contains -- so that launches
// with upper-bound grids find their work on the device.  Targets whose E is
// outside 1..EDM_MAX_E or leaves too few candidates get NaN rows in rho.
#include "edm_internal.cuh"
#include "launchers.h"

namespace edm {

__global__ void __launch_bounds__(1024) ccm_plan_kernel(const int32_t *__restrict__ optE, CcmPlanSpec sp,
                                                        int32_t *__restrict__ counts, int32_t *__restrict__ pi,
                                                        TileMeta *__restrict__ meta, SlotDesc *__restrict__ slots)
{
    __shared__ int cnt[EDM_MAX_E + 2];
    __shared__ int start[EDM_MAX_E + 2];
    __shared__ int tstart[EDM_MAX_E + 2];
    __shared__ int ok_E[EDM_MAX_E + 2];
    const int N = sp.N;
    if (threadIdx.x < EDM_MAX_E + 2) {
        cnt[threadIdx.x] = 0;
        const int E = threadIdx.x;
        int ok = 0;
        if (E >= 1 && E <= EDM_MAX_E) {
            const int A = max((E - 1) * sp.tau, sp.s_lo);
            const int cand = sp.T - sp.Tp - A - (sp.excl >= 0 ? 2 * sp.excl + 1 : 0);
            ok = cand >= E + 1;
        }
        ok_E[E] = ok;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const int E = optE[j];
        const bool valid = E >= 1 && E <= EDM_MAX_E && ok_E[E];
        atomicAdd(&cnt[valid ? E : 0], 1);
        if (!valid && sp.rho) {
            for (int u = 0; u < sp.planes; ++u) {
                float *row = sp.rho + (size_t)u * sp.plane_stride + (size_t)j * sp.ld_rho;
                for (int64_t c = 0; c < sp.row_len; ++c)
                    row[c] = CUDART_NAN_F;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0, ts = 0;
        for (int E = 1; E <= EDM_MAX_E; ++E) {
            start[E] = s;
            tstart[E] = ts;
            s += cnt[E];
            ts += (cnt[E] + plan_tile_width(E, sp.f16, sp.RB) - 1) / plan_tile_width(E, sp.f16, sp.RB);
        }
        start[EDM_MAX_E + 1] = s;
        tstart[EDM_MAX_E + 1] = ts;
        for (int E = 0; E <= EDM_MAX_E; ++E)
            counts[E] = cnt[E];
        counts[EDM_MAX_E + 1] = ts;  // tiles in use
        if (sp.starts)
            for (int E = 0; E <= EDM_MAX_E + 1; ++E)
                sp.starts[E] = E == 0 ? 0 : start[E];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    // warp E-1 places the targets of E in index order (stable) and writes
    // that E's tiles
    for (int E = warp + 1; E <= EDM_MAX_E; E += nwarps) {
        if (cnt[E] == 0)
            continue;
        int pos = start[E];
        for (int j0 = 0; j0 < N; j0 += 32) {
            const int j = j0 + lane;
            const bool hit = j < N && optE[j] == E;
            const unsigned b = __ballot_sync(0xffffffffu, hit);
            if (hit)
                pi[pos + __popc(b & ((1u << lane) - 1u))] = j;
            pos += __popc(b);
        }
        const int w = plan_tile_width(E, sp.f16, sp.RB);
        const int fl = (sp.f16 && E + 1 <= kF16MaxK) ? kTileF16 : 0;
        for (int c = lane * w, t = tstart[E] + lane; c < cnt[E]; c += 32 * w, t += 32)
            meta[t] = TileMeta{E, start[E] + c, min(w, cnt[E] - c), fl};
    }
    // unused tile slots carry E = 0 (their CTAs return at once)
    for (int t = tstart[EDM_MAX_E + 1] + threadIdx.x; t < sp.n_tiles_max; t += blockDim.x)
        meta[t] = TileMeta{0, 0, 0, 0};
    // launch slots: group g covers E in [g_lo[g], g_hi[g]], cut into target
    // blocks of tiles_per_block tiles (0: not cut)
    for (int g = warp; g < sp.n_groups; g += nwarps) {
        const int elo = sp.g_lo[g], ehi = sp.g_hi[g];
        const int gb = tstart[elo], ge = tstart[ehi + 1];
        const int tpb = sp.tiles_per_block > 0 ? sp.tiles_per_block : max(1, ge - gb);
        for (int tb = lane; tb < sp.tb_max[g]; tb += 32) {
            const int b0 = min(ge, gb + tb * tpb);
            const int b1 = min(ge, b0 + tpb);
            uint32_t sel = 0u;
            for (int E = elo; E <= ehi; ++E)  // E present among tiles [b0, b1)
                if (cnt[E] > 0 && tstart[E] < b1 && tstart[E + 1] > b0)
                    sel |= 1u << (E - 1);
            slots[sp.slot0[g] + tb] = SlotDesc{b0, b1 - b0, sel, 0};
        }
    }
}

// Convergence subsets: subset u (bit s of masks[u * words + s / 32] allows
// candidate s) must leave E+1 candidates, beyond the exclusion window, for
// the largest E in use; a subset that does not gets NaN for its whole rho
// plane (rho + u * plane_stride, N rows of N values).  One CTA per subset,
// launched after the subset's cross map.
__global__ void __launch_bounds__(256) subset_check_kernel(const uint32_t *__restrict__ masks, int64_t words,
                                                           const int32_t *__restrict__ counts, int N, int T, int tau,
                                                           int Tp, int excl, float *__restrict__ rho, int64_t ld_rho,
                                                           int64_t plane_stride)
{
    __shared__ int c_sh;
    int E_top = 0;
    for (int E = EDM_MAX_E; E >= 1 && E_top == 0; --E)
        if (counts[E] > 0)
            E_top = E;
    if (E_top == 0)
        return;
    const uint32_t *m = masks + (size_t)blockIdx.x * words;
    const int lo = (E_top - 1) * tau, hi = T - 1 - Tp;
    if (threadIdx.x == 0)
        c_sh = 0;
    __syncthreads();
    int c = 0;
    for (int s = lo + threadIdx.x; s <= hi; s += blockDim.x)
        c += (m[s >> 5] >> (s & 31)) & 1u;
    atomicAdd(&c_sh, c);
    __syncthreads();
    const int have = c_sh - (excl >= 0 ? 2 * excl + 1 : 0);
    if (have >= E_top + 1)
        return;
    float *plane = rho + (size_t)blockIdx.x * plane_stride;
    for (int64_t q = threadIdx.x; q < (int64_t)N * N; q += blockDim.x)
        plane[(q / N) * ld_rho + q % N] = CUDART_NAN_F;
}

cudaError_t launch_subset_check(const uint32_t *masks, int n_sub, int64_t words, const int32_t *counts, int N, int T,
                                int tau, int Tp, int excl, float *rho, int64_t ld_rho, int64_t plane_stride,
                                cudaStream_t st)
{
    subset_check_kernel<<<n_sub, 256, 0, st>>>(masks, words, counts, N, T, tau, Tp, excl, rho, ld_rho, plane_stride);
    return cudaGetLastError();
}

cudaError_t launch_ccm_plan(const int32_t *optE, const CcmPlanSpec &sp, int32_t *counts, int32_t *pi, TileMeta *meta,
                            SlotDesc *slots, cudaStream_t st)
{
    ccm_plan_kernel<<<1, 1024, 0, st>>>(optE, sp, counts, pi, meta, slots);
    return cudaGetLastError();
}

}  // namespace edm
