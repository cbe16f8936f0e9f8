// ccm_noalloc.cu -- edm_ccm_rho_noalloc: the cross-map phase with all its
// scratch in one statically allocated device array, for callers that cannot
// allocate device memory themselves (no cudaMalloc/cudaFree, no allocating
// library routine, no host heap either).
//
// The scratch array below is a file-scope __device__ object: every GPU that
// loads this library holds it until the process exits.  Host code never
// uses its name as an address; the first call on each device resolves the
// device address with cudaGetSymbolAddress (that device current, under a
// lock) and keeps it for later calls, so a device reset after that first
// call is not supported.  All calls share the array and see the previous
// call's contents; the kernels write everything they read except the E
// counters of the plan, which the plan kernel clears itself.  Calls whose
// GPU work overlaps (different streams, or host threads) race on the array.
#include <cstdio>
#include <mutex>

#include "launchers.h"

namespace edm {

// 64 MiB: target tiles + plan + kNN tables of one library block.
constexpr size_t kStaticScratchBytes = 64ull << 20;
static __device__ __align__(256) unsigned char g_ccm_scratch[kStaticScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
void *g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

// Layout of the plan and tiles inside the static array.
struct NaLayout {
    size_t counts, pi, omom, meta, tiles, tables, table_bytes;
    int64_t n_tiles_max;
};

NaLayout na_layout(int64_t N, int64_t T, int RB)
{
    NaLayout w;
    w.n_tiles_max = (N + RB / 4 - 1) / (RB / 4) + EDM_MAX_E;
    size_t off = 0;
    w.counts = off;
    off += 256;
    w.pi = off;
    off += al256((size_t)N * sizeof(int32_t));
    w.omom = off;
    off += al256((size_t)w.n_tiles_max * 32 * sizeof(float2));
    w.meta = off;
    off += al256((size_t)w.n_tiles_max * sizeof(TileMeta));
    w.tiles = off;
    off += al256((size_t)w.n_tiles_max * (size_t)T * RB);
    w.tables = off;
    w.table_bytes = off < kStaticScratchBytes ? kStaticScratchBytes - off : 0;
    return w;
}

TableLayout na_table_layout(uint32_t sel, int64_t T, const edm_params *p)
{
    TableLayout lay;
    lay.Tq_pad = (int)(((T - p->Tp) + 31) / 32 * 32);
    int64_t off = 0;
    for (int E = 0; E <= EDM_MAX_E; ++E) {
        lay.off_w[E] = -1;
        lay.off_i[E] = -1;
    }
    for (int E = 1; E <= EDM_MAX_E; ++E) {
        if (!((sel >> (E - 1)) & 1u))
            continue;
        lay.off_w[E] = off;
        off += (int64_t)al256((size_t)(E + 1) * lay.Tq_pad * sizeof(float));
        lay.off_i[E] = off;
        off += (int64_t)al256((size_t)(E + 1) * lay.Tq_pad * sizeof(uint16_t));
    }
    lay.lib_stride = off;
    return lay;
}

int tile_width(int E, bool f16, int RB) { return (f16 && E + 1 <= kF16MaxK) ? RB / 2 : RB / 4; }

}  // namespace

// One CTA: count targets per E (counters cleared here), stable counting
// sort of target indices by E into pi, and the tile list.  counts[0] flags
// an optE value outside 1..EDM_MAX_E.
__global__ void __launch_bounds__(1024) na_plan_kernel(const int32_t *__restrict__ optE, int N, int f16, int RB,
                                                       int32_t *__restrict__ counts, int32_t *__restrict__ pi,
                                                       TileMeta *__restrict__ meta)
{
    __shared__ int cnt[EDM_MAX_E + 2];
    __shared__ int start[EDM_MAX_E + 2];
    __shared__ int tstart[EDM_MAX_E + 2];
    if (threadIdx.x < EDM_MAX_E + 2)
        cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        int E = optE[j];
        atomicAdd(&cnt[(E >= 1 && E <= EDM_MAX_E) ? E : 0], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0, ts = 0;
        for (int E = 1; E <= EDM_MAX_E; ++E) {
            start[E] = s;
            tstart[E] = ts;
            s += cnt[E];
            const int w = (f16 && E + 1 <= kF16MaxK) ? RB / 2 : RB / 4;
            ts += (cnt[E] + w - 1) / w;
        }
        for (int E = 0; E <= EDM_MAX_E; ++E)
            counts[E] = cnt[E];
    }
    __syncthreads();
    // warp e-1 places the targets of E = e in index order (stable)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int E = warp + 1; E <= EDM_MAX_E; E += blockDim.x / 32) {
        int pos = start[E];
        for (int j0 = 0; j0 < N; j0 += 32) {
            const int j = j0 + lane;
            const bool hit = j < N && optE[j] == E;
            const unsigned b = __ballot_sync(0xffffffffu, hit);
            if (hit)
                pi[pos + __popc(b & ((1u << lane) - 1u))] = j;
            pos += __popc(b);
        }
        if (lane == 0) {
            const bool wf16 = f16 && E + 1 <= kF16MaxK;
            const int w = wf16 ? RB / 2 : RB / 4;
            int t = tstart[E];
            for (int c = 0; c < cnt[E]; c += w, ++t)
                meta[t] = TileMeta{E, start[E] + c, min(w, cnt[E] - c), wf16 ? kTileF16 : 0};
        }
    }
}

}  // namespace edm

extern "C" int edm_ccm_rho_noalloc(const float *Y, int64_t N, int64_t T, int64_t ldY, const int32_t *optE,
                                   int64_t lib_begin, int64_t lib_count, const edm_params *params, float *rho,
                                   int64_t ld_rho, void *stream)
{
    using namespace edm;
    if (!params || !Y || !optE || !rho || N < 1 || T < 2 || ldY < T)
        return EDM_ERR_INVALID;
    if (params->tau < 1 || params->Tp < 0 || params->exclusion_radius < -1)
        return EDM_ERR_INVALID;
    if (params->precision != EDM_PRECISION_FP32 && params->precision != EDM_PRECISION_FP16_TARGETS)
        return EDM_ERR_INVALID;
    if (lib_begin < 0 || lib_count < 0 || lib_begin + lib_count > N || ld_rho < lib_count)
        return EDM_ERR_INVALID;
    // this call always builds tables with the warp kernel (EDM_FLAG_KNN_WARP
    // changes nothing); the non-finite scan and the scalar-gather lookup are
    // not offered here
    if (params->flags & ~EDM_FLAG_KNN_WARP)
        return EDM_ERR_UNSUPPORTED;
    if (T > EDM_MAX_T || N > 0x7fffffffLL || T > knn_max_T() || chunked_row_bytes((int)T) == 0)
        return EDM_ERR_UNSUPPORTED;
    const bool f16 = params->precision == EDM_PRECISION_FP16_TARGETS;
    const int RB = chunked_row_bytes((int)T);
    const NaLayout L = na_layout(N, T, RB);
    const TableLayout all = na_table_layout((1u << EDM_MAX_E) - 1u, T, params);
    // beyond the static array: reject before touching the device
    if (L.tables >= kStaticScratchBytes || L.table_bytes < (size_t)all.lib_stride)
        return EDM_ERR_WORKSPACE;
    if (lib_count == 0)
        return EDM_OK;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return EDM_ERR_CUDA;
    void *ptr = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            e = cudaGetSymbolAddress(&g_scratch_ptr[dev], g_ccm_scratch);
            if (e != cudaSuccess || !g_scratch_ptr[dev]) {
                g_scratch_ptr[dev] = nullptr;
                return EDM_ERR_CUDA;
            }
        }
        ptr = g_scratch_ptr[dev];
    }
    unsigned char *ws = (unsigned char *)ptr;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *counts_d = (int32_t *)(ws + L.counts);
    int32_t *pi_d = (int32_t *)(ws + L.pi);
    float2 *omom_d = (float2 *)(ws + L.omom);
    TileMeta *meta_d = (TileMeta *)(ws + L.meta);
    unsigned char *tiles_d = ws + L.tiles;
    uint8_t *tables_d = ws + L.tables;

    na_plan_kernel<<<1, 1024, 0, st>>>(optE, (int)N, f16 ? 1 : 0, RB, counts_d, pi_d, meta_d);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return EDM_ERR_CUDA;
    int32_t counts[EDM_MAX_E + 1];
    if ((e = cudaMemcpyAsync(counts, counts_d, sizeof counts, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return EDM_ERR_CUDA;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
        return EDM_ERR_CUDA;
    if (counts[0] != 0)
        return EDM_ERR_INVALID;
    int n_tiles = 0;
    for (int E = 1; E <= EDM_MAX_E; ++E) {
        if (counts[E] > 0 && (T - params->Tp - (int64_t)(E - 1) * params->tau -
                              (params->exclusion_radius >= 0 ? 2 * (int64_t)params->exclusion_radius + 1 : 0)) < E + 1)
            return EDM_ERR_INVALID;
        n_tiles += (counts[E] + tile_width(E, f16, RB) - 1) / tile_width(E, f16, RB);
    }
    if ((e = launch_prep_targets(Y, ldY, (int)T, params->tau, params->Tp, pi_d, meta_d, n_tiles, (float *)tiles_d,
                                 omom_d, st, RB)) != cudaSuccess)
        return EDM_ERR_CUDA;
    if (f16 && (e = launch_prep_targets_f16(Y, ldY, (int)T, params->tau, params->Tp, pi_d, meta_d, n_tiles, tiles_d,
                                            omom_d, st, RB)) != cudaSuccess)
        return EDM_ERR_CUDA;

    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // one E group at a time (all its tiles), libraries in blocks that fit
    // the table area of the static array
    int tile0 = 0;
    for (int E = 1; E <= EDM_MAX_E; ++E) {
        const int ntE = (counts[E] + tile_width(E, f16, RB) - 1) / tile_width(E, f16, RB);
        if (ntE == 0)
            continue;
        const uint32_t sel = 1u << (E - 1);
        const TableLayout lay = na_table_layout(sel, T, params);
        int64_t per_block = (int64_t)(L.table_bytes / (size_t)lay.lib_stride);
        per_block = per_block < 1 ? 1 : (per_block > 65535 ? 65535 : per_block);
        for (int64_t lb0 = 0; lb0 < lib_count; lb0 += per_block) {
            const int nlb = (int)((lib_count - lb0) < per_block ? (lib_count - lb0) : per_block);
            if ((e = launch_knn_tables(Y, ldY, lib_begin + lb0, nlb, (int)T, params->tau, params->Tp,
                                       params->exclusion_radius, sel, lay, tables_d, st)) != cudaSuccess)
                return EDM_ERR_CUDA;
            LookupArgs a;
            a.tiles = (const float *)tiles_d;
            a.meta = meta_d;
            a.pi = pi_d;
            a.omom = omom_d;
            a.tables = tables_d;
            a.lay = lay;
            a.T = (int)T;
            a.tau = params->tau;
            a.Tp = params->Tp;
            a.s_lo = 0;
            a.lag = params->Tp;
            a.tile_begin = tile0;
            a.n_tiles = ntE;
            a.n_lib = nlb;
            int parts = (4 * sms + ntE - 1) / ntE;
            const int maxp = (nlb + 7) / 8;
            a.lib_parts = parts < 1 ? 1 : (parts > maxp ? maxp : parts);
            a.rho_col0 = lb0;
            a.rho = rho;
            a.ld_rho = ld_rho;
            if ((e = launch_lookup_multi(a, RB, st)) != cudaSuccess)
                return EDM_ERR_CUDA;
        }
        tile0 += ntE;
    }
    return EDM_OK;
}
