// edm_api.cu -- the C ABI (include/edm.h): argument checks, the host-side
// plan of the cross-map phase, and the kernel orchestration.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "launchers.h"

namespace {

thread_local int g_last_cuda = 0;
thread_local char g_msg[256];

int cuda_fail(cudaError_t e)
{
    g_last_cuda = (int)e;
    return EDM_ERR_CUDA;
}

#define EDM_CUDA(call)                                                                                                 \
    do {                                                                                                               \
        cudaError_t e_ = (call);                                                                                       \
        if (e_ != cudaSuccess)                                                                                         \
            return cuda_fail(e_);                                                                                      \
    } while (0)

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// --- launch accounting and optional per-launch event timing ----------------
struct ProfRec {
    cudaEvent_t a, b;
    int kernel;
    double units;
};
int64_t g_launches[EDM_KERNEL_COUNT] = {};
bool g_prof = false;
std::vector<ProfRec> g_recs;
double g_ms[EDM_KERNEL_COUNT], g_units[EDM_KERNEL_COUNT];
int64_t g_timed[EDM_KERNEL_COUNT];

struct LaunchScope {
    ProfRec rec{};
    bool on;
    cudaStream_t st;
    void add_launches(int kernel, int n) { g_launches[kernel] += n; }
    LaunchScope(int kernel, cudaStream_t s, double units, int launches = 1) : on(g_prof), st(s)
    {
        g_launches[kernel] += launches;
        if (on) {
            rec.kernel = kernel;
            rec.units = units;
            cudaEventCreate(&rec.a);
            cudaEventCreate(&rec.b);
            cudaEventRecord(rec.a, st);
        }
    }
    ~LaunchScope()
    {
        if (on) {
            cudaEventRecord(rec.b, st);
            g_recs.push_back(rec);
        }
    }
};

thread_local int64_t g_bad_series = -1;

// EDM_FLAG_VALIDATE: returns EDM_OK, or EDM_ERR_INVALID with the first bad
// series recorded, or EDM_ERR_CUDA.
int validate_series(const float *Y, int64_t N, int64_t T, int64_t ldY, const edm_params *p, cudaStream_t st)
{
    g_bad_series = -1;
    if (!(p->flags & EDM_FLAG_VALIDATE))
        return EDM_OK;
    int64_t bad = -1;
    cudaError_t e = edm::first_nonfinite_series(Y, N, T, ldY, st, &bad);
    if (e != cudaSuccess)
        return cuda_fail(e);
    if (bad >= 0) {
        g_bad_series = bad;
        return EDM_ERR_INVALID;
    }
    return EDM_OK;
}

int check_common(const edm_params *p)
{
    g_bad_series = -1;
    if (!p)
        return EDM_ERR_INVALID;
    if (p->tau < 1 || p->Tp < 0 || p->exclusion_radius < -1)
        return EDM_ERR_INVALID;
    if (p->precision != EDM_PRECISION_FP32 && p->precision != EDM_PRECISION_FP16_TARGETS)
        return EDM_ERR_INVALID;
    return EDM_OK;
}

// Candidates a phase-2 query is guaranteed to have at dimension E.
int64_t ccm_min_candidates(int64_t T, int E, const edm_params *p)
{
    int64_t n = T - p->Tp - (int64_t)(E - 1) * p->tau;
    if (p->exclusion_radius >= 0)
        n -= 2 * (int64_t)p->exclusion_radius + 1;
    return n;
}

int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 148;
    return n > 0 ? n : 148;
}

// Budgets for the L2-resident working set of the cross-map phase.
constexpr size_t kTileBlockBytes = 64ull << 20;  // target tiles per block
constexpr size_t kTableBytes = 48ull << 20;      // kNN tables per library block (L2 target)
constexpr int64_t kMinLibBlock = 1024;           // library block floor (series up to 4,096 steps)

// Library block floor for series of length T.  Up to 4,096 steps: 1,024
// libraries (every block re-streams all target tiles through shared
// memory, so larger blocks stream them fewer times; at N = 101,729 and
// T = 1,500 the step took 17.16 s against 17.31 s with 256-library blocks).
// Long series give every library thousands of kNN queries, so fewer
// libraries fill the GPU and the floor shrinks with T (keeping the table
// area near 1.4 GB at most).
int64_t min_lib_block(int64_t T) { return T <= 4096 ? kMinLibBlock : std::max<int64_t>(16, 256 * 4096 / T); }

int tq_pad(int64_t T, const edm_params *p) { return (int)(((T - p->Tp) + 31) / 32 * 32); }

edm::TableLayout make_layout(uint32_t sel, int64_t T, const edm_params *p)
{
    edm::TableLayout lay;
    lay.Tq_pad = tq_pad(T, p);
    int64_t off = 0;
    for (int E = 0; E <= EDM_MAX_E; ++E) {
        lay.off_w[E] = -1;
        lay.off_i[E] = -1;
    }
    for (int E = 1; E <= EDM_MAX_E; ++E) {
        if (!((sel >> (E - 1)) & 1u))
            continue;
        lay.off_w[E] = off;
        off += (int64_t)align256((size_t)(E + 1) * lay.Tq_pad * sizeof(float));
        lay.off_i[E] = off;
        off += (int64_t)align256((size_t)(E + 1) * lay.Tq_pad * sizeof(uint16_t));
    }
    lay.lib_stride = off;
    return lay;
}

struct CcmWs {
    size_t pi, omom, meta, tiles, tables, counts, slots, total;
    int64_t n_tiles_max;
    size_t table_bytes;  // L2-sized budget
    size_t table_cap;    // allocated table area
};

// Tile row bytes for a call: 128 (32 FP32 / 64 FP16 targets per row) when
// a tile of T rows fits shared memory, else 64; the scalar path uses 128.
int ccm_row_bytes(int64_t T, const edm_params *p)
{
    if (p->flags & EDM_FLAG_LOOKUP_SCALAR)
        return 128;
    int rb = edm::chunked_row_bytes((int)std::min<int64_t>(T, EDM_MAX_T));
    return rb ? rb : 128;
}

CcmWs ccm_ws_layout(int64_t N, int64_t T, const edm_params *p)
{
    CcmWs w;
    const int RB = ccm_row_bytes(T, p);
    w.n_tiles_max = (N + RB / 4 - 1) / (RB / 4) + EDM_MAX_E;
    size_t off = 0;
    w.pi = off;
    off += align256((size_t)N * sizeof(int32_t));
    w.omom = off;
    off += align256((size_t)N * sizeof(float2));
    w.meta = off;
    off += align256((size_t)w.n_tiles_max * sizeof(edm::TileMeta));
    // device-side plan: per-E counts and the launch slots (at most one per
    // group and target block)
    w.counts = off;
    off += 256;
    w.slots = off;
    off += align256((size_t)edm::kMaxPlanGroups * (size_t)(w.n_tiles_max + 1) * sizeof(edm::SlotDesc));
    w.tiles = off;
    off += align256((size_t)w.n_tiles_max * (size_t)T * RB);
    w.tables = off;
    edm::TableLayout all = make_layout((1u << EDM_MAX_E) - 1u, T, p);
    w.table_bytes = std::max(kTableBytes, (size_t)all.lib_stride);
    w.table_cap = std::max(w.table_bytes, (size_t)std::min<int64_t>(N, min_lib_block(T)) * (size_t)all.lib_stride);
    off += align256(w.table_cap);
    w.total = off;
    return w;
}

}  // namespace

namespace edm {

static __device__ unsigned long long g_first_bad;

__global__ void nonfinite_kernel(const float *__restrict__ Y, int64_t N, int64_t T, int64_t ldY)
{
    for (int64_t i = blockIdx.x; i < N; i += gridDim.x) {
        bool bad = false;
        for (int64_t t = threadIdx.x; t < T; t += blockDim.x)
            bad |= !isfinite(Y[i * ldY + t]);
        if (__syncthreads_or(bad) && threadIdx.x == 0)
            atomicMin(&g_first_bad, (unsigned long long)i);
    }
}

cudaError_t first_nonfinite_series(const float *Y, int64_t N, int64_t T, int64_t ldY, cudaStream_t st,
                                   int64_t *first_bad)
{
    static std::mutex mu;  // one scan at a time uses the device word
    std::lock_guard<std::mutex> lock(mu);
    const unsigned long long none = ~0ull;
    cudaError_t e = cudaMemcpyToSymbolAsync(g_first_bad, &none, sizeof none, 0, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess)
        return e;
    nonfinite_kernel<<<(unsigned)std::min<int64_t>(N, 4096), 256, 0, st>>>(Y, N, T, ldY);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    unsigned long long r = none;
    if ((e = cudaMemcpyFromSymbolAsync(&r, g_first_bad, sizeof r, 0, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
        return e;
    *first_bad = r == none ? -1 : (int64_t)r;
    return cudaSuccess;
}

void note_launches(int kernel, int64_t n) { g_launches[kernel] += n; }
bool profiling() { return g_prof; }
void prof_push(int kernel, cudaEvent_t a, cudaEvent_t b, double units)
{
    ProfRec r;
    r.a = a;
    r.b = b;
    r.kernel = kernel;
    r.units = units;
    g_recs.push_back(r);
}
}  // namespace edm

extern "C" {

int edm_version(void) { return 0x000100; }

int64_t edm_launch_count(int kernel)
{
    return (kernel >= 0 && kernel < EDM_KERNEL_COUNT) ? g_launches[kernel] : -1;
}

int edm_profile_enable(int on)
{
    g_prof = on != 0;
    return EDM_OK;
}

int edm_profile_read(int kernel, double *ms, int64_t *launches, double *units)
{
    if (kernel < 0 || kernel >= EDM_KERNEL_COUNT)
        return EDM_ERR_INVALID;
    for (ProfRec &r : g_recs) {
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess)
            return cuda_fail(e);
        float f = 0.f;
        cudaEventElapsedTime(&f, r.a, r.b);
        g_ms[r.kernel] += f;
        g_units[r.kernel] += r.units;
        g_timed[r.kernel]++;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_recs.clear();
    if (ms)
        *ms = g_ms[kernel];
    if (launches)
        *launches = g_timed[kernel];
    if (units)
        *units = g_units[kernel];
    g_ms[kernel] = 0.0;
    g_units[kernel] = 0.0;
    g_timed[kernel] = 0;
    return EDM_OK;
}

int edm_last_cuda_error(void) { return g_last_cuda; }

int64_t edm_last_bad_series(void) { return g_bad_series; }

int edm_knn_counters(int64_t *reranks, int64_t *exhaustive, int reset)
{
    unsigned long long c[2] = {0ull, 0ull};
    cudaError_t e = edm::knn_counters(c, reset != 0);
    if (e != cudaSuccess)
        return cuda_fail(e);
    if (reranks)
        *reranks = (int64_t)c[0];
    if (exhaustive)
        *exhaustive = (int64_t)c[1];
    return EDM_OK;
}

int edm_wait_timeouts(int64_t *count, int reset)
{
    cudaError_t (*readers[])(unsigned long long *, bool) = {
        edm::knn_wait_timeouts, edm::knn_thread_wait_timeouts, edm::lookup_multi128_wait_timeouts,
        edm::lookup_multi128_lag_wait_timeouts, edm::lookup_multi64_wait_timeouts,
        edm::lookup_multi64_lag_wait_timeouts, edm::backward_wait_timeouts};
    unsigned long long tot = 0ull;
    for (auto rd : readers) {
        unsigned long long c = 0ull;
        cudaError_t e = rd(&c, reset != 0);
        if (e != cudaSuccess)
            return cuda_fail(e);
        tot += c;
    }
    if (count)
        *count = (int64_t)tot;
    return EDM_OK;
}

const char *edm_status_string(int status)
{
    switch (status) {
    case EDM_OK: return "EDM_OK";
    case EDM_ERR_INVALID: return "EDM_ERR_INVALID: invalid argument";
    case EDM_ERR_WORKSPACE: return "EDM_ERR_WORKSPACE: workspace too small";
    case EDM_ERR_TIMEOUT: return "EDM_ERR_TIMEOUT: a bounded device wait gave up";
    case EDM_ERR_UNSUPPORTED: return "EDM_ERR_UNSUPPORTED: outside this library's limits";
    case EDM_ERR_CUDA:
        snprintf(g_msg, sizeof g_msg, "EDM_ERR_CUDA: %s", cudaGetErrorString((cudaError_t)g_last_cuda));
        return g_msg;
    default: return "unknown status";
    }
}

int edm_optimal_E(const float *Y, int64_t N, int64_t T, int64_t ldY, const edm_params *params, int32_t *optE,
                  float *rho_by_E, void *stream)
{
    int rc = check_common(params);
    if (rc)
        return rc;
    if (!Y || !optE || N < 1 || T < 4 || ldY < T || params->E_max < 1)
        return EDM_ERR_INVALID;
    if (params->E_max > EDM_MAX_E || T > EDM_MAX_T)
        return EDM_ERR_UNSUPPORTED;
    const int64_t h = T / 2;
    const int64_t span = (int64_t)(params->E_max - 1) * params->tau;
    if (h - params->Tp - span < params->E_max + 1 || (T - h) - params->Tp - span < 2)
        return EDM_ERR_INVALID;
    if (T > edm::knn_max_T())
        return EDM_ERR_UNSUPPORTED;
    if ((rc = validate_series(Y, N, T, ldY, params, (cudaStream_t)stream)) != EDM_OK)
        return rc;
    {
        LaunchScope ls(EDM_KERNEL_SIMPLEX, (cudaStream_t)stream, (double)N);
        EDM_CUDA(edm::launch_simplex(Y, N, (int)T, ldY, params->E_max, params->tau, params->Tp, optE, rho_by_E,
                                     (cudaStream_t)stream));
    }
    return EDM_OK;
}

int edm_knn_table(const float *Y, int64_t n_lib, int64_t T, int64_t ldY, int32_t E, const edm_params *params,
                  int32_t *idx, float *w, int64_t Tq, void *stream)
{
    int rc = check_common(params);
    if (rc)
        return rc;
    if (!Y || !idx || !w || n_lib < 1 || T < 2 || ldY < T || E < 1)
        return EDM_ERR_INVALID;
    if (E > EDM_MAX_E || T > EDM_MAX_T || n_lib > 65535)
        return EDM_ERR_UNSUPPORTED;
    if (Tq != T - params->Tp - (int64_t)(E - 1) * params->tau || Tq < 1)
        return EDM_ERR_INVALID;
    if (ccm_min_candidates(T, E, params) < E + 1)
        return EDM_ERR_INVALID;
    if (T > edm::knn_max_T())
        return EDM_ERR_UNSUPPORTED;
    {
        LaunchScope ls(EDM_KERNEL_KNN, (cudaStream_t)stream, (double)n_lib);
        EDM_CUDA(edm::launch_knn_public(Y, ldY, (int)n_lib, (int)T, E, params->tau, params->Tp,
                                        params->exclusion_radius, idx, w, (cudaStream_t)stream,
                                        (params->flags & EDM_FLAG_KNN_WARP) != 0));
    }
    return EDM_OK;
}

size_t edm_ccm_workspace_bytes(int64_t N, int64_t T, const edm_params *params)
{
    if (!params || N < 1 || T < 2)
        return 0;
    return ccm_ws_layout(N, T, params).total;
}

}  // extern "C"

namespace {

// A group of the device-side plan: targets of E in [elo, ehi] (static E
// set `sel` for the table layout), tb_max target-block slots from slot0 on,
// at most tiles_upper tiles per slot.
struct DevGroup {
    int elo, ehi;
    uint32_t sel;
    int slot0, tb_max, tiles_upper;
};

// Plan of the cross-map phase: targets grouped by E (stable) and tiles,
// either planned on the host (tiles known here) or on the device (dev:
// groups of fixed E ranges whose tile ranges live in slots_d).
struct CcmPlan {
    std::vector<edm::TileMeta> tiles;
    int32_t *pi_d;
    float2 *omom_d;
    edm::TileMeta *meta_d;
    float *tiles_d;
    uint8_t *tables_d;
    bool want_f16, scalar;
    bool l2;  // long series: tiles stay in global memory (FP32 only)
    int RB;
    CcmWs L;
    bool dev = false;
    std::vector<DevGroup> groups;
    int32_t *counts_d = nullptr;
    edm::SlotDesc *slots_d = nullptr;
};

int ccm_validate(int64_t N, int64_t T, int64_t ldY, const edm_params *params)
{
    int rc = check_common(params);
    if (rc)
        return rc;
    if (N < 1 || T < 2 || ldY < T)
        return EDM_ERR_INVALID;
    if (T > EDM_MAX_T || N > 0x7fffffffLL)
        return EDM_ERR_UNSUPPORTED;
    const bool scalar = (params->flags & EDM_FLAG_LOOKUP_SCALAR) != 0;
    if (scalar && params->precision != EDM_PRECISION_FP32)
        return EDM_ERR_INVALID;
    if (T > edm::knn_max_T() || (scalar && edm::lookup_smem_bytes((int)T) > 227u * 1024u))
        return EDM_ERR_UNSUPPORTED;
    return EDM_OK;
}

// Plan from host optE, upload it, stage the target tiles.
int ccm_prepare(const float *Y, int64_t N, int64_t T, int64_t ldY, const int32_t *E_host, const edm_params *params,
                void *ws, cudaStream_t st, CcmPlan &P)
{
    P.L = ccm_ws_layout(N, T, params);
    const CcmWs &L = P.L;
    P.scalar = (params->flags & EDM_FLAG_LOOKUP_SCALAR) != 0;
    P.RB = ccm_row_bytes(T, params);
    P.l2 = !P.scalar && edm::lookup_needs_l2((int)T);
    int64_t count[EDM_MAX_E + 2] = {0};
    for (int64_t j = 0; j < N; ++j) {
        int E = E_host[(size_t)j];
        if (E < 1 || E > EDM_MAX_E || ccm_min_candidates(T, E, params) < E + 1)
            return EDM_ERR_INVALID;
        count[E]++;
    }
    int64_t start[EDM_MAX_E + 2] = {0};
    for (int E = 1; E <= EDM_MAX_E; ++E)
        start[E + 1] = start[E] + count[E];
    std::vector<int32_t> pi((size_t)N);
    {
        int64_t fill[EDM_MAX_E + 2];
        memcpy(fill, start, sizeof fill);
        for (int64_t j = 0; j < N; ++j)
            pi[(size_t)fill[E_host[(size_t)j]]++] = (int32_t)j;
    }
    P.tiles.clear();
    P.want_f16 = params->precision == EDM_PRECISION_FP16_TARGETS && !P.l2;
    for (int E = 1; E <= EDM_MAX_E; ++E) {
        const bool f16 = P.want_f16 && E + 1 <= edm::kF16MaxK;
        const int width = f16 ? P.RB / 2 : P.RB / 4;
        for (int64_t c = 0; c < count[E]; c += width)
            P.tiles.push_back(edm::TileMeta{E, (int)(start[E] + c), (int)std::min<int64_t>(width, count[E] - c),
                                            f16 ? edm::kTileF16 : 0});
    }
    const int n_tiles = (int)P.tiles.size();
    unsigned char *wsb = (unsigned char *)ws;
    P.pi_d = (int32_t *)(wsb + L.pi);
    P.omom_d = (float2 *)(wsb + L.omom);
    P.meta_d = (edm::TileMeta *)(wsb + L.meta);
    P.tiles_d = (float *)(wsb + L.tiles);
    P.tables_d = (uint8_t *)(wsb + L.tables);
    EDM_CUDA(cudaMemcpyAsync(P.pi_d, pi.data(), (size_t)N * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    EDM_CUDA(cudaMemcpyAsync(P.meta_d, P.tiles.data(), P.tiles.size() * sizeof(edm::TileMeta), cudaMemcpyHostToDevice,
                             st));
    {
        LaunchScope ls(EDM_KERNEL_PREP, st, (double)N);
        EDM_CUDA(edm::launch_prep_targets(Y, ldY, (int)T, params->tau, params->Tp, P.pi_d, P.meta_d, n_tiles, P.tiles_d,
                                          P.omom_d, st, P.RB));
        if (P.want_f16)
            EDM_CUDA(edm::launch_prep_targets_f16(Y, ldY, (int)T, params->tau, params->Tp, P.pi_d, P.meta_d, n_tiles,
                                                  (uint8_t *)P.tiles_d, P.omom_d, st, P.RB));
    }
    // (pageable sources are staged before cudaMemcpyAsync returns, so the
    // host vectors may go away now)
    return EDM_OK;
}

// Whether every E in 1..EDM_MAX_E keeps E+1 candidates (queries and
// candidates from s_lo on): then the device plan can take any optE without
// a host check.
bool all_E_usable(int64_t T, const edm_params *p, int64_t s_lo)
{
    for (int E = 1; E <= EDM_MAX_E; ++E) {
        const int64_t A = std::max<int64_t>((int64_t)(E - 1) * p->tau, s_lo);
        const int64_t cand = T - p->Tp - A - (p->exclusion_radius >= 0 ? 2 * (int64_t)p->exclusion_radius + 1 : 0);
        if (cand < E + 1)
            return false;
    }
    return true;
}

// The host plan (one synchronisation to read optE) serves EDM_FLAG_VALIDATE
// (every optE checked, EDM_ERR_INVALID reported), the scalar comparison
// lookup, and series too short for some E; everything else plans on the
// device.
bool host_plan_needed(int64_t T, const edm_params *p, int64_t s_lo)
{
    return (p->flags & (EDM_FLAG_VALIDATE | EDM_FLAG_LOOKUP_SCALAR)) != 0 || !all_E_usable(T, p, s_lo);
}

// Plan on the device from device optE (no host synchronisation): fixed
// groups -- one over every E when the tiles sit in shared memory or all fit
// one target block, else (long series, tiles read from L2) one per E up to
// knn_thread_max_E() and one for the larger E, cut into target blocks --
// whose tile ranges the plan kernel writes into launch slots; targets with
// an unusable E get NaN rows (nan_* spec).  Then stage the target tiles.
int ccm_prepare_dev(const float *Y, int64_t N, int64_t T, int64_t ldY, const int32_t *optE_d, const edm_params *params,
                    void *ws, cudaStream_t st, CcmPlan &P, int s_lo, float *nan_rho, int64_t ld_rho, int64_t row_len,
                    int planes, int64_t plane_stride)
{
    P.L = ccm_ws_layout(N, T, params);
    const CcmWs &L = P.L;
    P.dev = true;
    P.scalar = false;
    P.RB = ccm_row_bytes(T, params);
    P.l2 = edm::lookup_needs_l2((int)T);
    P.want_f16 = params->precision == EDM_PRECISION_FP16_TARGETS && !P.l2;
    unsigned char *wsb = (unsigned char *)ws;
    P.pi_d = (int32_t *)(wsb + L.pi);
    P.omom_d = (float2 *)(wsb + L.omom);
    P.meta_d = (edm::TileMeta *)(wsb + L.meta);
    P.tiles_d = (float *)(wsb + L.tiles);
    P.tables_d = (uint8_t *)(wsb + L.tables);
    P.counts_d = (int32_t *)(wsb + L.counts);
    P.slots_d = (edm::SlotDesc *)(wsb + L.slots);
    const int f16 = P.want_f16 ? 1 : 0;
    const int n_tiles_max = (int)L.n_tiles_max;
    const int tpb = (int)std::max<size_t>(1, kTileBlockBytes / ((size_t)T * P.RB));
    P.groups.clear();
    auto upper = [&](int elo, int ehi) {
        int u = 0;
        if (elo == ehi)
            return (int)((N + edm::plan_tile_width(elo, f16, P.RB) - 1) / edm::plan_tile_width(elo, f16, P.RB));
        u = (int)((N + P.RB / 4 - 1) / (P.RB / 4)) + (ehi - elo + 1);
        return std::min(u, n_tiles_max);
    };
    if (n_tiles_max <= tpb || !P.l2) {
        P.groups.push_back(DevGroup{1, EDM_MAX_E, (1u << EDM_MAX_E) - 1u, 0, 1, n_tiles_max});
    } else {
        const int thr = edm::knn_thread_max_E();
        for (int E = 1; E <= thr; ++E)
            P.groups.push_back(DevGroup{E, E, 1u << (E - 1), 0, 1, upper(E, E)});
        uint32_t rare = 0;
        for (int E = thr + 1; E <= EDM_MAX_E; ++E)
            rare |= 1u << (E - 1);
        P.groups.push_back(DevGroup{thr + 1, EDM_MAX_E, rare, 0, 1, upper(thr + 1, EDM_MAX_E)});
    }
    edm::CcmPlanSpec sp{};
    sp.N = (int)N;
    sp.T = (int)T;
    sp.tau = params->tau;
    sp.Tp = params->Tp;
    sp.excl = params->exclusion_radius;
    sp.s_lo = s_lo;
    sp.f16 = f16;
    sp.RB = P.RB;
    sp.n_tiles_max = n_tiles_max;
    sp.n_groups = (int)P.groups.size();
    sp.tiles_per_block = P.l2 ? tpb : 0;
    int slot = 0;
    for (size_t g = 0; g < P.groups.size(); ++g) {
        DevGroup &G = P.groups[g];
        if (P.l2) {
            G.tb_max = (G.tiles_upper + tpb - 1) / tpb;
            G.tiles_upper = std::min(G.tiles_upper, tpb);
        }
        G.slot0 = slot;
        slot += G.tb_max;
        sp.g_lo[g] = G.elo;
        sp.g_hi[g] = G.ehi;
        sp.tb_max[g] = G.tb_max;
        sp.slot0[g] = G.slot0;
    }
    if ((size_t)slot > (size_t)edm::kMaxPlanGroups * (size_t)(L.n_tiles_max + 1))
        return EDM_ERR_UNSUPPORTED;
    sp.rho = nan_rho;
    sp.ld_rho = ld_rho;
    sp.row_len = row_len;
    sp.planes = planes;
    sp.plane_stride = plane_stride;
    {
        LaunchScope ls(EDM_KERNEL_PLAN, st, (double)N);
        EDM_CUDA(edm::launch_ccm_plan(optE_d, sp, P.counts_d, P.pi_d, P.meta_d, P.slots_d, st));
    }
    {
        LaunchScope ls(EDM_KERNEL_PREP, st, (double)N);
        EDM_CUDA(edm::launch_prep_targets(Y, ldY, (int)T, params->tau, params->Tp, P.pi_d, P.meta_d, n_tiles_max,
                                          P.tiles_d, P.omom_d, st, P.RB));
        if (P.want_f16)
            EDM_CUDA(edm::launch_prep_targets_f16(Y, ldY, (int)T, params->tau, params->Tp, P.pi_d, P.meta_d,
                                                  n_tiles_max, (uint8_t *)P.tiles_d, P.omom_d, st, P.RB));
    }
    return EDM_OK;
}

// Time-delay form: lags lag_min .. lag_min + n_lags - 1 cross-mapped from the
// same tables (queries and candidates from s_lo on); omom holds the
// observation sums of each lag ([n_lags][N]); lag l writes rho + l * stride.
struct LagSpec {
    int lag_min, n_lags, s_lo;
    const float2 *omom;
    int64_t rho_stride;
};

// Convergence form: each library block's tables are built once per
// candidate subset u (mask u of words 32-bit words) and cross-mapped into
// rho + u * rho_stride.
struct SubsetSpec {
    const uint32_t *masks;
    int n_sub;
    int64_t words;
    int64_t rho_stride;
};

// Cross map of libraries [lib_begin, lib_begin + lib_count) into rho
// (target-major, ld_rho) with a prepared plan.
int ccm_execute(const CcmPlan &P, const float *Y, int64_t N, int64_t T, int64_t ldY, int64_t lib_begin,
                int64_t lib_count, const edm_params *params, float *rho, int64_t ld_rho, cudaStream_t st,
                const LagSpec *lags = nullptr, const SubsetSpec *subsets = nullptr)
{
    const CcmWs &L = P.L;
    const std::vector<edm::TileMeta> &tiles = P.tiles;
    const int n_tiles = (int)tiles.size();
    const bool scalar = P.scalar;
    int32_t *pi_d = P.pi_d;
    float2 *omom_d = P.omom_d;
    edm::TileMeta *meta_d = P.meta_d;
    float *tiles_d = P.tiles_d;
    uint8_t *tables_d = P.tables_d;
    const int sms = sm_count();
    // shared-memory tiles: at least ~16 CTAs per SM in all (one CTA per SM
    // is resident), so the last wave is a small tail; tiles in L2: 4 per SM
    // per register class
    const int want = (P.l2 ? 4 : 16) * sms;
    // --- target groups x library blocks ----------------------------------------
    // Tiles in shared memory: one group over every E; a library block's
    // tables (one warp-kernel sweep per library builds every E in use) are
    // read by all tiles, which stream through shared memory, the largest E
    // first; each warp prefetches its next library's table into L2.  Tiles
    // read from L2 (long series): one group per E up to knn_thread_max_E()
    // (the tables of that E, one build per library) and one for the larger
    // E, each cut into L2-sized target blocks so its tiles stay resident
    // while every library block sweeps them.  Either way every (library, E)
    // table is built once per target block.
    struct LaunchGroup {
        uint32_t sel;                  // E set of the table layout
        int tb0, ntb;                  // host plan: tile range
        const edm::SlotDesc *slot;     // device plan: the slot
        int grid;                      // device plan: upper-bound grid
        bool first;                    // device plan: carries the launch's pair count
    };
    std::vector<LaunchGroup> groups;
    if (P.dev) {
        for (size_t g = 0; g < P.groups.size(); ++g) {
            const DevGroup &G = P.groups[g];
            for (int tb = 0; tb < G.tb_max; ++tb)
                groups.push_back(LaunchGroup{G.sel, 0, 0, P.slots_d + G.slot0 + tb,
                                             G.tiles_upper + (P.l2 ? 2 : 1) * want, g == 0 && tb == 0});
        }
    } else {
        const size_t tile_bytes = (size_t)T * P.RB;
        const int tiles_per_block = (int)std::max<size_t>(1, kTileBlockBytes / tile_bytes);
        std::vector<std::pair<int, int>> ranges;  // tile ranges [first, last)
        // tiles in shared memory, or all tiles within one target block: one
        // group, so one warp-kernel sweep per library builds the tables of
        // every E in use (measured at N = 101,729, T = 1,500: kNN 4.45 s
        // against 5.05 s for per-E groups with the thread kernel for E <= 6,
        // lookup 11.24 against 11.41 s with the largest-E tiles scheduled
        // first)
        if (n_tiles <= tiles_per_block || !P.l2)
            ranges.emplace_back(0, n_tiles);
        for (int t0 = ranges.empty() ? 0 : n_tiles; t0 < n_tiles;) {
            const int E = tiles[(size_t)t0].E;
            int t1 = t0 + 1;
            if (E <= edm::knn_thread_max_E())
                while (t1 < n_tiles && tiles[(size_t)t1].E == E)
                    ++t1;
            else
                t1 = n_tiles;
            if (P.l2)
                for (int b = t0; b < t1; b += tiles_per_block)
                    ranges.emplace_back(b, std::min(t1, b + tiles_per_block));
            else
                ranges.emplace_back(t0, t1);
            t0 = t1;
        }
        for (const auto &r : ranges) {
            uint32_t sel = 0;
            for (int t = r.first; t < r.second; ++t)
                sel |= 1u << (tiles[(size_t)t].E - 1);
            groups.push_back(LaunchGroup{sel, r.first, r.second - r.first, nullptr, 0, false});
        }
    }
    for (const auto &g : groups) {
        const uint32_t sel = g.sel;
        const uint32_t *sel_dev = g.slot ? &g.slot->sel : nullptr;
        const edm::TableLayout lay = make_layout(sel, T, params);
        // L2-sized library blocks; blocks of rare-E target blocks (many E,
        // few tiles) may spill to HBM rather than shrink below kMinLibBlock
        const int64_t per_block = std::min<int64_t>(
            65535, std::max<int64_t>(std::min<int64_t>(min_lib_block(T), (int64_t)(L.table_cap / (size_t)lay.lib_stride)),
                                     (int64_t)(L.table_bytes / (size_t)lay.lib_stride)));
        for (int64_t lb0 = 0; lb0 < lib_count; lb0 += per_block)
          for (int su = 0; su < (subsets ? subsets->n_sub : 1); ++su) {
            const int nlb = (int)std::min<int64_t>(per_block, lib_count - lb0);
            {
                int n_knn = 1;
                LaunchScope ls(EDM_KERNEL_KNN, st, (double)nlb * __builtin_popcount(sel), 0);
                if (subsets)  // candidate subsets: the warp kernel (mask test per candidate)
                    EDM_CUDA(edm::launch_knn_tables(Y, ldY, lib_begin + lb0, nlb, (int)T, params->tau, params->Tp,
                                                    params->exclusion_radius, sel, lay, tables_d, st, 64, sel_dev, 0,
                                                    subsets->masks + (size_t)su * subsets->words));
                else
                    EDM_CUDA(edm::launch_knn_tables_auto(Y, ldY, lib_begin + lb0, nlb, (int)T, params->tau,
                                                         params->Tp, params->exclusion_radius, sel, lay, tables_d, st,
                                                         (params->flags & EDM_FLAG_KNN_WARP) != 0,
                                                         lags ? lags->s_lo : 0, &n_knn, sel_dev));
                ls.add_launches(EDM_KERNEL_KNN, n_knn);
            }
            // pairs of this launch (device plan: the whole block's N x nlb is
            // counted on the first group's launches)
            double pairs = 0.0;
            if (g.slot) {
                pairs = g.first ? (double)N * (double)nlb : 0.0;
            } else {
                int64_t targets = 0;
                for (int t = g.tb0; t < g.tb0 + g.ntb; ++t)
                    targets += tiles[(size_t)t].count;
                pairs = (double)targets * (double)nlb;
            }
            edm::LookupArgs a;
            a.tiles = tiles_d;
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
            a.n_lib = nlb;
            a.rho_col0 = lb0;
            a.rho = subsets ? rho + su * subsets->rho_stride : rho;
            a.ld_rho = ld_rho;
            if (scalar) {
                // comparison path (host plan only): one launch per run of equal E
                for (int r0 = g.tb0; r0 < g.tb0 + g.ntb;) {
                    const int E = tiles[(size_t)r0].E;
                    int r1 = r0;
                    int64_t tg = 0;
                    while (r1 < g.tb0 + g.ntb && tiles[(size_t)r1].E == E)
                        tg += tiles[(size_t)r1++].count;
                    a.tile_begin = r0;
                    a.n_tiles = r1 - r0;
                    int parts = (4 * sms + a.n_tiles - 1) / a.n_tiles;
                    a.lib_parts = std::max(1, std::min(parts, (nlb + 7) / 8));
                    LaunchScope ls(EDM_KERNEL_LOOKUP, st, (double)tg * (double)nlb);
                    EDM_CUDA(edm::launch_lookup(a, E, st));
                    r0 = r1;
                }
            } else {
                int n_small = 0;
                if (g.slot) {
                    a.slot = g.slot;
                    a.want = want;
                    a.tile_begin = 0;
                    a.n_tiles = g.grid;
                    a.lib_parts = 1;
                } else {
                    a.tile_begin = g.tb0;
                    a.n_tiles = g.ntb;
                    int parts = (want + g.ntb - 1) / g.ntb;
                    a.lib_parts = std::max(1, std::min(parts, (nlb + 7) / 8));
                    // tiles read from L2: one launch per register class present
                    while (P.l2 && n_small < g.ntb && tiles[(size_t)(g.tb0 + n_small)].E + 1 <= edm::kL2SplitK)
                        ++n_small;
                }
                const int n_lk = lags ? lags->n_lags : 1;
                const int lk_launches = !P.l2 ? 1 : (g.slot ? 2 : (n_small > 0) + (g.ntb - n_small > 0));
                for (int li = 0; li < n_lk; ++li) {
                    if (lags) {
                        a.s_lo = lags->s_lo;
                        a.lag = lags->lag_min + li;
                        a.omom = lags->omom + (size_t)li * N;
                        a.rho = rho + li * lags->rho_stride;
                    }
                    LaunchScope ls(EDM_KERNEL_LOOKUP, st, pairs, lk_launches);
                    if (P.l2) {
                        EDM_CUDA(edm::launch_lookup_l2(a, n_small, sms, st));
                    } else {
                        EDM_CUDA(edm::launch_lookup_multi(a, P.RB, st));
                    }
                }
            }
        }
    }
    return EDM_OK;
}

}  // namespace

extern "C" {

int edm_ccm_rho(const float *Y, int64_t N, int64_t T, int64_t ldY, const int32_t *optE, int64_t lib_begin,
                int64_t lib_count, const edm_params *params, float *rho, int64_t ld_rho, void *ws, size_t ws_bytes,
                void *stream)
{
    int rc = ccm_validate(N, T, ldY, params);
    if (rc)
        return rc;
    if (!Y || !optE || !rho || !ws)
        return EDM_ERR_INVALID;
    if (lib_begin < 0 || lib_count < 0 || lib_begin + lib_count > N || ld_rho < lib_count)
        return EDM_ERR_INVALID;
    if (ws_bytes < ccm_ws_layout(N, T, params).total)
        return EDM_ERR_WORKSPACE;
    if ((rc = validate_series(Y, N, T, ldY, params, (cudaStream_t)stream)) != EDM_OK)
        return rc;
    if (lib_count == 0)
        return EDM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    CcmPlan P;
    if (host_plan_needed(T, params, 0)) {
        std::vector<int32_t> E_host((size_t)N);
        EDM_CUDA(cudaMemcpyAsync(E_host.data(), optE, (size_t)N * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        EDM_CUDA(cudaStreamSynchronize(st));
        rc = ccm_prepare(Y, N, T, ldY, E_host.data(), params, ws, st, P);
    } else {
        rc = ccm_prepare_dev(Y, N, T, ldY, optE, params, ws, st, P, 0, rho, ld_rho, lib_count, 1, 0);
    }
    if (rc)
        return rc;
    return ccm_execute(P, Y, N, T, ldY, lib_begin, lib_count, params, rho, ld_rho, st);
}

size_t edm_ccm_rho_lags_workspace_bytes(int64_t N, int64_t T, int32_t lag_min, int32_t lag_max,
                                        const edm_params *params)
{
    if (!params || N < 1 || T < 2 || lag_max < lag_min)
        return 0;
    edm_params pe = *params;
    pe.Tp = std::max(lag_max, 0);
    return ccm_ws_layout(N, T, &pe).total + align256((size_t)(lag_max - lag_min + 1) * N * sizeof(float2));
}

int edm_ccm_rho_lags(const float *Y, int64_t N, int64_t T, int64_t ldY, const int32_t *optE, int32_t lag_min,
                     int32_t lag_max, const edm_params *params, float *rho, int64_t ld_rho, void *ws, size_t ws_bytes,
                     void *stream)
{
    if (!params || lag_max < lag_min || lag_max - lag_min >= 4096 || lag_max > 65535 || lag_min < -65535)
        return EDM_ERR_INVALID;
    edm_params pe = *params;
    pe.Tp = std::max(lag_max, 0);
    int rc = ccm_validate(N, T, ldY, &pe);
    if (rc)
        return rc;
    if (pe.flags & EDM_FLAG_LOOKUP_SCALAR)
        return EDM_ERR_UNSUPPORTED;
    if (!Y || !optE || !rho || !ws || ld_rho < N)
        return EDM_ERR_INVALID;
    const int n_lags = lag_max - lag_min + 1;
    const int s_lo = std::max(0, -lag_min);
    const size_t base = ccm_ws_layout(N, T, &pe).total;
    if (ws_bytes < base + align256((size_t)n_lags * N * sizeof(float2)))
        return EDM_ERR_WORKSPACE;
    if ((rc = validate_series(Y, N, T, ldY, &pe, (cudaStream_t)stream)) != EDM_OK)
        return rc;
    cudaStream_t st = (cudaStream_t)stream;
    CcmPlan P;
    if (host_plan_needed(T, &pe, s_lo)) {
        std::vector<int32_t> E_host((size_t)N);
        EDM_CUDA(cudaMemcpyAsync(E_host.data(), optE, (size_t)N * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        EDM_CUDA(cudaStreamSynchronize(st));
        for (int64_t j = 0; j < N; ++j) {  // every lag's window must hold k neighbours
            const int E = E_host[(size_t)j];
            if (E < 1 || E > EDM_MAX_E)
                return EDM_ERR_INVALID;
            const int64_t A = std::max<int64_t>((int64_t)(E - 1) * pe.tau, s_lo);
            int64_t cand = (T - pe.Tp) - A;
            if (pe.exclusion_radius >= 0)
                cand -= 2 * (int64_t)pe.exclusion_radius + 1;
            if (cand < E + 1)
                return EDM_ERR_INVALID;
        }
        rc = ccm_prepare(Y, N, T, ldY, E_host.data(), &pe, ws, st, P);
    } else {
        rc = ccm_prepare_dev(Y, N, T, ldY, optE, &pe, ws, st, P, s_lo, rho, ld_rho, N, n_lags, N * ld_rho);
    }
    if (rc)
        return rc;
    float2 *omom_l = (float2 *)((unsigned char *)ws + base);
    const int n_tiles_l = P.dev ? (int)P.L.n_tiles_max : (int)P.tiles.size();
    {
        LaunchScope ls(EDM_KERNEL_PREP, st, (double)N * n_lags, n_lags);
        for (int li = 0; li < n_lags; ++li)
            EDM_CUDA(edm::launch_obs_moments(P.tiles_d, P.RB, P.meta_d, n_tiles_l, (int)T, pe.tau, pe.Tp, s_lo,
                                             lag_min + li, omom_l + (size_t)li * N, st));
    }
    LagSpec spec{lag_min, n_lags, s_lo, omom_l, N * ld_rho};
    return ccm_execute(P, Y, N, T, ldY, 0, N, &pe, rho, ld_rho, st, &spec);
}

int edm_ccm_rho_subsets(const float *Y, int64_t N, int64_t T, int64_t ldY, const int32_t *optE,
                        const uint32_t *masks, int32_t n_sub, int64_t words, const edm_params *params, float *rho,
                        int64_t ld_rho, void *ws, size_t ws_bytes, void *stream)
{
    int rc = ccm_validate(N, T, ldY, params);
    if (rc)
        return rc;
    if (params->flags & EDM_FLAG_LOOKUP_SCALAR)
        return EDM_ERR_UNSUPPORTED;
    if (!Y || !optE || !masks || !rho || !ws || n_sub < 1 || words * 32 < T || ld_rho < N)
        return EDM_ERR_INVALID;
    if (ws_bytes < ccm_ws_layout(N, T, params).total)
        return EDM_ERR_WORKSPACE;
    if ((rc = validate_series(Y, N, T, ldY, params, (cudaStream_t)stream)) != EDM_OK)
        return rc;
    cudaStream_t st = (cudaStream_t)stream;
    SubsetSpec spec{masks, n_sub, words, N * ld_rho};
    if (!host_plan_needed(T, params, 0)) {
        // planned on the device; a subset that leaves too few candidates for
        // the largest E in use gets a NaN plane afterwards
        CcmPlan P;
        rc = ccm_prepare_dev(Y, N, T, ldY, optE, params, ws, st, P, 0, rho, ld_rho, N, n_sub, N * ld_rho);
        if (rc)
            return rc;
        if ((rc = ccm_execute(P, Y, N, T, ldY, 0, N, params, rho, ld_rho, st, nullptr, &spec)) != EDM_OK)
            return rc;
        EDM_CUDA(edm::launch_subset_check(masks, n_sub, words, P.counts_d, (int)N, (int)T, params->tau, params->Tp,
                                          params->exclusion_radius, rho, ld_rho, N * ld_rho, st));
        return EDM_OK;
    }
    std::vector<int32_t> E_host((size_t)N);
    std::vector<uint32_t> m_host((size_t)n_sub * (size_t)words);
    EDM_CUDA(cudaMemcpyAsync(E_host.data(), optE, (size_t)N * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    EDM_CUDA(cudaMemcpyAsync(m_host.data(), masks, m_host.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    EDM_CUDA(cudaStreamSynchronize(st));
    // every query of every subset must keep E+1 candidates: allowed points in
    // the candidate range, less the exclusion window, at the largest E in use
    int E_top = 0;
    for (int64_t j = 0; j < N; ++j)
        E_top = std::max(E_top, (int)E_host[(size_t)j]);
    if (E_top < 1 || E_top > EDM_MAX_E)
        return EDM_ERR_INVALID;
    const int64_t lo = (int64_t)(E_top - 1) * params->tau, hi = T - 1 - params->Tp;
    for (int u = 0; u < n_sub; ++u) {
        int64_t c = 0;
        for (int64_t s2 = lo; s2 <= hi; ++s2)
            c += (m_host[(size_t)u * words + (size_t)(s2 >> 5)] >> (s2 & 31)) & 1u;
        if (params->exclusion_radius >= 0)
            c -= 2 * (int64_t)params->exclusion_radius + 1;
        if (c < E_top + 1)
            return EDM_ERR_INVALID;
    }
    CcmPlan P;
    rc = ccm_prepare(Y, N, T, ldY, E_host.data(), params, ws, st, P);
    if (rc)
        return rc;
    return ccm_execute(P, Y, N, T, ldY, 0, N, params, rho, ld_rho, st, nullptr, &spec);
}

size_t edm_ccm_host_workspace_bytes(int64_t N, int64_t T, int64_t block, const edm_params *params)
{
    if (!params || N < 1 || T < 2)
        return 0;
    if (block <= 0)
        block = std::min<int64_t>(N, std::max<int64_t>(256, (int64_t)((1ull << 30) / ((size_t)N * 4))));
    return align256((size_t)N * T * 4) + align256((size_t)N * 4) + 2 * align256((size_t)N * block * 4) +
           ccm_ws_layout(N, T, params).total;
}

int edm_ccm_host(const float *Y_host, int64_t N, int64_t T, const edm_params *params, int32_t *optE_host,
                 float *rho_host, int64_t ld_rho, int64_t block, void *ws, size_t ws_bytes, void *stream)
{
    int rc = ccm_validate(N, T, T, params);
    if (rc)
        return rc;
    if (!Y_host || !optE_host || !rho_host || !ws || ld_rho < N)
        return EDM_ERR_INVALID;
    if (block <= 0)
        block = std::min<int64_t>(N, std::max<int64_t>(256, (int64_t)((1ull << 30) / ((size_t)N * 4))));
    block = std::min<int64_t>(block, N);
    if (ws_bytes < edm_ccm_host_workspace_bytes(N, T, block, params))
        return EDM_ERR_WORKSPACE;
    const int64_t h = T / 2;
    const int64_t span = (int64_t)(params->E_max - 1) * params->tau;
    if (params->E_max < 1 || params->E_max > EDM_MAX_E || h - params->Tp - span < params->E_max + 1 ||
        (T - h) - params->Tp - span < 2)
        return EDM_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *w = (unsigned char *)ws;
    float *Yd = (float *)w;
    w += align256((size_t)N * T * 4);
    int32_t *optE_d = (int32_t *)w;
    w += align256((size_t)N * 4);
    float *blk[2];
    blk[0] = (float *)w;
    w += align256((size_t)N * block * 4);
    blk[1] = (float *)w;
    w += align256((size_t)N * block * 4);
    void *ccm_ws = w;

    EDM_CUDA(cudaMemcpyAsync(Yd, Y_host, (size_t)N * T * 4, cudaMemcpyHostToDevice, st));
    {
        LaunchScope ls(EDM_KERNEL_SIMPLEX, st, (double)N);
        EDM_CUDA(edm::launch_simplex(Yd, N, (int)T, T, params->E_max, params->tau, params->Tp, optE_d, nullptr, st));
    }
    EDM_CUDA(cudaMemcpyAsync(optE_host, optE_d, (size_t)N * 4, cudaMemcpyDeviceToHost, st));
    EDM_CUDA(cudaStreamSynchronize(st));
    CcmPlan P;
    rc = ccm_prepare(Yd, N, T, T, optE_host, params, ccm_ws, st, P);
    if (rc)
        return rc;
    // library blocks: compute on `st`, copy back on a second stream while
    // the next block computes (two device buffers)
    cudaStream_t cp = nullptr;
    cudaEvent_t done_c[2] = {nullptr, nullptr}, done_d[2] = {nullptr, nullptr};
    cudaError_t e = cudaStreamCreateWithFlags(&cp, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaEventCreateWithFlags(&done_c[b], cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&done_d[b], cudaEventDisableTiming);
    }
    int k = 0;
    for (int64_t b0 = 0; b0 < N && e == cudaSuccess && rc == EDM_OK; b0 += block, ++k) {
        const int64_t nb = std::min<int64_t>(block, N - b0);
        const int buf = k & 1;
        if (k >= 2 && (e = cudaStreamWaitEvent(st, done_d[buf], 0)) != cudaSuccess)
            break;
        rc = ccm_execute(P, Yd, N, T, T, b0, nb, params, blk[buf], nb, st);
        if (rc)
            break;
        if ((e = cudaEventRecord(done_c[buf], st)) != cudaSuccess || (e = cudaStreamWaitEvent(cp, done_c[buf], 0)) != cudaSuccess)
            break;
        e = cudaMemcpy2DAsync(rho_host + b0, (size_t)ld_rho * 4, blk[buf], (size_t)nb * 4, (size_t)nb * 4, (size_t)N,
                              cudaMemcpyDeviceToHost, cp);
        if (e == cudaSuccess)
            e = cudaEventRecord(done_d[buf], cp);
    }
    cudaError_t e2 = cudaStreamSynchronize(cp);
    if (e == cudaSuccess)
        e = e2;
    for (int b = 0; b < 2; ++b) {
        if (done_c[b])
            cudaEventDestroy(done_c[b]);
        if (done_d[b])
            cudaEventDestroy(done_d[b]);
    }
    if (cp)
        cudaStreamDestroy(cp);
    if (rc)
        return rc;
    if (e != cudaSuccess)
        return cuda_fail(e);
    EDM_CUDA(cudaStreamSynchronize(st));
    return EDM_OK;
}

// ---------------------------------------------------------------------------
// Adjoint
// ---------------------------------------------------------------------------
namespace {
// Table budget of the adjoint: all libraries at once when they fit in 1 GB
// (the library pass runs one CTA per library of a block, so larger blocks
// fill the GPU and the kNN and target passes run fewer times), else blocks
// of as many libraries as 1 GB holds.
constexpr size_t kBwTableBytes = 1ull << 30;

struct BwWs {
    size_t pi, e_start, counts, meta, obar, stats, tables, table_bytes, total;
    int64_t n_tiles_max;
};

BwWs bw_layout(int64_t N, int64_t T, const edm_params *p)
{
    BwWs w;
    size_t off = 0;
    w.pi = off;
    off += align256((size_t)N * 4);
    w.e_start = off;
    off += 256;
    // device-side plan (counts, and the tile list the plan kernel writes
    // for 32-target tiles)
    w.counts = off;
    off += 256;
    w.n_tiles_max = (N + 31) / 32 + EDM_MAX_E;
    w.meta = off;
    off += align256((size_t)w.n_tiles_max * sizeof(edm::TileMeta));
    w.obar = off;
    off += align256((size_t)N * 4);
    w.stats = off;
    off += align256((size_t)N * (size_t)N * 16);
    w.tables = off;
    edm::TableLayout all = make_layout((1u << EDM_MAX_E) - 1u, T, p);
    w.table_bytes = std::max(std::min(kBwTableBytes, (size_t)N * all.lib_stride), (size_t)all.lib_stride);
    off += align256(w.table_bytes);
    w.total = off;
    return w;
}
}  // namespace

size_t edm_ccm_backward_workspace_bytes(int64_t N, int64_t T, const edm_params *params)
{
    if (!params || N < 1 || T < 2)
        return 0;
    return bw_layout(N, T, params).total;
}

int edm_ccm_rho_backward(const float *Y, int64_t N, int64_t T, int64_t ldY, const int32_t *optE,
                         const float *grad_rho, int64_t ld_g, const edm_params *params, float *grad_Y, void *ws,
                         size_t ws_bytes, void *stream)
{
    int rc = check_common(params);
    if (rc)
        return rc;
    if (!Y || !optE || !grad_rho || !grad_Y || !ws || N < 1 || T < 2 || ldY < T || ld_g < N)
        return EDM_ERR_INVALID;
    if (T > EDM_MAX_T || N > 0x7fffffffLL || T - params->Tp > edm::bw_max_T() || T > edm::knn_max_T())
        return EDM_ERR_UNSUPPORTED;
    const BwWs L = bw_layout(N, T, params);
    if (ws_bytes < L.total)
        return EDM_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *wsb = (unsigned char *)ws;
    // the target permutation by E and the E ranges, planned on the device
    // (targets whose E is unusable are left out: no rho, no gradient)
    {
        edm::CcmPlanSpec sp{};
        sp.N = (int)N;
        sp.T = (int)T;
        sp.tau = params->tau;
        sp.Tp = params->Tp;
        sp.excl = params->exclusion_radius;
        sp.f16 = 0;
        sp.RB = 128;
        sp.n_tiles_max = (int)L.n_tiles_max;
        sp.n_groups = 1;  // one slot: the E in use, for the kNN sweep
        sp.g_lo[0] = 1;
        sp.g_hi[0] = EDM_MAX_E;
        sp.tb_max[0] = 1;
        sp.slot0[0] = 0;
        sp.starts = (int32_t *)(wsb + L.e_start);
        LaunchScope ls(EDM_KERNEL_PLAN, st, (double)N);
        EDM_CUDA(edm::launch_ccm_plan(optE, sp, (int32_t *)(wsb + L.counts), (int32_t *)(wsb + L.pi),
                                      (edm::TileMeta *)(wsb + L.meta), (edm::SlotDesc *)(wsb + L.counts + 128), st));
    }
    // tables for every E in the layout; the kNN sweep builds only the E in
    // use (device mask)
    const uint32_t sel = (1u << EDM_MAX_E) - 1u;
    const uint32_t *sel_dev = &((const edm::SlotDesc *)(wsb + L.counts + 128))->sel;
    const int kmax = EDM_MAX_E + 1;
    EDM_CUDA(cudaMemset2DAsync(grad_Y, (size_t)ldY * 4, 0, (size_t)T * 4, (size_t)N, st));
    const edm::TableLayout lay = make_layout(sel, T, params);
    const int64_t per_block =
        std::min<int64_t>(65535, std::max<int64_t>(1, (int64_t)(L.table_bytes / (size_t)lay.lib_stride)));
    for (int64_t lb0 = 0; lb0 < N; lb0 += per_block) {
        const int nlb = (int)std::min<int64_t>(per_block, N - lb0);
        {
            LaunchScope ls(EDM_KERNEL_KNN, st, (double)nlb * __builtin_popcount(sel));
            int n_knn = 1;
            EDM_CUDA(edm::launch_knn_tables_auto(Y, ldY, lb0, nlb, (int)T, params->tau, params->Tp,
                                                 params->exclusion_radius, sel, lay, wsb + L.tables, st,
                                                 (params->flags & EDM_FLAG_KNN_WARP) != 0, 0, &n_knn, sel_dev));
            ls.add_launches(EDM_KERNEL_KNN, n_knn - 1);
        }
        edm::BwArgs a;
        a.Y = Y;
        a.ldY = ldY;
        a.T = (int)T;
        a.tau = params->tau;
        a.Tp = params->Tp;
        a.excl = params->exclusion_radius;
        a.optE = optE;
        a.grad_rho = grad_rho;
        a.ld_g = ld_g;
        a.tables = wsb + L.tables;
        a.lay = lay;
        a.lib0 = lb0;
        a.n_lib = nlb;
        a.N = (int)N;
        a.stats = (float4 *)(wsb + L.stats);
        a.obar = (float *)(wsb + L.obar);
        a.pi = (const int32_t *)(wsb + L.pi);
        a.e_start = (const int32_t *)(wsb + L.e_start);
        a.grad_Y = grad_Y;
        EDM_CUDA(edm::launch_backward(a, kmax, st));
    }
    return EDM_OK;
}

}  // extern "C"
