// batched.cu -- many independent datasets of uneven N and T in one
// CUDA-graph launch (edm_ccm_rho_batched).
//
// Every dataset runs the same kernels as edm_optimal_E + edm_ccm_rho, but
// the grouping of its targets by E is planned on the device (no host round
// trip), so the whole batch -- phase 1, plan, staging, kNN tables and
// lookup of every dataset -- is stream-captured once into a CUDA graph and
// replayed with one cudaGraphLaunch.  Launch shapes that depend on the
// data are upper bounds: tiles past a dataset's real tile count carry E = 0
// and exit at once, and the kNN kernel reads the set of E in use from
// device memory.  Datasets are spread over a few parallel graph branches
// (longest-processing-time first), each branch owning a workspace region
// for its tiles and tables, so small datasets do not leave the GPU idle.
//
// Tile shapes are chosen by measurement: the first call times the kNN
// query points per CTA and the lookup grid split on the largest dataset of
// each (series length, size, precision) class and caches the winners.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "launchers.h"

namespace edm {

namespace {

constexpr int kBranches = 4;    // parallel graph branches
constexpr int kGraphCache = 8;  // instantiated graphs kept

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

// Tables for every E <= E_max (the E in use are only known on the device).
TableLayout all_e_layout(int64_t T, const edm_params *p)
{
    TableLayout lay;
    lay.Tq_pad = (int)(((T - p->Tp) + 31) / 32 * 32);
    int64_t off = 0;
    for (int E = 0; E <= EDM_MAX_E; ++E)
        lay.off_w[E] = lay.off_i[E] = -1;
    for (int E = 1; E <= p->E_max; ++E) {
        lay.off_w[E] = off;
        off += (int64_t)al256((size_t)(E + 1) * lay.Tq_pad * sizeof(float));
        lay.off_i[E] = off;
        off += (int64_t)al256((size_t)(E + 1) * lay.Tq_pad * sizeof(uint16_t));
    }
    lay.lib_stride = off;
    return lay;
}

// Upper bound on the tiles of N targets: FP32 tiles of RB/4 targets, one
// partial tile per E.
int tiles_max(int64_t N, int RB, int E_max) { return (int)((N + RB / 4 - 1) / (RB / 4)) + E_max; }

struct SetPlan {
    size_t meta_area;  // counts[64] + sel, pi[N], omom[N], meta[n_tiles_max]
    int RB, n_tiles_max, branch;
};
struct BranchArea {
    size_t tiles, tables;  // region offsets
};
struct BatchLayout {
    std::vector<SetPlan> sets;
    std::vector<BranchArea> br;
    size_t total;
};

double set_cost(const edm_dataset &d)
{
    const double N = (double)d.N, T = (double)d.T;
    return N * N * T + 4.0 * N * T * T;  // lookup + kNN, roughly
}

size_t set_meta_bytes(int64_t N, int n_tiles_max)
{
    return 256 + al256((size_t)N * 4) + al256((size_t)N * sizeof(float2)) + al256((size_t)n_tiles_max * sizeof(TileMeta));
}

BatchLayout batch_layout(const edm_dataset *sets, int n, const edm_params *p)
{
    BatchLayout B;
    const int nb = std::min(kBranches, n);
    std::vector<int> order((size_t)n);
    for (int d = 0; d < n; ++d)
        order[(size_t)d] = d;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return set_cost(sets[a]) > set_cost(sets[b]); });
    std::vector<double> load((size_t)nb, 0.0);
    std::vector<size_t> tiles_need((size_t)nb, 0), tables_need((size_t)nb, 0);
    B.sets.resize((size_t)n);
    for (int d : order) {
        const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[(size_t)b] += set_cost(sets[d]);
        SetPlan &s = B.sets[(size_t)d];
        s.RB = chunked_row_bytes((int)sets[d].T);
        s.n_tiles_max = tiles_max(sets[d].N, s.RB, p->E_max);
        s.branch = b;
        tiles_need[(size_t)b] = std::max(tiles_need[(size_t)b], (size_t)s.n_tiles_max * (size_t)sets[d].T * s.RB);
        tables_need[(size_t)b] =
            std::max(tables_need[(size_t)b], (size_t)sets[d].N * (size_t)all_e_layout(sets[d].T, p).lib_stride);
    }
    size_t off = 0;
    for (int d = 0; d < n; ++d) {
        B.sets[(size_t)d].meta_area = off;
        off += set_meta_bytes(sets[d].N, B.sets[(size_t)d].n_tiles_max);
    }
    B.br.resize((size_t)nb);
    for (int b = 0; b < nb; ++b) {
        B.br[(size_t)b].tiles = off;
        off += al256(tiles_need[(size_t)b]);
        B.br[(size_t)b].tables = off;
        off += al256(tables_need[(size_t)b]);
    }
    B.total = off;
    return B;
}

// --- autotuner ----------------------------------------------------------
struct Tune {
    int q_per_cta;     // kNN query points per CTA
    int parts_factor;  // lookup CTAs ~ parts_factor x SMs
};
struct TuneEntry {
    int cls;
    Tune t;
};
std::vector<TuneEntry> g_tune;

int tune_class(const edm_dataset &d, int precision)
{
    int nb = 0;
    while ((64ll << nb) < d.N && nb < 15)
        ++nb;
    return (int)((d.T + 511) / 512) * 64 + nb * 2 + precision;
}

bool tune_find(int cls, Tune &out)
{
    for (const TuneEntry &e : g_tune)
        if (e.cls == cls) {
            out = e.t;
            return true;
        }
    return false;
}

int sm_count_dev()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 148;
    return n > 0 ? n : 148;
}

// --- graph cache ----------------------------------------------------------
struct GraphEntry {
    std::vector<edm_dataset> sets;
    edm_params params;
    void *ws;
    size_t ws_bytes;
    int device;
    cudaGraphExec_t exec;
    int64_t launches[EDM_KERNEL_COUNT];
    double pairs;
};
std::vector<GraphEntry> g_graphs;
std::mutex g_mu;

bool same_call(const GraphEntry &g, const edm_dataset *sets, int n, const edm_params *p, void *ws, size_t ws_bytes,
               int dev)
{
    return g.device == dev && g.ws == ws && g.ws_bytes == ws_bytes && (int)g.sets.size() == n &&
           memcmp(&g.params, p, sizeof *p) == 0 && memcmp(g.sets.data(), sets, sizeof(edm_dataset) * (size_t)n) == 0;
}

}  // namespace

// Device plan of one dataset: per-E counts, stable counting sort of the
// target indices by E, the tile list (tiles past the real count get E = 0)
// and the set of E in use.  One CTA; N <= 65535.
__global__ void __launch_bounds__(1024) batch_plan_kernel(const int32_t *__restrict__ optE, int N, int f16, int RB,
                                                          int n_tiles_max, int32_t *__restrict__ pi,
                                                          TileMeta *__restrict__ meta, uint32_t *__restrict__ sel)
{
    __shared__ int cnt[EDM_MAX_E + 1];
    __shared__ int start[EDM_MAX_E + 1];
    __shared__ int tstart[EDM_MAX_E + 1];
    __shared__ int total_tiles;
    if (threadIdx.x <= EDM_MAX_E)
        cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const int E = optE[j];
        atomicAdd(&cnt[(E >= 1 && E <= EDM_MAX_E) ? E : 0], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0, ts = 0;
        uint32_t m = 0;
        for (int E = 1; E <= EDM_MAX_E; ++E) {
            start[E] = s;
            tstart[E] = ts;
            s += cnt[E];
            const int w = (f16 && E + 1 <= kF16MaxK) ? RB / 2 : RB / 4;
            ts += (cnt[E] + w - 1) / w;
            if (cnt[E])
                m |= 1u << (E - 1);
        }
        total_tiles = min(ts, n_tiles_max);
        *sel = m;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int E = warp + 1; E <= EDM_MAX_E; E += blockDim.x / 32) {
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
        const bool wf16 = f16 && E + 1 <= kF16MaxK;
        const int w = wf16 ? RB / 2 : RB / 4;
        const int nt = (cnt[E] + w - 1) / w;
        for (int c = lane; c < nt; c += 32) {
            const int t = tstart[E] + c;
            if (t < n_tiles_max)
                meta[t] = TileMeta{E, start[E] + c * w, min(w, cnt[E] - c * w), wf16 ? kTileF16 : 0};
        }
    }
    for (int t = total_tiles + threadIdx.x; t < n_tiles_max; t += blockDim.x)
        meta[t] = TileMeta{0, 0, 0, 0};
}

namespace {

struct SetPtrs {
    int32_t *pi;
    float2 *omom;
    TileMeta *meta;
    uint32_t *sel;
    unsigned char *tiles;
    uint8_t *tables;
};

SetPtrs set_ptrs(const BatchLayout &B, int d, unsigned char *ws, int64_t N)
{
    const SetPlan &s = B.sets[(size_t)d];
    unsigned char *m = ws + s.meta_area;
    SetPtrs P;
    P.sel = (uint32_t *)m;
    P.pi = (int32_t *)(m + 256);
    P.omom = (float2 *)(m + 256 + al256((size_t)N * 4));
    P.meta = (TileMeta *)(m + 256 + al256((size_t)N * 4) + al256((size_t)N * sizeof(float2)));
    P.tiles = ws + B.br[(size_t)s.branch].tiles;
    P.tables = ws + B.br[(size_t)s.branch].tables;
    return P;
}

// Phase 1, plan and target staging of one dataset.
cudaError_t enqueue_front(const edm_dataset &d, const SetPlan &sp, const SetPtrs &P, const edm_params *p,
                          cudaStream_t st)
{
    cudaError_t e;
    const int T = (int)d.T;
    if ((e = launch_simplex(d.Y, d.N, T, d.ldY, p->E_max, p->tau, p->Tp, d.optE, nullptr, st)) != cudaSuccess)
        return e;
    const bool f16 = p->precision == EDM_PRECISION_FP16_TARGETS;
    batch_plan_kernel<<<1, 1024, 0, st>>>(d.optE, (int)d.N, f16 ? 1 : 0, sp.RB, sp.n_tiles_max, P.pi, P.meta, P.sel);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    if ((e = launch_prep_targets(d.Y, d.ldY, T, p->tau, p->Tp, P.pi, P.meta, sp.n_tiles_max, (float *)P.tiles, P.omom,
                                 st, sp.RB)) != cudaSuccess)
        return e;
    if (f16)
        e = launch_prep_targets_f16(d.Y, d.ldY, T, p->tau, p->Tp, P.pi, P.meta, sp.n_tiles_max, P.tiles, P.omom, st,
                                    sp.RB);
    return e;
}

cudaError_t enqueue_knn(const edm_dataset &d, const SetPtrs &P, const edm_params *p, int q_per_cta, cudaStream_t st)
{
    // the E in use are known on the device only: the warp kernel serves them
    // all in one sweep
    return launch_knn_tables(d.Y, d.ldY, 0, (int)d.N, (int)d.T, p->tau, p->Tp, p->exclusion_radius,
                             (1u << p->E_max) - 1u, all_e_layout(d.T, p), P.tables, st, q_per_cta, P.sel);
}

cudaError_t enqueue_lookup(const edm_dataset &d, const SetPlan &sp, const SetPtrs &P, const edm_params *p,
                           int parts_factor, int sms, cudaStream_t st)
{
    LookupArgs a;
    a.tiles = (const float *)P.tiles;
    a.meta = P.meta;
    a.pi = P.pi;
    a.omom = P.omom;
    a.tables = P.tables;
    a.lay = all_e_layout(d.T, p);
    a.T = (int)d.T;
    a.tau = p->tau;
    a.Tp = p->Tp;
    a.s_lo = 0;
    a.lag = p->Tp;
    a.tile_begin = 0;
    a.n_tiles = sp.n_tiles_max;
    a.n_lib = (int)d.N;
    // the real tile count is about N / (RB/4) (or half that in FP16)
    const int real_tiles = std::max(1, (int)((d.N + sp.RB / 4 - 1) / (sp.RB / 4)));
    const int parts = (parts_factor * sms + real_tiles - 1) / real_tiles;
    a.lib_parts = std::max(1, std::min(parts, (int)((d.N + 7) / 8)));
    a.rho_col0 = 0;
    a.rho = d.rho;
    a.ld_rho = d.ld_rho;
    return launch_lookup_multi(a, sp.RB, st);
}

cudaError_t enqueue_set(const edm_dataset &d, const SetPlan &sp, const SetPtrs &P, const edm_params *p,
                        const Tune &tn, int sms, cudaStream_t st)
{
    cudaError_t e;
    if ((e = enqueue_front(d, sp, P, p, st)) != cudaSuccess)
        return e;
    if ((e = enqueue_knn(d, P, p, tn.q_per_cta, st)) != cudaSuccess)
        return e;
    return enqueue_lookup(d, sp, P, p, tn.parts_factor, sms, st);
}

// Best of two timed runs of `fn` on `st` (ms), or 1e30 on error.
template <class Fn>
float time_best(Fn fn, cudaStream_t st)
{
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess)
        return 1e30f;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return 1e30f;
    }
    float best = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(a, st);
        cudaError_t e = fn();
        cudaEventRecord(b, st);
        if (cudaEventSynchronize(b) != cudaSuccess || e != cudaSuccess) {
            best = 1e30f;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        best = std::min(best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

// Measure the tile shapes of every class not yet in the cache on the
// class's largest dataset.
cudaError_t autotune(const edm_dataset *sets, int n, const BatchLayout &B, unsigned char *ws, const edm_params *p,
                     int sms, cudaStream_t st)
{
    static const int qs[] = {32, 64, 128};
    static const int fs[] = {2, 4, 8};
    for (int d = 0; d < n; ++d) {
        const int cls = tune_class(sets[d], p->precision);
        Tune have;
        if (tune_find(cls, have))
            continue;
        int rep = d;
        for (int k = d + 1; k < n; ++k)
            if (tune_class(sets[k], p->precision) == cls && sets[k].N > sets[rep].N)
                rep = k;
        const edm_dataset &ds = sets[rep];
        const SetPlan &sp = B.sets[(size_t)rep];
        const SetPtrs P = set_ptrs(B, rep, ws, ds.N);
        cudaError_t e = enqueue_front(ds, sp, P, p, st);
        if (e != cudaSuccess)
            return e;
        Tune best{64, 4};
        float best_ms = 1e30f;
        for (int q : qs) {
            float ms = time_best([&] { return enqueue_knn(ds, P, p, q, st); }, st);
            if (ms < best_ms) {
                best_ms = ms;
                best.q_per_cta = q;
            }
        }
        if ((e = enqueue_knn(ds, P, p, best.q_per_cta, st)) != cudaSuccess)
            return e;
        best_ms = 1e30f;
        for (int f : fs) {
            float ms = time_best([&] { return enqueue_lookup(ds, sp, P, p, f, sms, st); }, st);
            if (ms < best_ms) {
                best_ms = ms;
                best.parts_factor = f;
            }
        }
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
            return e;
        g_tune.push_back(TuneEntry{cls, best});
    }
    return cudaGetLastError();
}

int check_batch(const edm_dataset *sets, int n, const edm_params *p)
{
    if (!sets || n < 1 || !p)
        return EDM_ERR_INVALID;
    if (p->tau < 1 || p->Tp < 0 || p->exclusion_radius < -1 || p->E_max < 1)
        return EDM_ERR_INVALID;
    if (p->precision != EDM_PRECISION_FP32 && p->precision != EDM_PRECISION_FP16_TARGETS)
        return EDM_ERR_INVALID;
    if (p->flags & EDM_FLAG_LOOKUP_SCALAR)
        return EDM_ERR_UNSUPPORTED;
    if (p->E_max > EDM_MAX_E)
        return EDM_ERR_UNSUPPORTED;
    for (int d = 0; d < n; ++d) {
        const edm_dataset &s = sets[d];
        if (!s.Y || !s.optE || !s.rho || s.N < 1 || s.T < 4 || s.ldY < s.T || s.ld_rho < s.N)
            return EDM_ERR_INVALID;
        if (s.T > EDM_MAX_T || s.N > 65535 || s.T > knn_max_T() || chunked_row_bytes((int)s.T) == 0)
            return EDM_ERR_UNSUPPORTED;
        const int64_t h = s.T / 2, span = (int64_t)(p->E_max - 1) * p->tau;
        if (h - p->Tp - span < p->E_max + 1 || (s.T - h) - p->Tp - span < 2)
            return EDM_ERR_INVALID;
        // phase 2 at the largest E phase 1 may pick
        int64_t cand = s.T - p->Tp - span;
        if (p->exclusion_radius >= 0)
            cand -= 2 * (int64_t)p->exclusion_radius + 1;
        if (cand < p->E_max + 1)
            return EDM_ERR_INVALID;
    }
    return EDM_OK;
}

cudaError_t capture(const edm_dataset *sets, int n, const BatchLayout &B, unsigned char *ws, const edm_params *p,
                    int sms, cudaStream_t origin, cudaGraphExec_t *exec)
{
    const int nb = (int)B.br.size();
    cudaStream_t bs[kBranches] = {};
    cudaEvent_t fork = nullptr, join[kBranches] = {};
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int b = 0; b < nb && e == cudaSuccess; ++b) {
        e = cudaStreamCreateWithFlags(&bs[b], cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&join[b], cudaEventDisableTiming);
    }
    cudaGraph_t graph = nullptr;
    if (e == cudaSuccess)
        e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t ce = cudaEventRecord(fork, origin);
        for (int b = 0; b < nb && ce == cudaSuccess; ++b)
            ce = cudaStreamWaitEvent(bs[b], fork, 0);
        for (int d = 0; d < n && ce == cudaSuccess; ++d) {
            const SetPlan &sp = B.sets[(size_t)d];
            Tune tn{64, 4};
            tune_find(tune_class(sets[d], p->precision), tn);
            ce = enqueue_set(sets[d], sp, set_ptrs(B, d, ws, sets[d].N), p, tn, sms, bs[sp.branch]);
        }
        for (int b = 0; b < nb && ce == cudaSuccess; ++b) {
            ce = cudaEventRecord(join[b], bs[b]);
            if (ce == cudaSuccess)
                ce = cudaStreamWaitEvent(origin, join[b], 0);
        }
        e = cudaStreamEndCapture(origin, &graph);
        if (ce != cudaSuccess)
            e = ce;
    }
    if (e == cudaSuccess)
        e = cudaGraphInstantiate(exec, graph, 0);
    if (graph)
        cudaGraphDestroy(graph);
    for (int b = 0; b < nb; ++b) {
        if (join[b])
            cudaEventDestroy(join[b]);
        if (bs[b])
            cudaStreamDestroy(bs[b]);
    }
    if (fork)
        cudaEventDestroy(fork);
    return e;
}

int replay(GraphEntry &g, cudaStream_t st)
{
    cudaEvent_t a = nullptr, b = nullptr;
    const bool prof = profiling();
    if (prof) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, st);
    }
    const cudaError_t e = cudaGraphLaunch(g.exec, st);
    if (prof) {
        cudaEventRecord(b, st);
        prof_push(EDM_KERNEL_BATCH, a, b, g.pairs);
    }
    if (e != cudaSuccess)
        return EDM_ERR_CUDA;
    for (int k = 0; k < EDM_KERNEL_COUNT; ++k)
        note_launches(k, g.launches[k]);
    return EDM_OK;
}

}  // namespace

}  // namespace edm

extern "C" {

size_t edm_ccm_rho_batched_workspace_bytes(const edm_dataset *sets, int32_t n_sets, const edm_params *params)
{
    if (edm::check_batch(sets, n_sets, params) != EDM_OK)
        return 0;
    return edm::batch_layout(sets, n_sets, params).total;
}

int edm_ccm_rho_batched(const edm_dataset *sets, int32_t n_sets, const edm_params *params, void *ws, size_t ws_bytes,
                        void *stream)
{
    using namespace edm;
    int rc = check_batch(sets, n_sets, params);
    if (rc)
        return rc;
    if (!ws)
        return EDM_ERR_INVALID;
    const BatchLayout B = batch_layout(sets, n_sets, params);
    if (ws_bytes < B.total)
        return EDM_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return EDM_ERR_CUDA;

    std::lock_guard<std::mutex> lock(g_mu);
    for (GraphEntry &g : g_graphs)
        if (same_call(g, sets, n_sets, params, ws, ws_bytes, dev))
            return replay(g, st);

    // First call: tune on a private stream ordered after `stream`'s work,
    // then capture on it.
    unsigned char *w = (unsigned char *)ws;
    const int sms = sm_count_dev();
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
        return EDM_ERR_CUDA;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess)
        e = autotune(sets, n_sets, B, w, params, sms, cs);
    GraphEntry g;
    g.exec = nullptr;
    if (e == cudaSuccess)
        e = capture(sets, n_sets, B, w, params, sms, cs, &g.exec);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess)
        return EDM_ERR_CUDA;
    g.sets.assign(sets, sets + n_sets);
    g.params = *params;
    g.ws = ws;
    g.ws_bytes = ws_bytes;
    g.device = dev;
    g.pairs = 0.0;
    for (int k = 0; k < EDM_KERNEL_COUNT; ++k)
        g.launches[k] = 0;
    const bool f16 = params->precision == EDM_PRECISION_FP16_TARGETS;
    for (int d = 0; d < n_sets; ++d) {
        g.launches[EDM_KERNEL_SIMPLEX] += 1;
        g.launches[EDM_KERNEL_PLAN] += 1;
        g.launches[EDM_KERNEL_PREP] += f16 ? 2 : 1;
        g.launches[EDM_KERNEL_KNN] += 1;
        g.launches[EDM_KERNEL_LOOKUP] += 1;
        g.pairs += (double)sets[d].N * (double)sets[d].N;
    }
    if ((int)g_graphs.size() >= kGraphCache) {
        cudaGraphExecDestroy(g_graphs.front().exec);
        g_graphs.erase(g_graphs.begin());
    }
    g_graphs.push_back(g);
    return replay(g_graphs.back(), st);
}

int edm_ccm_rho_batched_reset(void)
{
    using namespace edm;
    std::lock_guard<std::mutex> lock(g_mu);
    if (cudaDeviceSynchronize() != cudaSuccess)
        return EDM_ERR_CUDA;
    for (GraphEntry &g : g_graphs)
        cudaGraphExecDestroy(g.exec);
    g_graphs.clear();
    g_tune.clear();
    return EDM_OK;
}

}  // extern "C"
