// knn_kernels.cu -- phase 1 (simplex projection, optimal E) and phase 2 kNN
// tables on sm_103a.  Both stage one series in shared memory and run the
// warp-per-query kNN of knn_core.cuh (Algorithm 3's all-to-all distances
// computed on the fly, no materialised embedding).
#include "bulk_copy.cuh"
#include "knn_core.cuh"
#include "launchers.h"

namespace edm {

constexpr int kKnnWarps = 8;
constexpr int kKnnThreads = kKnnWarps * 32;

// The staged series is padded: `front` +inf values before it (reads of lags
// before the series start) and 32*J + 4 after it (the tail of the last
// candidate chunk).  front is a multiple of 4 floats.
static int front_pad(int E_hi, int tau) { return ((E_hi - 1) * tau + 3) & ~3; }

__host__ __device__ static size_t series_floats(int T, int front, int J) { return ((size_t)front + T + 32 * J + 4 + 3) & ~(size_t)3; }

// Shared memory: the padded series, then per warp a KnnWarpScratch, then
// per warp the distance scratch of 32 * J floats.
static size_t knn_smem_bytes_exact(int T, int front, int J)
{
    return series_floats(T, front, J) * sizeof(float) +
           (size_t)kKnnWarps * (sizeof(KnnWarpScratch) + knn_d2s_bytes(J)) + 64;
}

// Dynamic shared memory a kNN CTA may take (the simplex kernel also holds
// about 7 KB of static reductions; 227 KB is the per-CTA limit).
constexpr size_t kKnnSmemCap = 216 * 1024;

// Register slots per lane: the preferred J for the candidate count, lowered
// (more, shorter candidate chunks) while the staged series and the per-warp
// scratch would not fit kKnnSmemCap -- long series (T beyond about 30,000).
static int fit_J(int J, int T, int front)
{
    while (J > 8 && knn_smem_bytes_exact(T, front, J) > kKnnSmemCap)
        J = J == 48 ? 32 : J - 8;
    return J;
}

int knn_max_T()
{
    // J = 8, front for E = EDM_MAX_E at tau = 1
    const size_t fixed = (size_t)kKnnWarps * (sizeof(KnnWarpScratch) + knn_d2s_bytes(8)) + 64;
    const size_t floats = (kKnnSmemCap - fixed) / sizeof(float);
    return (int)(floats - (size_t)front_pad(EDM_MAX_E, 1) - 32 * 8 - 4 - 4);
}

// Distance scratch of warp w (behind the per-warp KnnWarpScratch array).
__device__ __forceinline__ float *warp_d2s(KnnWarpScratch *scratch, int J)
{
    return reinterpret_cast<float *>(scratch + kKnnWarps) + (size_t)warp_id() * 32 * J;
}

EDM_WAIT_TIMEOUT_READER(knn_wait_timeouts)

// ---------------------------------------------------------------------------
// Phase 1: simplex projection of every series over E = 1..E_max.
// ---------------------------------------------------------------------------
struct SimplexMoments {
    // Kahan-compensated running sums of (p-c), (p-c)^2, (p-c)(o-c), (o-c), (o-c)^2
    float s[5];
    float comp[5];
    __device__ void add(int i, float v)
    {
        float y = v - comp[i];
        float t = s[i] + y;
        comp[i] = (t - s[i]) - y;
        s[i] = t;
    }
};

struct SimplexEmit {
    static constexpr int kLaneMinK = 0;  // the grown list seeds every selection (measured faster here)
    const float *lib;  // library half (shared)
    const float *tgt;  // target half (shared)
    int Tp;
    int t;
    float shift;
    SimplexMoments mom;  // this lane's moments (lane = E-1)
    __device__ void operator()(int E, int k, int s, float w, bool act)
    {
        float contrib = act ? w * lib[s + Tp] : 0.f;
        float p = warp_sum(contrib);
        if (lane_id() == E - 1) {
            float pc = p - shift;
            float oc = tgt[t + Tp] - shift;
            mom.add(0, pc);
            mom.add(1, pc * pc);
            mom.add(2, pc * oc);
            mom.add(3, oc);
            mom.add(4, oc * oc);
        }
    }
};

template <int J>
__global__ void __launch_bounds__(kKnnThreads, 2) simplex_kernel(const float *__restrict__ Y, int64_t ldY, int T,
                                                                 int E_max, int tau, int Tp, int front,
                                                                 int32_t *__restrict__ optE,
                                                                 float *__restrict__ rho_by_E)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int total = (int)series_floats(T, front, J);
    float *x = reinterpret_cast<float *>(smem) + front;
    KnnWarpScratch *scratch = reinterpret_cast<KnnWarpScratch *>(smem + (size_t)total * sizeof(float));
    __shared__ double red[kKnnWarps][EDM_MAX_E][5];
    __shared__ double shift_sh;
    __shared__ double rho_sh[EDM_MAX_E];

    const int64_t i = blockIdx.x;
    // the series in shared memory with +inf padding (a lag that falls
    // outside the series makes the distance +inf)
    if (!stage_series_bulk(reinterpret_cast<float *>(smem), Y + i * ldY, T, front, total))
        return;

    // shift for the moments: the series mean (Pearson is shift invariant)
    if (threadIdx.x < 32) {
        double a = 0.0;
        for (int t = threadIdx.x; t < T; t += 32)
            a += (double)x[t];
        a = warp_sum_d(a);
        if (threadIdx.x == 0)
            shift_sh = a / (double)T;
    }
    __syncthreads();

    const int h = T / 2;
    const float *lib = x;
    const float *tgt = x + h;
    const int Tt = T - h;
    const int lane = lane_id(), warp = warp_id();
    KnnWarpScratch &sc = scratch[warp];

    SimplexEmit emit;
    emit.lib = lib;
    emit.tgt = tgt;
    emit.Tp = Tp;
    emit.t = 0;
    emit.shift = (float)shift_sh;
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        emit.mom.s[m] = 0.f;
        emit.mom.comp[m] = 0.f;
    }

    const int t_end = Tt - 1 - Tp;  // last query (E = 1)
    for (int t = warp; t <= t_end; t += kKnnWarps) {
        int E_lim = min(E_max, t / tau + 1);
        KnnQuery q;
        q.xq = tgt;
        q.xc = lib;
        q.t = t;
        q.s_first = 0;
        q.s_last = h - 1 - Tp;
        q.tau = tau;
        q.same = 0;
        q.excl = -1;
        q.E_lim = E_lim;
        q.sel = E_lim >= 32 ? 0xffffffffu : ((1u << E_lim) - 1u);
        q.mask = nullptr;
        q.d2s = warp_d2s(scratch, J);
        emit.t = t;
        knn_query<J>(q, sc, emit);
    }

    if (lane < E_max) {
#pragma unroll
        for (int m = 0; m < 5; ++m)
            red[warp][lane][m] = (double)emit.mom.s[m] - (double)emit.mom.comp[m];
    }
    __syncthreads();
    if (threadIdx.x < E_max) {
        const int e = threadIdx.x;
        double S[5] = {0, 0, 0, 0, 0};
        for (int w = 0; w < kKnnWarps; ++w)
            for (int m = 0; m < 5; ++m)
                S[m] += red[w][e][m];
        const int E = e + 1;
        double n = (double)(Tt - Tp - (E - 1) * tau);
        double cov = n * S[2] - S[0] * S[3];
        double vp = n * S[1] - S[0] * S[0];
        double vo = n * S[4] - S[3] * S[3];
        double r = (vp > 0.0 && vo > 0.0) ? cov / sqrt(vp * vo) : CUDART_NAN;
        rho_sh[e] = r;
        if (rho_by_E)
            rho_by_E[i * E_max + e] = (float)r;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int best = 1;
        double bv = 0.0;
        bool any = false;
        for (int e = 0; e < E_max; ++e) {
            double v = rho_sh[e];
            if (isnan(v))
                continue;
            if (!any || v > bv) {
                bv = v;
                best = e + 1;
                any = true;
            }
        }
        optE[i] = best;
    }
}

// ---------------------------------------------------------------------------
// Phase 2 tables.
// ---------------------------------------------------------------------------
struct EmitInternal {
    static constexpr int kLaneMinK = 12;  // lane-minimum bound first for K <= 12
    uint8_t *lib_base;
    const TableLayout *lay;
    int t, tau, Tp;
    __device__ void operator()(int E, int k, int s, float w, bool act)
    {
        if (!act)
            return;
        const int r = t - (E - 1) * tau;
        const int n = lane_id();
        float *wp = reinterpret_cast<float *>(lib_base + lay->off_w[E]);
        uint16_t *ip = reinterpret_cast<uint16_t *>(lib_base + lay->off_i[E]);
        wp[(size_t)n * lay->Tq_pad + r] = w;
        ip[(size_t)n * lay->Tq_pad + r] = (uint16_t)(s + Tp);
    }
};

struct EmitPublic {
    static constexpr int kLaneMinK = 12;
    int32_t *idx;
    float *w;
    int t, tau, k_fixed;
    __device__ void operator()(int E, int k, int s, float wv, bool act)
    {
        if (!act)
            return;
        const int r = t - (E - 1) * tau;
        const int n = lane_id();
        idx[(size_t)r * k + n] = s;
        w[(size_t)r * k + n] = wv;
    }
};

template <int J, bool kPublic>
__global__ void __launch_bounds__(kKnnThreads, 2)
    knn_tables_kernel(const float *__restrict__ Y, int64_t ldY, int64_t lib0, int T, int tau, int Tp, int excl,
                      uint32_t sel, int q_per_cta, int front, int s_lo, const __grid_constant__ TableLayout lay,
                      uint8_t *__restrict__ tables,
                      int32_t *__restrict__ pub_idx, float *__restrict__ pub_w, int pub_E,
                      const uint32_t *__restrict__ sel_dev, const uint32_t *__restrict__ cand_mask)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int total = (int)series_floats(T, front, J);
    float *x = reinterpret_cast<float *>(smem) + front;
    KnnWarpScratch *scratch = reinterpret_cast<KnnWarpScratch *>(smem + (size_t)total * sizeof(float));

    const int lib = blockIdx.y;
    if (sel_dev)
        sel &= *sel_dev;  // E set planned on the device
    if (!sel)
        return;
    if (!stage_series_bulk(reinterpret_cast<float *>(smem), Y + (lib0 + lib) * ldY, T, front, total))
        return;

    const int warp = warp_id();
    KnnWarpScratch &sc = scratch[warp];
    const int E_hi = 32 - __clz(sel);  // highest selected E
    int E_lo = __ffs(sel);             // lowest selected E
    // queries and candidates start at s_lo as well (0 for the plain cross map)
    const int t_first = max(max((int)blockIdx.x * q_per_cta, (E_lo - 1) * tau), s_lo);
    const int t_stop = min((int)(blockIdx.x + 1) * q_per_cta, T - Tp);

    EmitInternal ei{tables + (size_t)lib * lay.lib_stride, &lay, 0, tau, Tp};
    const int kp = pub_E + 1;
    const int Tq = T - Tp - (pub_E - 1) * tau;
    EmitPublic ep{pub_idx + (size_t)lib * Tq * kp, pub_w + (size_t)lib * Tq * kp, 0, tau, kp};

    for (int t = t_first + warp; t < t_stop; t += kKnnWarps) {
        int E_lim = min(E_hi, t / tau + 1);
        uint32_t s_t = sel & (E_lim >= 32 ? 0xffffffffu : ((1u << E_lim) - 1u));
        if (!s_t)
            continue;
        E_lim = 32 - __clz(s_t);
        KnnQuery q;
        q.xq = x;
        q.xc = x;
        q.t = t;
        q.s_first = s_lo;
        q.s_last = T - 1 - Tp;
        q.tau = tau;
        q.same = 1;
        q.excl = excl;
        q.E_lim = E_lim;
        q.sel = s_t;
        q.mask = cand_mask;
        q.d2s = warp_d2s(scratch, J);
        if (kPublic) {
            ep.t = t;
            knn_query<J>(q, sc, ep);
        } else {
            ei.t = t;
            knn_query<J>(q, sc, ei);
        }
    }
}

// ---------------------------------------------------------------------------
static int pick_J(int n_slots)
{
    int need = (n_slots + 31) / 32;
    if (need <= 8)
        return 8;
    if (need <= 16)
        return 16;
    if (need <= 24)
        return 24;
    if (need <= 32)
        return 32;
    return 48;
}

template <int J>
static cudaError_t simplex_J(const float *Y, int64_t N, int T, int64_t ldY, int E_max, int tau, int Tp, int32_t *optE,
                             float *rho_by_E, cudaStream_t st)
{
    const int front = front_pad(E_max, tau);
    size_t smem = knn_smem_bytes_exact(T, front, J);
    cudaError_t e = cudaFuncSetAttribute(simplex_kernel<J>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    for (int64_t b = 0; b < N; b += 0x7fffffff) {
        int64_t n = N - b < 0x7fffffff ? N - b : 0x7fffffff;
        simplex_kernel<J><<<(unsigned)n, kKnnThreads, smem, st>>>(Y + b * ldY, ldY, T, E_max, tau, Tp, front, optE + b,
                                                                   rho_by_E ? rho_by_E + b * E_max : nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_simplex(const float *Y, int64_t N, int T, int64_t ldY, int E_max, int tau, int Tp, int32_t *optE,
                           float *rho_by_E, cudaStream_t st)
{
    const int h = T / 2;
    switch (fit_J(pick_J(h - Tp), T, front_pad(E_max, tau))) {
    case 8: return simplex_J<8>(Y, N, T, ldY, E_max, tau, Tp, optE, rho_by_E, st);
    case 16: return simplex_J<16>(Y, N, T, ldY, E_max, tau, Tp, optE, rho_by_E, st);
    case 24: return simplex_J<24>(Y, N, T, ldY, E_max, tau, Tp, optE, rho_by_E, st);
    case 32: return simplex_J<32>(Y, N, T, ldY, E_max, tau, Tp, optE, rho_by_E, st);
    default: return simplex_J<48>(Y, N, T, ldY, E_max, tau, Tp, optE, rho_by_E, st);
    }
}

template <int J, bool kPublic>
static cudaError_t knn_J(const float *Y, int64_t ldY, int64_t lib0, int n_lib, int T, int tau, int Tp, int excl, int s_lo,
                         uint32_t sel, const TableLayout &lay, uint8_t *tables, int32_t *pidx, float *pw, int pE,
                         cudaStream_t st, int q_per_cta, const uint32_t *sel_dev, const uint32_t *cand_mask)
{
    const int E_hi = 32 - __builtin_clz(sel);
    const int front = front_pad(E_hi, tau);
    size_t smem = knn_smem_bytes_exact(T, front, J);
    cudaError_t e =
        cudaFuncSetAttribute(knn_tables_kernel<J, kPublic>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    dim3 grid((unsigned)((T - Tp + q_per_cta - 1) / q_per_cta), (unsigned)n_lib);
    knn_tables_kernel<J, kPublic><<<grid, kKnnThreads, smem, st>>>(Y, ldY, lib0, T, tau, Tp, excl, sel, q_per_cta,
                                                                    front, s_lo, lay, tables, pidx, pw, pE, sel_dev,
                                                                    cand_mask);
    return cudaGetLastError();
}

template <bool kPublic>
static cudaError_t knn_dispatch(const float *Y, int64_t ldY, int64_t lib0, int n_lib, int T, int tau, int Tp, int excl, int s_lo,
                                uint32_t sel, const TableLayout &lay, uint8_t *tables, int32_t *pidx, float *pw,
                                int pE, cudaStream_t st, int q = 64, const uint32_t *sel_dev = nullptr,
                                const uint32_t *cand_mask = nullptr)
{
    switch (fit_J(pick_J(T - Tp - s_lo), T, front_pad(32 - __builtin_clz(sel), tau))) {
    case 8: return knn_J<8, kPublic>(Y, ldY, lib0, n_lib, T, tau, Tp, excl, s_lo, sel, lay, tables, pidx, pw, pE, st, q, sel_dev, cand_mask);
    case 16: return knn_J<16, kPublic>(Y, ldY, lib0, n_lib, T, tau, Tp, excl, s_lo, sel, lay, tables, pidx, pw, pE, st, q, sel_dev, cand_mask);
    case 24: return knn_J<24, kPublic>(Y, ldY, lib0, n_lib, T, tau, Tp, excl, s_lo, sel, lay, tables, pidx, pw, pE, st, q, sel_dev, cand_mask);
    case 32: return knn_J<32, kPublic>(Y, ldY, lib0, n_lib, T, tau, Tp, excl, s_lo, sel, lay, tables, pidx, pw, pE, st, q, sel_dev, cand_mask);
    default: return knn_J<48, kPublic>(Y, ldY, lib0, n_lib, T, tau, Tp, excl, s_lo, sel, lay, tables, pidx, pw, pE, st, q, sel_dev, cand_mask);
    }
}

cudaError_t launch_knn_tables(const float *Y, int64_t ldY, int64_t lib0, int n_lib, int T, int tau, int Tp, int excl,
                              uint32_t sel, const TableLayout &lay, uint8_t *tables, cudaStream_t st, int q_per_cta,
                              const uint32_t *sel_dev, int s_lo, const uint32_t *cand_mask)
{
    return knn_dispatch<false>(Y, ldY, lib0, n_lib, T, tau, Tp, excl, s_lo, sel, lay, tables, nullptr, nullptr, 1, st,
                               q_per_cta, sel_dev, cand_mask);
}

// Which kernel builds the tables of the E set `sel`: the thread-per-query
// kernel for a single E <= knn_thread_max_E() at tau = 1, else the warp
// kernel.  (Splitting a multi-E set into per-E thread launches measured
// slower on the full step than the warp kernel's one shared sweep: 7.76 vs
// 7.10 s of kNN at N = 101,729, T = 1,500.)
static bool use_thread_kernel(int tau, uint32_t sel, bool force_warp)
{
    return !force_warp && tau == 1 && __builtin_popcount(sel) == 1 && 32 - __builtin_clz(sel) <= knn_thread_max_E();
}

cudaError_t launch_knn_tables_auto(const float *Y, int64_t ldY, int64_t lib0, int n_lib, int T, int tau, int Tp,
                                   int excl, uint32_t sel, const TableLayout &lay, uint8_t *tables, cudaStream_t st,
                                   bool force_warp, int s_lo, int *n_launches, const uint32_t *sel_dev)
{
    const bool thread = use_thread_kernel(tau, sel, force_warp);
    if (n_launches)
        *n_launches = thread ? __builtin_popcount(sel) : 1;
    if (!thread)
        return launch_knn_tables(Y, ldY, lib0, n_lib, T, tau, Tp, excl, sel, lay, tables, st, 64, sel_dev, s_lo);
    for (int E = 1; E <= 32 - __builtin_clz(sel); ++E) {
        if (!((sel >> (E - 1)) & 1u))
            continue;
        cudaError_t e = launch_knn_thread(Y, ldY, lib0, n_lib, T, Tp, excl, E, lay, tables, st, sel_dev, s_lo);
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

cudaError_t launch_knn_public(const float *Y, int64_t ldY, int n_lib, int T, int E, int tau, int Tp, int excl,
                              int32_t *idx, float *w, cudaStream_t st, bool force_warp)
{
    if (!force_warp && tau == 1 && E <= knn_thread_max_E())
        return launch_knn_thread_public(Y, ldY, n_lib, T, E, Tp, excl, idx, w, st);
    TableLayout lay{};
    return knn_dispatch<true>(Y, ldY, 0, n_lib, T, tau, Tp, excl, 0, 1u << (E - 1), lay, nullptr, idx, w, E, st);
}

cudaError_t knn_counters(unsigned long long out[2], bool reset)
{
    cudaError_t e = cudaMemcpyFromSymbol(out, g_knn_counts, sizeof(unsigned long long) * 2);
    if (e == cudaSuccess && reset) {
        const unsigned long long z[2] = {0ull, 0ull};
        e = cudaMemcpyToSymbol(g_knn_counts, z, sizeof z);
    }
    unsigned long long th[2] = {0ull, 0ull};
    if (e == cudaSuccess)
        e = knn_thread_counters(th, reset);
    out[0] += th[0];
    out[1] += th[1];
    return e;
}

}  // namespace edm
