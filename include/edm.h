/*
 * edm.h -- C ABI of the GB300 (sm_103a) all-pairs Convergent Cross Mapping
 * library (the data-parallel hot path of mpEDM, arXiv 2011.11082).
 *
 * The paper states the problem as: input N time series of length L, the
 * maximum embedding dimension E_max and the lag tau; output the optimal
 * embedding dimension of every series and the N x N causal map rho
 * (Sec. III-A, Algorithm 1 and Algorithm 2).  The entry points below follow
 * that statement.
 *
 * Conventions for every entry point
 *   - Pointers named Y, x, optE, rho, idx, w, grad_* and ws are DEVICE
 *     pointers owned by the caller; the library never frees them.  Pointers
 *     to edm_params and to host arrays are read during the call only.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; unless stated otherwise a call does
 *     not synchronise and returns before the GPU finishes.
 *   - Series are float32, series-major: series i occupies Y[i*ldY .. i*ldY+T).
 *   - Return value: EDM_OK (0) or an EDM_ERR_* code.  EDM_ERR_CUDA keeps the
 *     CUDA error for edm_status_string() and edm_last_cuda_error().
 *   - Non-finite input values are the caller's responsibility (results are
 *     then undefined but every memory access stays in bounds).
 *   - There is no CPU fallback: without a usable sm_103a device every
 *     compute entry point returns EDM_ERR_CUDA.
 */
#ifndef EDM_H
#define EDM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EDM_OK 0
#define EDM_ERR_INVALID 1     /* bad argument: null pointer, size, or T too short */
#define EDM_ERR_CUDA 2        /* a CUDA call failed (see edm_last_cuda_error) */
#define EDM_ERR_WORKSPACE 3   /* ws too small; see the matching *_workspace_bytes */
#define EDM_ERR_TIMEOUT 4     /* a bounded device wait gave up */
#define EDM_ERR_UNSUPPORTED 5 /* valid request outside this library's limits */

/* Largest embedding dimension the kernels are built for. */
#define EDM_MAX_E 20
/* Upper bound on the series length (indices are kept in 16 bits).  The kNN
   kernels stage a whole series in shared memory, which lowers the practical
   limit to about 46,000 steps: longer series return EDM_ERR_UNSUPPORTED. */
#define EDM_MAX_T 65535

#define EDM_PRECISION_FP32 0         /* targets staged as float32 */
#define EDM_PRECISION_FP16_TARGETS 1 /* targets staged as float16 (for E <= 11; larger
                                        E stay float32); the FP32 table weights enter
                                        each FMA as float16 copies; exact products,
                                        FP32 accumulation.  Series longer than about
                                        3,100 steps (target tiles read from L2, not
                                        shared memory) always stage float32 */

/* flags */
#define EDM_FLAG_NONE 0u
/* phase 2: use the scalar-gather lookup kernels instead of the 16-byte
   chunked ones (FP32 targets only; kept for comparison) */
#define EDM_FLAG_LOOKUP_SCALAR 1u
/* edm_optimal_E / edm_ccm_rho: first scan Y for non-finite values; if a
   series holds one, return EDM_ERR_INVALID without computing and keep its
   index for edm_last_bad_series().  The scan synchronises `stream`. */
#define EDM_FLAG_VALIDATE 2u
/* kNN tables: always use the warp-per-query kernel (by default a table set
   of one E <= 6 at tau = 1 uses the thread-per-query kernel; same
   neighbours, weights equal up to the summation order) */
#define EDM_FLAG_KNN_WARP 4u

typedef struct edm_params {
    int32_t E_max;            /* phase 1 searches E = 1..E_max (<= EDM_MAX_E) */
    int32_t tau;              /* lag between embedding coordinates, >= 1 */
    int32_t Tp;               /* prediction horizon, >= 0 (1 = one step ahead) */
    int32_t exclusion_radius; /* phase 2: a query skips candidates with |s-t| <= r;
                                 0 = itself only, -1 = keep itself */
    int32_t precision;        /* EDM_PRECISION_* (phase 2 target staging) */
    uint32_t flags;           /* EDM_FLAG_* */
} edm_params;

/*
 * Phase 1, simplex projection (Algorithm 1, its simplex phase; Sec. II-B).
 * For every series i: library = first floor(T/2) samples, target = the rest,
 * both embedded within themselves with lags (0, tau, .., (E-1)tau) counted
 * backwards; each target point's E+1 nearest library points (ascending
 * distance, ties to the smaller index) give the forecast
 * sum_n w_n lib(s_n+Tp), w = exp(-d/d_1)/sum; rho_E = Pearson(observed,
 * forecast); optE[i] = argmax_E rho_E (NaN never wins, ties -> smaller E,
 * all-NaN -> 1).
 *   Y         [N][ldY] float32, ldY >= T
 *   optE      [N] int32 out
 *   rho_by_E  [N][E_max] float32 out, or NULL
 * Requires floor(T/2) - Tp - (E_max-1)*tau >= E_max + 1 and
 * T - floor(T/2) - Tp - (E_max-1)*tau >= 2, else EDM_ERR_INVALID.
 */
int edm_optimal_E(const float *Y, int64_t N, int64_t T, int64_t ldY, const edm_params *params,
                  int32_t *optE, float *rho_by_E, void *stream);

/*
 * Phase 2 kNN tables (Algorithm 2, its kNN step; Algorithms 3/4; the table
 * reuse of Sec. III-B).  For each of n_lib library series and one E: every
 * embedded point t in [(E-1)tau, T-1-Tp] (row r = t-(E-1)tau) gets its E+1
 * nearest embedded points s of the same series in the same range
 * (skipping |s-t| <= exclusion_radius), ascending (d^2, s), and the
 * normalised weights exp(-d/d_1)/sum.  Neighbour order is exact with
 * respect to float64 distances of the float32 inputs.
 *   Y     [n_lib][ldY] float32
 *   idx   [n_lib][Tq][E+1] int32 out: neighbour times s (not shifted by Tp)
 *   w     [n_lib][Tq][E+1] float32 out
 *   Tq    must equal T - Tp - (E-1)*tau
 */
int edm_knn_table(const float *Y, int64_t n_lib, int64_t T, int64_t ldY, int32_t E,
                  const edm_params *params, int32_t *idx, float *w, int64_t Tq, void *stream);

/*
 * Phase 2 cross map (Algorithm 2, its lookup and corrcoef steps; Algorithm 5).
 * For libraries i in [lib_begin, lib_begin+lib_count) and every target j:
 * prediction p(t) = sum_n w[t,n] y_j(s_n+Tp) with library i's table at
 * E = optE[j], observation o(t) = y_j(t+Tp), rho(i,j) = Pearson(o, p).
 *   Y      [N][ldY] float32
 *   optE   [N] int32 (device), each in 1..EDM_MAX_E
 *   rho    TARGET-MAJOR output: rho[j*ld_rho + (i - lib_begin)] = rho(i, j)
 *          for every target j in 0..N-1; ld_rho >= lib_count.  (The
 *          library-major causal map of the paper is the transpose view.)
 *   ws     device workspace of at least edm_ccm_workspace_bytes(N, T, params)
 * The grouping of targets by E is planned on the device, so the call does
 * not synchronise and never reads optE back: launches are sized for the
 * worst case and surplus blocks return at once.  A target whose optE is
 * outside 1..EDM_MAX_E gets NaN in every column of its row.  Three cases
 * plan on the host instead and synchronise `stream` once: EDM_FLAG_VALIDATE
 * (optE is checked there; a bad value returns EDM_ERR_INVALID),
 * EDM_FLAG_LOOKUP_SCALAR, and series too short for E = EDM_MAX_E (fewer
 * than E+1 candidates beyond the exclusion window; a target of such an E
 * returns EDM_ERR_INVALID).
 * Targets are staged in tiles of 32 (64 FP16) series; up to about 3,100
 * steps a tile sits in shared memory during the lookup, longer series (the
 * time-step sweep of the paper's Sec. IV reaches 40,000) read their tiles
 * from global memory / L2 with the same results up to summation order.
 */
int edm_ccm_rho(const float *Y, int64_t N, int64_t T, int64_t ldY, const int32_t *optE,
                int64_t lib_begin, int64_t lib_count, const edm_params *params,
                float *rho, int64_t ld_rho, void *ws, size_t ws_bytes, void *stream);

/* Workspace edm_ccm_rho needs for N series of length T (bytes). */
size_t edm_ccm_workspace_bytes(int64_t N, int64_t T, const edm_params *params);

/*
 * Time-delay cross mapping (the lagged cross-map skill the paper's adjacency
 * maps come from, Sec. II-A; not defined there): for every lag l in
 * lag_min..lag_max, rho_l(i, j) = corrcoef(y_j(t + l), sum_n w[t,n]
 * y_j(s_n + l)) from ONE kNN table per library and E (E = optE[j]), built
 * over the points whose every lag stays inside the series: queries =
 * candidates = t in [max((E-1)tau, -lag_min), T-1-max(lag_max, 0)].  A single
 * lag l = Tp >= 0 gives exactly edm_ccm_rho with horizon Tp.  params->Tp is
 * ignored; all N libraries.
 *   rho   [n_lags][N][ld_rho] target-major per lag:
 *         rho[(l - lag_min) * N * ld_rho + j * ld_rho + i] = rho_l(i -> j)
 *   ws    edm_ccm_rho_lags_workspace_bytes(N, T, lag_min, lag_max, params)
 * Planned on the device like edm_ccm_rho (no synchronisation; an optE
 * outside 1..EDM_MAX_E gives NaN rows in every lag).  When the lag window
 * is too short for E = EDM_MAX_E, or with EDM_FLAG_VALIDATE, the call plans
 * on the host (one synchronisation) and every E in optE must keep E+1
 * candidates in its window, else EDM_ERR_INVALID.
 */
int edm_ccm_rho_lags(const float *Y, int64_t N, int64_t T, int64_t ldY, const int32_t *optE, int32_t lag_min,
                     int32_t lag_max, const edm_params *params, float *rho, int64_t ld_rho, void *ws,
                     size_t ws_bytes, void *stream);
size_t edm_ccm_rho_lags_workspace_bytes(int64_t N, int64_t T, int32_t lag_min, int32_t lag_max,
                                        const edm_params *params);

/*
 * CCM convergence (the library-size test of the original CCM that the paper
 * leaves out, Sec. III-A): the cross map of every library (as edm_ccm_rho
 * with all N libraries) with each library's candidate points restricted to
 * a subset, for n_sub subsets; queries are every embedded point.  The
 * subsets are inputs (draw them with any seeded generator): subset u allows
 * candidate time s when bit s of masks[u * words + s / 32] is set.
 * Averaging rho over subsets of equal size L gives the convergence curve
 * rho(L).  With every bit set the result is edm_ccm_rho's.
 *   masks  DEVICE uint32 [n_sub][words], words >= ceil(T / 32)
 *   rho    [n_sub][N][ld_rho] target-major per subset
 *   ws     edm_ccm_workspace_bytes(N, T, params)
 * Each subset must leave E+1 candidates (beyond the exclusion window) for
 * the largest E in optE.  Planned on the device (no synchronisation): a
 * subset that does not gets NaN in its whole plane.  With EDM_FLAG_VALIDATE
 * (or series too short for E = EDM_MAX_E) the call plans on the host,
 * synchronising once, and such a subset returns EDM_ERR_INVALID.
 */
int edm_ccm_rho_subsets(const float *Y, int64_t N, int64_t T, int64_t ldY, const int32_t *optE,
                        const uint32_t *masks, int32_t n_sub, int64_t words, const edm_params *params, float *rho,
                        int64_t ld_rho, void *ws, size_t ws_bytes, void *stream);

/*
 * Both phases end to end with HOST buffers (the problem as the paper states
 * it: series in, optimal E and the causal map out).  Copies Y to the device,
 * runs phase 1, reads optE back, then phase 2 in blocks of `block` libraries
 * whose target-major results stream back on a second stream while the next
 * block computes.  Returns after everything has landed in host memory.
 *   Y_host     [N][T] float32 (pinned memory gives full copy bandwidth)
 *   optE_host  [N] int32 out
 *   rho_host   [N][ld_rho] float32 out, target-major like edm_ccm_rho:
 *              rho_host[j*ld_rho + i] = rho(library i -> target j); ld_rho >= N
 *   block      libraries per block (<= 0: about 1 GiB of results per block)
 *   ws         DEVICE workspace of edm_ccm_host_workspace_bytes(N, T, block, params)
 */
int edm_ccm_host(const float *Y_host, int64_t N, int64_t T, const edm_params *params, int32_t *optE_host,
                 float *rho_host, int64_t ld_rho, int64_t block, void *ws, size_t ws_bytes, void *stream);
size_t edm_ccm_host_workspace_bytes(int64_t N, int64_t T, int64_t block, const edm_params *params);

/*
 * Batched form (not in the paper; the paper runs one dataset per job): many
 * independent datasets of uneven N and T, each through both phases --
 * optimal E (as edm_optimal_E) and its full causal map (as edm_ccm_rho with
 * all N libraries) -- in ONE CUDA-graph launch.
 *   sets      HOST array of n_sets descriptors (read during the call):
 *               Y     [N][ldY] float32 device series of that dataset
 *               optE  [N] int32 device out
 *               rho   [N][ld_rho] float32 device out, target-major like
 *                     edm_ccm_rho: rho[j*ld_rho + i] = rho(library i -> target j)
 *   ws        device workspace of edm_ccm_rho_batched_workspace_bytes(...)
 * Each dataset needs the edm_optimal_E length condition for params->E_max,
 * N <= 65535, and T short enough for a target tile to sit in shared memory
 * (about 3,100 steps; longer series return EDM_ERR_UNSUPPORTED); the E grouping of its
 * targets is planned on the device, so the call never synchronises with
 * the GPU after its first use.
 * First call with a given (sets, params, ws, ws_bytes): the library times
 * candidate tile shapes on the batch's own data (kNN query points per CTA,
 * lookup grid split; cached per series-length, size and precision class),
 * then captures every launch of the batch -- datasets spread over parallel
 * graph branches, each branch with its own workspace region -- into a CUDA
 * graph and keeps the instantiated graph (up to 8, oldest dropped first).
 * That first call synchronises `stream` and must not itself run inside a
 * stream capture.  Later calls with identical arguments replay the graph
 * with one cudaGraphLaunch on `stream`, asynchronously.  The cached graph
 * holds the pointers it was captured with: reuse it only while those
 * buffers stay allocated.
 * The results are those of the per-dataset calls (same kernels and tile
 * shapes within a dataset's tile).
 */
typedef struct edm_dataset {
    const float *Y;
    int64_t N, T, ldY;
    int32_t *optE;
    float *rho;
    int64_t ld_rho;
} edm_dataset;

int edm_ccm_rho_batched(const edm_dataset *sets, int32_t n_sets, const edm_params *params, void *ws,
                        size_t ws_bytes, void *stream);
size_t edm_ccm_rho_batched_workspace_bytes(const edm_dataset *sets, int32_t n_sets, const edm_params *params);
/* Drop every cached batched graph and tuning result (synchronises the device). */
int edm_ccm_rho_batched_reset(void);

/*
 * Adjoint of the cross map (not in the paper): given G = dL/d rho,
 * grad_Y = dL/dY for L = sum_ij G(i,j) rho(i,j), with every kNN index and
 * every optE held at the values the forward pass finds (the tables are
 * rebuilt exactly).  Through the target y_j: the prediction p(t) and the
 * observation y_j(t+Tp); through the library x_i: the weights
 * exp(-d/d_1)/sum and d = sqrt(sum of squared lag differences).  Where a
 * distance is 0 the gradient through it is 0.
 *   grad_rho  TARGET-MAJOR like rho: grad_rho[j*ld_g + i] = dL/d rho(i,j),
 *             ld_g >= N
 *   grad_Y    [N][ldY] float32, overwritten
 *   ws        at least edm_ccm_backward_workspace_bytes(N, T, params):
 *             16 bytes per (library, target) pair of statistics, plus the
 *             kNN tables of every E for min(N, the libraries that fit in
 *             1 GB) libraries at once (about 1.4 KB per library and time
 *             step), processed in blocks of that many libraries
 * Requires T - Tp <= 3072.  A pair with a zero-variance side (rho NaN in
 * the forward map) contributes no gradient.  The E grouping is planned on the device (no
 * synchronisation); a target whose optE is outside 1..EDM_MAX_E (or leaves
 * fewer than E+1 candidates) contributes no gradient.
 * Summation order of the shared-memory accumulations varies between runs
 * (atomic adds), so the last bits of grad_Y may differ run to run.
 */
int edm_ccm_rho_backward(const float *Y, int64_t N, int64_t T, int64_t ldY, const int32_t *optE,
                         const float *grad_rho, int64_t ld_g, const edm_params *params, float *grad_Y,
                         void *ws, size_t ws_bytes, void *stream);
size_t edm_ccm_backward_workspace_bytes(int64_t N, int64_t T, const edm_params *params);

/*
 * Allocation-free variant of edm_ccm_rho, for callers that cannot allocate
 * device memory while they run: real-time loops that must not touch an
 * allocator, and hosts that hand this library a stream but no memory pool
 * (plugins and embedded runtimes that own all device memory themselves).
 * The paper has no counterpart: this is a deployment form of the same
 * cross map.  Inputs, outputs and results are those of edm_ccm_rho (with
 * params->flags limited to EDM_FLAG_KNN_WARP; any other flag returns
 * EDM_ERR_UNSUPPORTED); the scratch lives in one statically allocated
 * 64 MiB device array instead of a caller workspace, and the plan is built
 * on the device, so the call makes no cudaMalloc/cudaFree, no allocating
 * library call and no host heap allocation.
 *   - Problems whose scratch exceeds the array (target tiles of about
 *     N*T*4 bytes plus the kNN tables of at least one library) return
 *     EDM_ERR_WORKSPACE before touching the device; e.g. N = 2,048 and
 *     T = 1,500 fit, N = 16,384 and T = 1,500 do not.  Series longer than
 *     a shared-memory target tile allows (about 3,100 steps) return
 *     EDM_ERR_UNSUPPORTED.  An optE value outside 1..EDM_MAX_E returns
 *     EDM_ERR_INVALID.
 *   - The first call on each device resolves the array's device address
 *     (cudaGetSymbolAddress, that device current) and keeps it; make that
 *     first call before any stream capture.  A device reset after it is not
 *     supported.
 *   - Every GPU that loads the library holds the array until the process
 *     exits.  All calls share it and it keeps the previous call's contents;
 *     calls whose GPU work overlaps (other streams, other host threads)
 *     race on it.
 *   - It synchronises `stream` once (reading 84 bytes of per-E counts back
 *     to the host).
 */
int edm_ccm_rho_noalloc(const float *Y, int64_t N, int64_t T, int64_t ldY, const int32_t *optE,
                        int64_t lib_begin, int64_t lib_count, const edm_params *params,
                        float *rho, int64_t ld_rho, void *stream);

/* Series index found by the last EDM_FLAG_VALIDATE scan on this thread
   that failed (first series holding a non-finite value), else -1. */
int64_t edm_last_bad_series(void);

/*
 * Rare-path accounting of the kNN kernels on the current device (the
 * certified FP32 ranking of Sec. III-B's tables falls back to FP64 where a
 * gap between neighbour distances is within the FP32 error bound):
 *   reranks     queries whose kept entries were re-ranked in FP64
 *   exhaustive  queries re-solved by an exhaustive FP64 scan
 * Counts accumulate over every kNN launch since the last reset (reset != 0
 * clears them after reading).  Synchronises the device.
 */
int edm_knn_counters(int64_t *reranks, int64_t *exhaustive, int reset);

/*
 * Bounded device waits that gave up on the current device since load (or
 * the last reset != 0): the kNN and lookup kernels stage their series and
 * target tiles in shared memory with bulk copies completed on an mbarrier,
 * and poll it a bounded number of times.  A wait that gives up makes its
 * CTA skip its work (its outputs are left unwritten) and counts here, so a
 * healthy run reads 0.  (The adjoint's library pass, which double-buffers
 * target series the same way, loads a late series with plain loads instead
 * and counts here too.)  Synchronises the device.
 */
int edm_wait_timeouts(int64_t *count, int reset);

/* Human-readable text for a status code (includes the CUDA error if any). */
const char *edm_status_string(int status);

/* The CUDA error behind the last EDM_ERR_CUDA on this thread (0 if none). */
int edm_last_cuda_error(void);

/* Library version, e.g. 0x000100 = 0.1.0. */
int edm_version(void);

/*
 * Launch accounting and kernel timing (instrumentation, not part of the
 * method).  Kernel ids: */
#define EDM_KERNEL_SIMPLEX 0 /* phase 1 simplex projection */
#define EDM_KERNEL_KNN 1     /* phase 2 kNN tables */
#define EDM_KERNEL_PREP 2    /* target staging */
#define EDM_KERNEL_LOOKUP 3  /* fused lookup + rho */
#define EDM_KERNEL_PLAN 4    /* device-side E grouping (batched form) */
#define EDM_KERNEL_BATCH 5   /* a whole batched graph (timed as one; units = pairs) */
#define EDM_KERNEL_COUNT 6
/*
 * edm_launch_count: launches of that kernel since load (always counted).
 * edm_profile_enable(1): from now on record a CUDA event pair on the
 *   launching stream around every launch (process-wide, not thread-safe).
 * edm_profile_read: synchronise the recorded events and return, per kernel,
 *   the summed device time (ms), the launches timed and the work units
 *   they processed (pairs for LOOKUP, series for SIMPLEX, library tables
 *   for KNN, targets for PREP); then forget them.
 */
int64_t edm_launch_count(int kernel);
int edm_profile_enable(int on);
int edm_profile_read(int kernel, double *ms, int64_t *launches, double *units);

#ifdef __cplusplus
}
#endif

#endif /* EDM_H */
