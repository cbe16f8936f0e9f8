// launchers.h -- host-side launch helpers shared between the translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "edm.h"

namespace edm {

// Largest T the kNN kernels can stage in shared memory.
int knn_max_T();

// Phase 1: one CTA per series.  rho_by_E may be null.
cudaError_t launch_simplex(const float *Y, int64_t N, int T, int64_t ldY, int E_max, int tau, int Tp,
                           int32_t *optE, float *rho_by_E, cudaStream_t st);

// Internal table layout of one library block (consumed by the lookup).
struct TableLayout {
    int64_t lib_stride;             // bytes per library
    int64_t off_w[EDM_MAX_E + 1];   // byte offset of w[k][Tq_pad] per E (-1: absent)
    int64_t off_i[EDM_MAX_E + 1];   // byte offset of idx16[k][Tq_pad] per E
    int Tq_pad;                     // padded row count (multiple of 32)
};

// Phase 2 tables for n_lib libraries (series lib0 .. lib0+n_lib-1 of Y)
// for every E whose bit is set in sel, written in the internal layout.
// q_per_cta: query points per CTA; sel_dev (optional): device word ANDed
// into sel (E set planned on the device).
// s_lo: queries and candidates start at time s_lo (0 for the plain cross
// map; the time-delay form keeps every negative lag inside the series).
// cand_mask (optional, device): only candidates s with bit s of word s/32
// set (library subsets of the convergence test).
cudaError_t launch_knn_tables(const float *Y, int64_t ldY, int64_t lib0, int n_lib, int T, int tau, int Tp, int excl,
                              uint32_t sel, const TableLayout &lay, uint8_t *tables, cudaStream_t st,
                              int q_per_cta = 64, const uint32_t *sel_dev = nullptr, int s_lo = 0,
                              const uint32_t *cand_mask = nullptr);

// Thread-per-query tables for one E (tau = 1, E <= knn_thread_max_E() = 6),
// same results as the warp kernel (knn_thread.cu).
int knn_thread_max_E();
// sel_dev (optional): device E mask; the launch does nothing if bit E-1 is clear.
cudaError_t launch_knn_thread(const float *Y, int64_t ldY, int64_t lib0, int n_lib, int T, int Tp, int excl, int E,
                              const TableLayout &lay, uint8_t *tables, cudaStream_t st,
                              const uint32_t *sel_dev = nullptr, int s_lo = 0);
cudaError_t launch_knn_thread_public(const float *Y, int64_t ldY, int n_lib, int T, int E, int Tp, int excl,
                                     int32_t *idx, float *w, cudaStream_t st);
cudaError_t knn_thread_counters(unsigned long long out[2], bool reset);
// Tables for the E set `sel` with the cheaper kernel by a measured cost
// model: thread-per-query launches (one per E, all E <= knn_thread_max_E(),
// tau = 1) or one warp-kernel launch.  Returns the launches made in *n.
// sel_dev (optional): device E mask ANDed into sel.
cudaError_t launch_knn_tables_auto(const float *Y, int64_t ldY, int64_t lib0, int n_lib, int T, int tau, int Tp,
                                   int excl, uint32_t sel, const TableLayout &lay, uint8_t *tables, cudaStream_t st,
                                   bool force_warp = false, int s_lo = 0, int *n_launches = nullptr,
                                   const uint32_t *sel_dev = nullptr);

// FP64 re-rank / exhaustive-scan query counts of the kNN kernels on the
// current device (synchronises); reset clears them.
cudaError_t knn_counters(unsigned long long out[2], bool reset);

// Bounded bulk-copy waits that gave up, per translation unit (bulk_copy.cuh).
cudaError_t knn_wait_timeouts(unsigned long long *count, bool reset);
cudaError_t knn_thread_wait_timeouts(unsigned long long *count, bool reset);
cudaError_t lookup_multi128_wait_timeouts(unsigned long long *count, bool reset);
cudaError_t lookup_multi128_lag_wait_timeouts(unsigned long long *count, bool reset);
cudaError_t lookup_multi64_wait_timeouts(unsigned long long *count, bool reset);
cudaError_t lookup_multi64_lag_wait_timeouts(unsigned long long *count, bool reset);
cudaError_t backward_wait_timeouts(unsigned long long *count, bool reset);

// Public table format: idx int32 [n_lib][Tq][E+1] (unshifted), w float [n_lib][Tq][E+1].
cudaError_t launch_knn_public(const float *Y, int64_t ldY, int n_lib, int T, int E, int tau, int Tp, int excl,
                              int32_t *idx, float *w, cudaStream_t st, bool force_warp = false);

// Target tiles: one E each, time-major rows of 128 bytes (z-normalised):
// FP32 tiles hold 32 targets ([T][32] float); FP16 tiles (flag kTileF16)
// hold 64 ([T][32] half2, word w = targets w and w+32).
constexpr int kTileF16 = 1;
// FP16 tiles are used for E + 1 <= kF16MaxK; larger E stay FP32.
constexpr int kF16MaxK = 12;
struct TileMeta {
    int E;
    int first;  // first sorted position
    int count;  // targets in this tile (<= 32, or <= 64 for FP16)
    int flags;  // kTileF16
};

// RB: tile row bytes (128: 32 targets, 64: 16 targets per row)
cudaError_t launch_prep_targets(const float *Y, int64_t ldY, int T, int tau, int Tp, const int32_t *pi,
                                const TileMeta *meta, int n_tiles, float *tiles, float2 *omom, cudaStream_t st,
                                int RB = 128);

// Device-planned launch slot: a tile range and the E it contains.
struct SlotDesc {
    int tile_begin;
    int n_tiles;
    uint32_t sel;  // bit E-1: E present in the range
    int pad;
};

// Tiles per E: FP16 tiles hold 2x the targets of FP32 tiles (RB/2 vs RB/4).
__host__ __device__ inline int plan_tile_width(int E, int f16, int RB)
{
    return (f16 && E + 1 <= kF16MaxK) ? RB / 2 : RB / 4;
}

constexpr int kMaxPlanGroups = 8;

// Inputs of the device-side plan (ccm_plan.cu).
struct CcmPlanSpec {
    int N, T, tau, Tp, excl;
    int s_lo;             // first query/candidate time (time-delay form), else 0
    int f16, RB;          // FP16 tiles for E + 1 <= kF16MaxK when f16; tile row bytes
    int n_tiles_max;      // tile slots to fill (unused ones get E = 0)
    int n_groups;         // groups of E ranges, in tile order
    int g_lo[kMaxPlanGroups], g_hi[kMaxPlanGroups];
    int tiles_per_block;  // target-block cut of each group (0: none)
    int tb_max[kMaxPlanGroups];
    int slot0[kMaxPlanGroups];  // first slot of each group
    // NaN rows for targets whose E is unusable: rho + u*plane_stride +
    // j*ld_rho, row_len values, for u < planes (rho null: none)
    float *rho;
    int64_t ld_rho, row_len, plane_stride;
    int planes;
    int32_t *starts;  // optional: first sorted position of each E (E = 0..EDM_MAX_E+1)
};

// counts[0]: targets with an unusable E; counts[E]: targets of E;
// counts[EDM_MAX_E + 1]: tiles in use.  pi: target indices sorted by E.
cudaError_t launch_ccm_plan(const int32_t *optE, const CcmPlanSpec &sp, int32_t *counts, int32_t *pi, TileMeta *meta,
                            SlotDesc *slots, cudaStream_t st);
// NaN planes for convergence subsets that leave too few candidates.
cudaError_t launch_subset_check(const uint32_t *masks, int n_sub, int64_t words, const int32_t *counts, int N, int T,
                                int tau, int Tp, int excl, float *rho, int64_t ld_rho, int64_t plane_stride,
                                cudaStream_t st);

struct LookupArgs {
    const float *tiles;
    const TileMeta *meta;
    const int32_t *pi;
    const float2 *omom;
    const uint8_t *tables;
    TableLayout lay;
    int T, tau, Tp;
    int tile_begin, n_tiles;
    int n_lib;          // libraries in this block
    int lib_parts;      // grid.y: libraries split into this many parts
    int64_t rho_col0;   // column of the block's first library in rho
    float *rho;
    int64_t ld_rho;
    // time-delay form: the tables were built for horizon Tp over queries
    // and candidates t >= s_lo; this launch cross-maps at lag `lag`
    // (gathers y(s + lag), observes y(t + lag)).  Plain cross map: s_lo = 0,
    // lag = Tp (chunked kernels only).
    int s_lo;
    int lag;
    // device-planned launch (chunked and L2 kernels): the tile range comes
    // from *slot, the library split is chosen in the kernel for about `want`
    // CTAs, and the 1-D grid is an upper bound (surplus CTAs return).
    // slot == nullptr: tile_begin / n_tiles / lib_parts as given, grid
    // (n_tiles, lib_parts).  With a slot, n_tiles is the grid size.
    const SlotDesc *slot = nullptr;
    int want = 0;
};

// (tile, library part) of this CTA, or false when the CTA has no work.
// Tiles are sorted by ascending E and a tile's cost grows with E, so the
// blocks take them from the last one backwards: the costliest tiles start
// in the first wave and the cheap ones fill the tail.
__device__ __forceinline__ bool lookup_item(const LookupArgs &a, int &tile, int &part, int &parts)
{
    if (a.slot) {
        const int ntb = a.slot->n_tiles;
        if (ntb <= 0)
            return false;
        parts = (a.want + ntb - 1) / ntb;
        const int cap = (a.n_lib + 7) / 8;
        parts = parts < 1 ? 1 : (parts > cap ? cap : parts);
        if ((int)blockIdx.x >= ntb * parts)
            return false;
        tile = a.slot->tile_begin + ntb - 1 - (int)blockIdx.x / parts;
        part = (int)blockIdx.x % parts;
        return true;
    }
    tile = a.tile_begin + a.n_tiles - 1 - (int)blockIdx.x;
    part = (int)blockIdx.y;
    parts = a.lib_parts;
    return true;
}

// Observation sums (S_o, n S_oo - S_o^2) of every staged target at lag
// `lag` over the query times max((E-1)tau, s_lo) .. T-1-Tp of its tile's E,
// from the staged (FP32 or FP16) values.
cudaError_t launch_obs_moments(const float *tiles, int RB, const TileMeta *meta, int n_tiles, int T, int tau, int Tp,
                               int s_lo, int lag, float2 *omom, cudaStream_t st);

size_t lookup_smem_bytes(int T);
// All tiles in [tile_begin, tile_begin + n_tiles) must have this E.
cudaError_t launch_lookup(const LookupArgs &a, int E, cudaStream_t st);
// 16-byte chunked gathers (FP32 or FP16 tiles) with RB-byte tile rows.
size_t chunked_smem_bytes(int T, int RB);
// Widest tile row (128 or 64 bytes) whose tile fits shared memory; 0: none.
int chunked_row_bytes(int T);
// Tiles of any E / format in one launch (each CTA runs its tile's variant).
cudaError_t launch_lookup_multi(const LookupArgs &a, int RB, cudaStream_t st);
// Tiles too long for shared memory (T beyond about 3,500): FP32 tiles of
// 128-byte rows read from global memory / L2 (lookup_l2.cu).
// Two launches, one per register class: tiles with E + 1 <= kL2SplitK,
// then the larger E (tiles are sorted by E: n_small = tiles of the first
// class at the start of the range); sms = SM count.
constexpr int kL2SplitK = 9;
bool lookup_needs_l2(int T);
cudaError_t launch_lookup_l2(const LookupArgs &a, int n_small, int sms, cudaStream_t st);
cudaError_t launch_prep_targets_f16(const float *Y, int64_t ldY, int T, int tau, int Tp, const int32_t *pi,
                                    const TileMeta *meta, int n_tiles, uint8_t *tiles, float2 *omom, cudaStream_t st,
                                    int RB = 128);

// Validation pass (EDM_FLAG_VALIDATE): index of the first series holding a
// non-finite value, or -1 (synchronises `st`).
cudaError_t first_nonfinite_series(const float *Y, int64_t N, int64_t T, int64_t ldY, cudaStream_t st,
                                   int64_t *first_bad);

// Launch accounting shared by the translation units (edm_api.cu).
void note_launches(int kernel, int64_t n);
bool profiling();
// Takes ownership of the two events (destroyed by edm_profile_read).
void prof_push(int kernel, cudaEvent_t a, cudaEvent_t b, double units);

// Adjoint (backward.cu).
struct BwArgs {
    const float *Y;
    int64_t ldY;
    int T, tau, Tp, excl;
    const int32_t *optE;
    const float *grad_rho;
    int64_t ld_g;
    const uint8_t *tables;
    TableLayout lay;
    int64_t lib0;
    int n_lib;
    int N;
    float4 *stats;
    float *obar;
    const int32_t *pi;
    const int32_t *e_start;
    float *grad_Y;
};
int bw_max_T();
cudaError_t launch_backward(const BwArgs &a, int kmax, cudaStream_t st);

}  // namespace edm
