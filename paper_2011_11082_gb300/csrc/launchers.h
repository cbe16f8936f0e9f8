// launchers.h -- host-side launch helpers shared between the translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "edm.h"

namespace edm {

// Shared-memory bytes of the staged series plus per-warp kNN scratch.
size_t knn_smem_bytes(int T, int warps);
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
cudaError_t launch_knn_tables(const float *Y, int64_t ldY, int64_t lib0, int n_lib, int T, int tau, int Tp, int excl,
                              uint32_t sel, const TableLayout &lay, uint8_t *tables, cudaStream_t st,
                              int q_per_cta = 64, const uint32_t *sel_dev = nullptr);

// FP64 re-rank / exhaustive-scan query counts of the kNN kernels on the
// current device (synchronises); reset clears them.
cudaError_t knn_counters(unsigned long long out[2], bool reset);

// Public table format: idx int32 [n_lib][Tq][E+1] (unshifted), w float [n_lib][Tq][E+1].
cudaError_t launch_knn_public(const float *Y, int64_t ldY, int n_lib, int T, int E, int tau, int Tp, int excl,
                              int32_t *idx, float *w, cudaStream_t st);

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
};

size_t lookup_smem_bytes(int T);
// All tiles in [tile_begin, tile_begin + n_tiles) must have this E.
cudaError_t launch_lookup(const LookupArgs &a, int E, cudaStream_t st);
// 16-byte chunked gathers (FP32 or FP16 tiles) with RB-byte tile rows.
size_t chunked_smem_bytes(int T, int RB);
// Widest tile row (128 or 64 bytes) whose tile fits shared memory; 0: none.
int chunked_row_bytes(int T);
// Tiles of any E / format in one launch (each CTA runs its tile's variant).
cudaError_t launch_lookup_multi(const LookupArgs &a, int RB, cudaStream_t st);
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
    int T, tau, Tp;
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
