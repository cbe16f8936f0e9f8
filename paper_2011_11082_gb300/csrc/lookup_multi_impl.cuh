// lookup_multi_impl.cuh -- one instantiation of the multi-variant chunked
// lookup kernel and its launcher.  The including file defines EDM_RB (tile
// row bytes, 128 or 64), EDM_LAG (time-delay form), EDM_MULTI_NAME (kernel),
// EDM_MULTI_LAUNCH (launcher) and EDM_MULTI_TIMEOUTS (reader of the unit's
// bounded-wait counter); each combination is its own translation unit so the
// variants compile in parallel.
#include "lookup_chunked.cuh"

namespace edm {

// One launch for a block of tiles of mixed E (and FP16/FP32 tiles): each
// CTA runs the variant of its own tile, so a CTA only ever executes one
// specialisation's code.
__global__ void __launch_bounds__(kCkThreads, 1) EDM_MULTI_NAME(LookupArgs a)
{
    int tile, part, parts;
    if (!lookup_item(a, tile, part, parts))
        return;
    const TileMeta m = a.meta[tile];
    const bool f16 = (m.flags & kTileF16) != 0;
#define EDM_MK(KK)                                                                                                     \
    case KK:                                                                                                           \
        if (f16 && KK <= kF16MaxK)                                                                                     \
            lookup_chunk_body<(KK <= kF16MaxK ? KK : 2), true, EDM_RB, EDM_LAG>(a, tile, part, parts);                  \
        else                                                                                                           \
            lookup_chunk_body<KK, false, EDM_RB, EDM_LAG>(a, tile, part, parts);                                       \
        break;
    switch (m.E + 1) {
        EDM_MK(2)
        EDM_MK(3)
        EDM_MK(4)
        EDM_MK(5)
        EDM_MK(6)
        EDM_MK(7)
        EDM_MK(8)
        EDM_MK(9)
        EDM_MK(10)
        EDM_MK(11)
        EDM_MK(12)
        EDM_MK(13)
        EDM_MK(14)
        EDM_MK(15)
        EDM_MK(16)
        EDM_MK(17)
        EDM_MK(18)
        EDM_MK(19)
        EDM_MK(20)
        EDM_MK(21)
    default: break;
    }
#undef EDM_MK
}

EDM_WAIT_TIMEOUT_READER(EDM_MULTI_TIMEOUTS)

cudaError_t EDM_MULTI_LAUNCH(const LookupArgs &a, cudaStream_t st)
{
    if (a.n_tiles <= 0 || a.n_lib <= 0)
        return cudaSuccess;
    const size_t smem = chunked_smem_bytes(a.T, EDM_RB);
    cudaError_t e = cudaFuncSetAttribute(EDM_MULTI_NAME, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    const dim3 grid = a.slot ? dim3((unsigned)a.n_tiles) : dim3((unsigned)a.n_tiles, (unsigned)a.lib_parts);
    EDM_MULTI_NAME<<<grid, kCkThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace edm
