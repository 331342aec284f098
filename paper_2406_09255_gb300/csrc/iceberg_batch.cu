// Instantiations and launchers of the fused multi-table batch kernels (the
// warp-batched iceberg engine over many tables) and of the allocation-free
// fused find-or-put.
#include "cht_kernels.cuh"
#include "cht_launch.h"
#include "cht_warp.cuh"

namespace cht {

// ---- warp engine, fused batch ---------------------------------------------
static size_t batch_smem(int count) { return (size_t)((count + 2) & ~1) * 8; }

template <int T, int FPW0, int I, bool LOOKUP>
static cudaError_t run_batch(const LaunchParams &lp, const BatchDesc *bd, int count,
                             uint64_t total_chunks, unsigned long long *ctr) {
    void (*kern)(const BatchDesc *, int, unsigned long long *);
    if constexpr (I == 1)
        kern = k_iceberg_batch1<T, FPW0, LOOKUP>;
    else
        kern = k_iceberg_batch<T, FPW0, I, LOOKUP>;
    const size_t smem = batch_smem(count);
    const uint64_t warps_per_block = lp.cta / 32;
    uint64_t need = (total_chunks + warps_per_block - 1) / warps_per_block;
    uint64_t cap = (uint64_t)lp.sms * occupancy((const void *)kern, lp.cta, smem);
    if (lp.max_ctas > 0 && cap > (uint64_t)lp.max_ctas) cap = lp.max_ctas;
    int blocks = (int)(need < cap ? need : cap);
    if (blocks < 1) blocks = 1;
    kern<<<blocks, lp.cta, smem, lp.stream>>>(bd, count, ctr);
    return cudaGetLastError();
}

template <int T, int FPW0, bool LOOKUP>
static cudaError_t batch_by_items(const LaunchParams &lp, const BatchDesc *bd, int count,
                                  uint64_t total_chunks, unsigned long long *ctr) {
    switch (batch_items(lp.items)) {
        case 1: return run_batch<T, FPW0, 1, LOOKUP>(lp, bd, count, total_chunks, ctr);
        case 2: return run_batch<T, FPW0, 2, LOOKUP>(lp, bd, count, total_chunks, ctr);
        default: return run_batch<T, FPW0, 4, LOOKUP>(lp, bd, count, total_chunks, ctr);
    }
}

template <int T>
static cudaError_t batch_by_fpw(int fpw0, bool lookup, const LaunchParams &lp,
                                const BatchDesc *bd, int count, uint64_t total_chunks,
                                unsigned long long *ctr) {
    switch (fpw0) {
        case 1: return lookup ? batch_by_items<T, 1, true>(lp, bd, count, total_chunks, ctr)
                              : batch_by_items<T, 1, false>(lp, bd, count, total_chunks, ctr);
        case 2: return lookup ? batch_by_items<T, 2, true>(lp, bd, count, total_chunks, ctr)
                              : batch_by_items<T, 2, false>(lp, bd, count, total_chunks, ctr);
        case 3: return lookup ? batch_by_items<T, 3, true>(lp, bd, count, total_chunks, ctr)
                              : batch_by_items<T, 3, false>(lp, bd, count, total_chunks, ctr);
        case 4: return lookup ? batch_by_items<T, 4, true>(lp, bd, count, total_chunks, ctr)
                              : batch_by_items<T, 4, false>(lp, bd, count, total_chunks, ctr);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_iceberg_batch(int T, int fpw0, bool lookup, const LaunchParams &lp,
                                 const BatchDesc *bd, int count, uint64_t total_chunks,
                                 unsigned long long *ctr) {
    switch (T) {
        case 4: return batch_by_fpw<4>(fpw0, lookup, lp, bd, count, total_chunks, ctr);
        case 8: return batch_by_fpw<8>(fpw0, lookup, lp, bd, count, total_chunks, ctr);
        case 16: return batch_by_fpw<16>(fpw0, lookup, lp, bd, count, total_chunks, ctr);
    }
    return cudaErrorInvalidValue;
}

// fused find-or-put launch that allocates nothing on the host either: the
// grid comes from a direct occupancy query instead of the cached one
template <int FPW0>
static cudaError_t run_batch_noalloc(cudaStream_t s, int sms, const BatchDesc *bd, int count,
                                     uint64_t total_chunks) {
    constexpr int kCta = 256;
    auto kern = k_iceberg_batch<kStaticBatchTile, FPW0, kStaticBatchItems, false>;
    const size_t smem = batch_smem(count);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kCta, smem) != cudaSuccess ||
        occ < 1)
        occ = 1;
    const uint64_t need = (total_chunks + kCta / 32 - 1) / (kCta / 32);
    const uint64_t cap = (uint64_t)sms * occ;
    int blocks = (int)(need < cap ? need : cap);
    if (blocks < 1) blocks = 1;
    kern<<<blocks, kCta, smem, s>>>(bd, count, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_iceberg_batch_noalloc(int fpw0, cudaStream_t s, int sms, const BatchDesc *bd,
                                         int count, uint64_t total_chunks) {
    switch (fpw0) {
        case 1: return run_batch_noalloc<1>(s, sms, bd, count, total_chunks);
        case 2: return run_batch_noalloc<2>(s, sms, bd, count, total_chunks);
        case 3: return run_batch_noalloc<3>(s, sms, bd, count, total_chunks);
        case 4: return run_batch_noalloc<4>(s, sms, bd, count, total_chunks);
    }
    return cudaErrorInvalidValue;
}

}  // namespace cht
