// Instantiations and launcher of the iceberg find-or-put (Algorithm 1) and
// lookup (Section 2.3) kernels.
#include "cht_kernels.cuh"
#include "cht_launch.h"

namespace cht {

template <int T, int FPW0, bool LOOKUP>
static cudaError_t run(const LaunchParams &lp, const TableArgs &ta, const void *keys, uint64_t n,
                       uint8_t *status) {
    auto kern = k_iceberg<T, FPW0, LOOKUP>;
    const size_t smem = smem_bytes(lp.cta, lp.items);
    const int blocks = grid_blocks((const void *)kern, T, lp, n, smem);
    kern<<<blocks, lp.cta, smem, lp.stream>>>(ta, keys, n, status, lp.items);
    return cudaGetLastError();
}

template <int T>
static cudaError_t by_fpw(int fpw0, bool lookup, const LaunchParams &lp, const TableArgs &ta,
                          const void *keys, uint64_t n, uint8_t *status) {
    switch (fpw0) {
        case 1: return lookup ? run<T, 1, true>(lp, ta, keys, n, status)
                              : run<T, 1, false>(lp, ta, keys, n, status);
        case 2: return lookup ? run<T, 2, true>(lp, ta, keys, n, status)
                              : run<T, 2, false>(lp, ta, keys, n, status);
        case 3: return lookup ? run<T, 3, true>(lp, ta, keys, n, status)
                              : run<T, 3, false>(lp, ta, keys, n, status);
        case 4: return lookup ? run<T, 4, true>(lp, ta, keys, n, status)
                              : run<T, 4, false>(lp, ta, keys, n, status);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_iceberg(int T, int fpw0, bool lookup, const LaunchParams &lp,
                           const TableArgs &ta, const void *keys, uint64_t n, uint8_t *status) {
    switch (T) {
        case 4: return by_fpw<4>(fpw0, lookup, lp, ta, keys, n, status);
        case 8: return by_fpw<8>(fpw0, lookup, lp, ta, keys, n, status);
        case 16: return by_fpw<16>(fpw0, lookup, lp, ta, keys, n, status);
    }
    return cudaErrorInvalidValue;
}

}  // namespace cht

namespace cht {

template <int T, int FPW0, bool LOOKUP>
static cudaError_t run_batch(const LaunchParams &lp, const BatchDesc *bd, int count,
                             uint64_t total_chunks, unsigned long long *ctr) {
    auto kern = k_iceberg_batch<T, FPW0, LOOKUP>;
    const size_t smem = (size_t)((count + 2) & ~1) * 8 + smem_bytes(lp.cta, lp.items);
    const uint64_t tiles_per_block = lp.cta / T;
    uint64_t need = (total_chunks + tiles_per_block - 1) / tiles_per_block;
    uint64_t cap = (uint64_t)lp.sms * occupancy((const void *)kern, lp.cta, smem);
    if (lp.max_ctas > 0 && cap > (uint64_t)lp.max_ctas) cap = lp.max_ctas;
    int blocks = (int)(need < cap ? need : cap);
    if (blocks < 1) blocks = 1;
    kern<<<blocks, lp.cta, smem, lp.stream>>>(bd, count, lp.items, ctr);
    return cudaGetLastError();
}

template <int T>
static cudaError_t batch_by_fpw(int fpw0, bool lookup, const LaunchParams &lp,
                                const BatchDesc *bd, int count, uint64_t total_chunks,
                                unsigned long long *ctr) {
    switch (fpw0) {
        case 1: return lookup ? run_batch<T, 1, true>(lp, bd, count, total_chunks, ctr)
                              : run_batch<T, 1, false>(lp, bd, count, total_chunks, ctr);
        case 2: return lookup ? run_batch<T, 2, true>(lp, bd, count, total_chunks, ctr)
                              : run_batch<T, 2, false>(lp, bd, count, total_chunks, ctr);
        case 3: return lookup ? run_batch<T, 3, true>(lp, bd, count, total_chunks, ctr)
                              : run_batch<T, 3, false>(lp, bd, count, total_chunks, ctr);
        case 4: return lookup ? run_batch<T, 4, true>(lp, bd, count, total_chunks, ctr)
                              : run_batch<T, 4, false>(lp, bd, count, total_chunks, ctr);
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

}  // namespace cht

namespace cht {

// fused find-or-put launch that allocates nothing on the host either: the
// grid comes from a direct occupancy query instead of the cached one
template <int FPW0>
static cudaError_t run_batch_noalloc(cudaStream_t s, int sms, const BatchDesc *bd, int count,
                                     uint64_t total_chunks) {
    constexpr int T = 4, kItems = 2, kCta = 256;
    auto kern = k_iceberg_batch<T, FPW0, false>;
    const size_t smem = (size_t)((count + 2) & ~1) * 8 + smem_bytes(kCta, kItems);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kCta, smem) != cudaSuccess ||
        occ < 1)
        occ = 1;
    const uint64_t need = (total_chunks + kCta / T - 1) / (kCta / T);
    const uint64_t cap = (uint64_t)sms * occ;
    int blocks = (int)(need < cap ? need : cap);
    if (blocks < 1) blocks = 1;
    kern<<<blocks, kCta, smem, s>>>(bd, count, kItems, nullptr);
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
