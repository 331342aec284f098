// Iceberg find-or-put (Algorithm 1) and lookup (Section 2.3): dispatch, and
// the ordered per-tile engine used when the number of tiles is bounded
// (max_tiles > 0); unordered runs go to the warp-batched engine
// (iceberg_warp.cu).
#include "cht_kernels.cuh"
#include "cht_launch.h"
#include "cht_warp.cuh"

namespace cht {

// ---- ordered engine ------------------------------------------------------
template <int T, int FPW0, bool LOOKUP>
static cudaError_t run_ordered(const LaunchParams &lp, const TableArgs &ta, const void *keys,
                               uint64_t n, uint8_t *status, uint64_t *slots, const KVArgs *kv) {
    auto kern = k_iceberg<T, FPW0, LOOKUP>;
    const size_t smem = smem_bytes(lp.cta, lp.items);
    const int blocks = grid_blocks((const void *)kern, T, lp, n, smem);
    kern<<<blocks, lp.cta, smem, lp.stream>>>(ta, keys, n, status, slots, kv ? *kv : KVArgs{},
                                              lp.items);
    return cudaGetLastError();
}

template <int T, int FPW0, bool LOOKUP>
static cudaError_t single(const LaunchParams &lp, const TableArgs &ta, const void *keys,
                          uint64_t n, uint8_t *status, uint64_t *slots, const KVArgs *kv) {
    if (lp.max_tiles > 0) return run_ordered<T, FPW0, LOOKUP>(lp, ta, keys, n, status, slots, kv);
    return launch_iceberg_warp(T, FPW0, LOOKUP, lp, ta, keys, n, status, slots, kv);
}

template <int T>
static cudaError_t by_fpw(int fpw0, bool lookup, const LaunchParams &lp, const TableArgs &ta,
                          const void *keys, uint64_t n, uint8_t *status, uint64_t *slots,
                          const KVArgs *kv) {
    switch (fpw0) {
        case 1: return lookup ? single<T, 1, true>(lp, ta, keys, n, status, slots, kv)
                              : single<T, 1, false>(lp, ta, keys, n, status, slots, kv);
        case 2: return lookup ? single<T, 2, true>(lp, ta, keys, n, status, slots, kv)
                              : single<T, 2, false>(lp, ta, keys, n, status, slots, kv);
        case 3: return lookup ? single<T, 3, true>(lp, ta, keys, n, status, slots, kv)
                              : single<T, 3, false>(lp, ta, keys, n, status, slots, kv);
        case 4: return lookup ? single<T, 4, true>(lp, ta, keys, n, status, slots, kv)
                              : single<T, 4, false>(lp, ta, keys, n, status, slots, kv);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_iceberg(int T, int fpw0, bool lookup, const LaunchParams &lp,
                           const TableArgs &ta, const void *keys, uint64_t n, uint8_t *status,
                           uint64_t *slots, const KVArgs *kv) {
    switch (T) {
        case 4: return by_fpw<4>(fpw0, lookup, lp, ta, keys, n, status, slots, kv);
        case 8: return by_fpw<8>(fpw0, lookup, lp, ta, keys, n, status, slots, kv);
        case 16: return by_fpw<16>(fpw0, lookup, lp, ta, keys, n, status, slots, kv);
    }
    return cudaErrorInvalidValue;
}

}  // namespace cht
