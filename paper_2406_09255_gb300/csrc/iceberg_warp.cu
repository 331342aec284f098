// Instantiations and launchers of the iceberg engines for one table
// (find-or-put and lookup): the warp-batched chunk engine (one bucket load in
// flight per tile, lookups_in_flight = 1), or the level-1 stream kernel
// followed by the level-2 pass over the keys it left pending (4 or 8 loads
// in flight). Runs that return slot indices go to the instantiations in
// iceberg_slots.cu.
#include "cht_iceberg_stream.cuh"
#include "cht_kernels.cuh"
#include "cht_launch.h"
#include "cht_warp.cuh"

namespace cht {

// ---- stream form: level 1 as a stream of packed rounds, then level 2 ----
template <int T, int FPW0, int Q, bool LOOKUP>
static cudaError_t run_stream(const LaunchParams &lp, const TableArgs &ta, const void *keys,
                              uint64_t n, uint8_t *status) {
    auto k1 = k_iceberg_stream<T, FPW0, Q, LOOKUP>;
    k1<<<grid_blocks_warp((const void *)k1, lp, n), lp.cta, 0, lp.stream>>>(ta, keys, n,
                                                                           status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the level-2 pass reads every status and takes the pending keys
    auto k2 = k_iceberg_resume<T, FPW0, LOOKUP>;
    k2<<<grid_blocks_warp((const void *)k2, lp, n), lp.cta, 0, lp.stream>>>(ta, keys, n,
                                                                           status);
    return cudaGetLastError();
}

// ---- warp engine, one table ----------------------------------------------
template <int T, int FPW0, int I, bool LOOKUP>
static cudaError_t run_warp(const LaunchParams &lp, const TableArgs &ta, const void *keys,
                            uint64_t n, uint8_t *status, uint64_t *slots) {
    auto kern = k_iceberg_warp<T, FPW0, I, LOOKUP>;
    const int blocks = grid_blocks_warp((const void *)kern, lp, (n + I - 1) / I);
    kern<<<blocks, lp.cta, 0, lp.stream>>>(ta, keys, n, status);
    return cudaGetLastError();
}

template <int T, int FPW0, bool LOOKUP>
static cudaError_t by_items(const LaunchParams &lp, const TableArgs &ta, const void *keys,
                            uint64_t n, uint8_t *status, uint64_t *slots) {
    if (lp.in_flight == 4) return run_stream<T, FPW0, 4, LOOKUP>(lp, ta, keys, n, status);
    if (lp.in_flight == 8) return run_stream<T, FPW0, 8, LOOKUP>(lp, ta, keys, n, status);
    switch (batch_items(lp.items)) {
        case 1: return run_warp<T, FPW0, 1, LOOKUP>(lp, ta, keys, n, status, slots);
        case 2: return run_warp<T, FPW0, 2, LOOKUP>(lp, ta, keys, n, status, slots);
        default: return run_warp<T, FPW0, 4, LOOKUP>(lp, ta, keys, n, status, slots);
    }
}

template <int T, bool LOOKUP>
static cudaError_t by_fpw(int fpw0, const LaunchParams &lp, const TableArgs &ta,
                          const void *keys, uint64_t n, uint8_t *status, uint64_t *slots) {
    switch (fpw0) {
        case 1: return by_items<T, 1, LOOKUP>(lp, ta, keys, n, status, slots);
        case 2: return by_items<T, 2, LOOKUP>(lp, ta, keys, n, status, slots);
        case 3: return by_items<T, 3, LOOKUP>(lp, ta, keys, n, status, slots);
        case 4: return by_items<T, 4, LOOKUP>(lp, ta, keys, n, status, slots);
    }
    return cudaErrorInvalidValue;
}

template <bool LOOKUP>
static cudaError_t by_tile(int T, int fpw0, const LaunchParams &lp, const TableArgs &ta,
                           const void *keys, uint64_t n, uint8_t *status, uint64_t *slots) {
    switch (T) {
        case 4: return by_fpw<4, LOOKUP>(fpw0, lp, ta, keys, n, status, slots);
        case 8: return by_fpw<8, LOOKUP>(fpw0, lp, ta, keys, n, status, slots);
        case 16: return by_fpw<16, LOOKUP>(fpw0, lp, ta, keys, n, status, slots);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_iceberg_warp(int T, int fpw0, bool lookup, const LaunchParams &lp,
                                const TableArgs &ta, const void *keys, uint64_t n,
                                uint8_t *status, uint64_t *slots, const KVArgs *kv) {
    if (slots || (kv && kv->store))
        return launch_iceberg_warp_slots(T, fpw0, lookup, lp, ta, keys, n, status, slots,
                                         kv ? *kv : KVArgs{});
    return lookup ? by_tile<true>(T, fpw0, lp, ta, keys, n, status, slots)
                  : by_tile<false>(T, fpw0, lp, ta, keys, n, status, slots);
}

}  // namespace cht
