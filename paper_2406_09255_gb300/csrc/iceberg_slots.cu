// Instantiations of the warp-batched iceberg engine that also return each
// key's slot index and move values (find-or-put and lookup with slots, and
// the fused put / get of the key-value extension). One key per lane.
#include "cht_kernels.cuh"
#include "cht_launch.h"
#include "cht_warp.cuh"

namespace cht {

template <int T, int FPW0, bool LOOKUP>
static cudaError_t run(const LaunchParams &lp, const TableArgs &ta, const void *keys, uint64_t n,
                       uint8_t *status, uint64_t *slots, const KVArgs &kv) {
    auto kern = k_iceberg_warp_slots<T, FPW0, LOOKUP>;
    const int blocks = grid_blocks_warp((const void *)kern, lp, n);
    kern<<<blocks, lp.cta, 0, lp.stream>>>(ta, keys, n, status, slots, kv);
    return cudaGetLastError();
}

template <int T, bool LOOKUP>
static cudaError_t by_fpw(int fpw0, const LaunchParams &lp, const TableArgs &ta,
                          const void *keys, uint64_t n, uint8_t *status, uint64_t *slots,
                          const KVArgs &kv) {
    switch (fpw0) {
        case 1: return run<T, 1, LOOKUP>(lp, ta, keys, n, status, slots, kv);
        case 2: return run<T, 2, LOOKUP>(lp, ta, keys, n, status, slots, kv);
        case 3: return run<T, 3, LOOKUP>(lp, ta, keys, n, status, slots, kv);
        case 4: return run<T, 4, LOOKUP>(lp, ta, keys, n, status, slots, kv);
    }
    return cudaErrorInvalidValue;
}

template <bool LOOKUP>
static cudaError_t by_tile(int T, int fpw0, const LaunchParams &lp, const TableArgs &ta,
                           const void *keys, uint64_t n, uint8_t *status, uint64_t *slots,
                           const KVArgs &kv) {
    switch (T) {
        case 4: return by_fpw<4, LOOKUP>(fpw0, lp, ta, keys, n, status, slots, kv);
        case 8: return by_fpw<8, LOOKUP>(fpw0, lp, ta, keys, n, status, slots, kv);
        case 16: return by_fpw<16, LOOKUP>(fpw0, lp, ta, keys, n, status, slots, kv);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_iceberg_warp_slots(int T, int fpw0, bool lookup, const LaunchParams &lp,
                                      const TableArgs &ta, const void *keys, uint64_t n,
                                      uint8_t *status, uint64_t *slots, const KVArgs &kv) {
    return lookup ? by_tile<true>(T, fpw0, lp, ta, keys, n, status, slots, kv)
                  : by_tile<false>(T, fpw0, lp, ta, keys, n, status, slots, kv);
}

}  // namespace cht
