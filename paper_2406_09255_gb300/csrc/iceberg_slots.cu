// Instantiations of the warp-batched iceberg engine that also return each
// key's slot index (find-or-put and lookup with slots: the key-value
// extension). One key per lane.
#include "cht_kernels.cuh"
#include "cht_launch.h"
#include "cht_warp.cuh"

namespace cht {

template <int T, int FPW0, bool LOOKUP>
static cudaError_t run(const LaunchParams &lp, const TableArgs &ta, const void *keys, uint64_t n,
                       uint8_t *status, uint64_t *slots) {
    auto kern = k_iceberg_warp<T, FPW0, 1, LOOKUP, true>;
    const int blocks = grid_blocks_warp((const void *)kern, lp, n);
    kern<<<blocks, lp.cta, 0, lp.stream>>>(ta, keys, n, status, slots);
    return cudaGetLastError();
}

template <int T, bool LOOKUP>
static cudaError_t by_fpw(int fpw0, const LaunchParams &lp, const TableArgs &ta,
                          const void *keys, uint64_t n, uint8_t *status, uint64_t *slots) {
    switch (fpw0) {
        case 1: return run<T, 1, LOOKUP>(lp, ta, keys, n, status, slots);
        case 2: return run<T, 2, LOOKUP>(lp, ta, keys, n, status, slots);
        case 3: return run<T, 3, LOOKUP>(lp, ta, keys, n, status, slots);
        case 4: return run<T, 4, LOOKUP>(lp, ta, keys, n, status, slots);
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

cudaError_t launch_iceberg_warp_slots(int T, int fpw0, bool lookup, const LaunchParams &lp,
                                      const TableArgs &ta, const void *keys, uint64_t n,
                                      uint8_t *status, uint64_t *slots) {
    return lookup ? by_tile<true>(T, fpw0, lp, ta, keys, n, status, slots)
                  : by_tile<false>(T, fpw0, lp, ta, keys, n, status, slots);
}

}  // namespace cht
