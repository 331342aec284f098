// Instantiations and launcher of the cuckoo lookup kernels (Section 4.4).
#include "cht_kernels.cuh"
#include "cht_launch.h"

namespace cht {

template <int T, int FPW>
static cudaError_t run_rounds(const LaunchParams &lp, const TableArgs &ta, const void *keys,
                              uint64_t n, uint8_t *status) {
    auto kern = k_cuckoo_find<T, FPW>;
    const int blocks = grid_blocks_warp((const void *)kern, lp, n);
    kern<<<blocks, lp.cta, 0, lp.stream>>>(ta, keys, n, status);
    return cudaGetLastError();
}

template <int T, int FPW, int Q>
static cudaError_t run_stream(const LaunchParams &lp, const TableArgs &ta, const void *keys,
                              uint64_t n, uint8_t *status) {
    auto kern = k_cuckoo_find_stream<T, FPW, Q>;
    const int blocks = grid_blocks_warp((const void *)kern, lp, n);
    kern<<<blocks, lp.cta, 0, lp.stream>>>(ta, keys, n, status);
    return cudaGetLastError();
}

// lookups_in_flight: 1 = one bucket load in flight per tile (per-round form),
// 4 or 8 = that many per tile (stream form)
template <int T, int FPW>
static cudaError_t by_q(const LaunchParams &lp, const TableArgs &ta, const void *keys, uint64_t n,
                        uint8_t *status) {
    switch (lp.in_flight) {
        case 1: return run_rounds<T, FPW>(lp, ta, keys, n, status);
        case 4: return run_stream<T, FPW, 4>(lp, ta, keys, n, status);
        case 8: return run_stream<T, FPW, 8>(lp, ta, keys, n, status);
    }
    return cudaErrorInvalidValue;
}

template <int T>
static cudaError_t by_fpw(int fpw, const LaunchParams &lp, const TableArgs &ta, const void *keys,
                          uint64_t n, uint8_t *status) {
    switch (fpw) {
        case 1: return by_q<T, 1>(lp, ta, keys, n, status);
        case 2: return by_q<T, 2>(lp, ta, keys, n, status);
        case 3: return by_q<T, 3>(lp, ta, keys, n, status);
        case 4: return by_q<T, 4>(lp, ta, keys, n, status);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_cuckoo_find(int T, int fpw, const LaunchParams &lp, const TableArgs &ta,
                               const void *keys, uint64_t n, uint8_t *status) {
    switch (T) {
        case 4: return by_fpw<4>(fpw, lp, ta, keys, n, status);
        case 8: return by_fpw<8>(fpw, lp, ta, keys, n, status);
        case 16: return by_fpw<16>(fpw, lp, ta, keys, n, status);
    }
    return cudaErrorInvalidValue;
}

}  // namespace cht
