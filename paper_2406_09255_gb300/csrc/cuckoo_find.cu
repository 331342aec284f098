// Instantiations and launcher of the cuckoo lookup kernel (Section 4.4).
#include "cht_kernels.cuh"
#include "cht_launch.h"

namespace cht {

template <int T, int FPW, int P>
static cudaError_t run(const LaunchParams &lp, const TableArgs &ta, const void *keys, uint64_t n,
                       uint8_t *status) {
    auto kern = k_cuckoo_find<T, FPW, P>;
    const int blocks = grid_blocks_warp((const void *)kern, lp, n);
    kern<<<blocks, lp.cta, 0, lp.stream>>>(ta, keys, n, status);
    return cudaGetLastError();
}

template <int T, int FPW>
static cudaError_t by_p(const LaunchParams &lp, const TableArgs &ta, const void *keys, uint64_t n,
                        uint8_t *status) {
    switch (lp.in_flight) {
        case 1: return run<T, FPW, 1>(lp, ta, keys, n, status);
        case 2: return run<T, FPW, 2>(lp, ta, keys, n, status);
        case 4: return run<T, FPW, 4>(lp, ta, keys, n, status);
    }
    return cudaErrorInvalidValue;
}

template <int T>
static cudaError_t by_fpw(int fpw, const LaunchParams &lp, const TableArgs &ta, const void *keys,
                          uint64_t n, uint8_t *status) {
    switch (fpw) {
        case 1: return by_p<T, 1>(lp, ta, keys, n, status);
        case 2: return by_p<T, 2>(lp, ta, keys, n, status);
        case 3: return by_p<T, 3>(lp, ta, keys, n, status);
        case 4: return by_p<T, 4>(lp, ta, keys, n, status);
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
