// Instantiations and launchers of the cuckoo put (Algorithm 4): the ordered
// per-tile kernel when the number of tiles is bounded (max_tiles > 0, e.g. a
// sequential run); otherwise the stream kernel when tiles keep 4 or 8 loads
// in flight, or the warp-batched chunk kernel with one.
#include "cht_cuckoo_warp.cuh"
#include "cht_kernels.cuh"
#include "cht_launch.h"

namespace cht {

template <int T, int FPW>
static cudaError_t run_ordered(const LaunchParams &lp, const TableArgs &ta, const void *keys,
                               uint64_t n, uint8_t *status, uint64_t *dropped) {
    auto kern = k_cuckoo_insert<T, FPW>;
    const size_t smem = smem_bytes(lp.cta, lp.items);
    const int blocks = grid_blocks((const void *)kern, T, lp, n, smem);
    kern<<<blocks, lp.cta, smem, lp.stream>>>(ta, keys, n, status, dropped, lp.items);
    return cudaGetLastError();
}

template <int T, int FPW, int I>
static cudaError_t run_warp(const LaunchParams &lp, const TableArgs &ta, const void *keys,
                            uint64_t n, uint8_t *status, uint64_t *dropped) {
    auto kern = k_cuckoo_insert_warp<T, FPW, I>;
    const int blocks = grid_blocks_warp((const void *)kern, lp, (n + I - 1) / I);
    kern<<<blocks, lp.cta, 0, lp.stream>>>(ta, keys, n, status, dropped);
    return cudaGetLastError();
}

template <int T, int FPW, int Q>
static cudaError_t run_stream(const LaunchParams &lp, const TableArgs &ta, const void *keys,
                              uint64_t n, uint8_t *status, uint64_t *dropped) {
    auto kern = k_cuckoo_insert_stream<T, FPW, Q>;
    const int blocks = grid_blocks_warp((const void *)kern, lp, n);
    kern<<<blocks, lp.cta, 0, lp.stream>>>(ta, keys, n, status, dropped);
    return cudaGetLastError();
}

template <int T, int FPW>
static cudaError_t run(const LaunchParams &lp, const TableArgs &ta, const void *keys, uint64_t n,
                       uint8_t *status, uint64_t *dropped) {
    if (lp.max_tiles > 0) return run_ordered<T, FPW>(lp, ta, keys, n, status, dropped);
    if (lp.in_flight == 4) return run_stream<T, FPW, 4>(lp, ta, keys, n, status, dropped);
    if (lp.in_flight == 8) return run_stream<T, FPW, 8>(lp, ta, keys, n, status, dropped);
    switch (batch_items(lp.items)) {
        case 1: return run_warp<T, FPW, 1>(lp, ta, keys, n, status, dropped);
        case 2: return run_warp<T, FPW, 2>(lp, ta, keys, n, status, dropped);
        default: return run_warp<T, FPW, 4>(lp, ta, keys, n, status, dropped);
    }
}

template <int T>
static cudaError_t by_fpw(int fpw, const LaunchParams &lp, const TableArgs &ta, const void *keys,
                          uint64_t n, uint8_t *status, uint64_t *dropped) {
    switch (fpw) {
        case 1: return run<T, 1>(lp, ta, keys, n, status, dropped);
        case 2: return run<T, 2>(lp, ta, keys, n, status, dropped);
        case 3: return run<T, 3>(lp, ta, keys, n, status, dropped);
        case 4: return run<T, 4>(lp, ta, keys, n, status, dropped);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_cuckoo_insert(int T, int fpw, const LaunchParams &lp, const TableArgs &ta,
                                 const void *keys, uint64_t n, uint8_t *status,
                                 uint64_t *dropped) {
    switch (T) {
        case 4: return by_fpw<4>(fpw, lp, ta, keys, n, status, dropped);
        case 8: return by_fpw<8>(fpw, lp, ta, keys, n, status, dropped);
        case 16: return by_fpw<16>(fpw, lp, ta, keys, n, status, dropped);
    }
    return cudaErrorInvalidValue;
}

}  // namespace cht
