// Instantiations and launcher of the cuckoo lookup kernel (Section 4.4).
#include "cht_kernels.cuh"
#include "cht_launch.h"

namespace cht {

template <int T, int FPW>
static cudaError_t run(const LaunchParams &lp, const TableArgs &ta, const void *keys, uint64_t n,
                       uint8_t *status) {
    auto kern = k_cuckoo_find<T, FPW>;
    const size_t smem = smem_bytes(lp.cta, lp.items);
    const int blocks = grid_blocks((const void *)kern, T, lp, n, smem);
    kern<<<blocks, lp.cta, smem, lp.stream>>>(ta, keys, n, status, lp.items);
    return cudaGetLastError();
}

#define CHT_FPW_CASES(T)                                            \
    switch (fpw) {                                                  \
        case 1: return run<T, 1>(lp, ta, keys, n, status);          \
        case 2: return run<T, 2>(lp, ta, keys, n, status);          \
        case 3: return run<T, 3>(lp, ta, keys, n, status);          \
        case 4: return run<T, 4>(lp, ta, keys, n, status);          \
    }                                                               \
    break;

cudaError_t launch_cuckoo_find(int T, int fpw, const LaunchParams &lp, const TableArgs &ta,
                               const void *keys, uint64_t n, uint8_t *status) {
    switch (T) {
        case 4: CHT_FPW_CASES(4)
        case 8: CHT_FPW_CASES(8)
        case 16: CHT_FPW_CASES(16)
    }
    return cudaErrorInvalidValue;
}

}  // namespace cht
