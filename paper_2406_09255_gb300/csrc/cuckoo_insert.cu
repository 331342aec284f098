// Instantiations and launcher of the cuckoo put kernel (Algorithm 4).
#include "cht_kernels.cuh"
#include "cht_launch.h"

namespace cht {

template <int T, int FPW>
static cudaError_t run(const LaunchParams &lp, const TableArgs &ta, const void *keys, uint64_t n,
                       uint8_t *status, uint64_t *dropped) {
    auto kern = k_cuckoo_insert<T, FPW>;
    const size_t smem = smem_bytes(lp.cta, lp.items);
    const int blocks = grid_blocks((const void *)kern, T, lp, n, smem);
    kern<<<blocks, lp.cta, smem, lp.stream>>>(ta, keys, n, status, dropped, lp.items);
    return cudaGetLastError();
}

#define CHT_FPW_CASES(T)                                                            \
    switch (fpw) {                                                                  \
        case 1: return run<T, 1>(lp, ta, keys, n, status, dropped);                 \
        case 2: return run<T, 2>(lp, ta, keys, n, status, dropped);                 \
        case 3: return run<T, 3>(lp, ta, keys, n, status, dropped);                 \
        case 4: return run<T, 4>(lp, ta, keys, n, status, dropped);                 \
    }                                                                               \
    break;

cudaError_t launch_cuckoo_insert(int T, int fpw, const LaunchParams &lp, const TableArgs &ta,
                                 const void *keys, uint64_t n, uint8_t *status,
                                 uint64_t *dropped) {
    switch (T) {
        case 4: CHT_FPW_CASES(4)
        case 8: CHT_FPW_CASES(8)
        case 16: CHT_FPW_CASES(16)
    }
    return cudaErrorInvalidValue;
}

}  // namespace cht
