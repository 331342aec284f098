// Tables with 32- or 64-byte buckets (4 or 8 words: the bucket sizes of 8
// and 16 32-bit slots that Section 5.1 sweeps beside 32): instantiations of
// the cuckoo and iceberg kernels for those widths, with two words (16 bytes)
// per lane, i.e. tiles of 2 or 4 lanes. Cuckoo lookups and puts use the
// stream kernels (four loads in flight per tile), iceberg operations the
// warp-batched engine with one key per lane; a bounded number of tiles
// (max_tiles > 0) selects the ordered engines, as for 128-byte buckets.
#include "cht_cuckoo_warp.cuh"
#include "cht_kernels.cuh"
#include "cht_launch.h"
#include "cht_warp.cuh"

namespace cht {

template <int WPB, int FPW>
static cudaError_t cuckoo_insert(const LaunchParams &lp, const TableArgs &ta, const void *keys,
                                 uint64_t n, uint8_t *status, uint64_t *dropped) {
    constexpr int T = WPB / 2;
    if (lp.max_tiles > 0) {
        auto kern = k_cuckoo_insert<T, FPW, WPB>;
        const size_t smem = smem_bytes(lp.cta, lp.items);
        const int blocks = grid_blocks((const void *)kern, T, lp, n, smem);
        kern<<<blocks, lp.cta, smem, lp.stream>>>(ta, keys, n, status, dropped, lp.items);
    } else {
        auto kern = k_cuckoo_insert_stream<T, FPW, 4, WPB>;
        const int blocks = grid_blocks_warp((const void *)kern, lp, n);
        kern<<<blocks, lp.cta, 0, lp.stream>>>(ta, keys, n, status, dropped);
    }
    return cudaGetLastError();
}

template <int WPB, int FPW>
static cudaError_t cuckoo_find(const LaunchParams &lp, const TableArgs &ta, const void *keys,
                               uint64_t n, uint8_t *status) {
    constexpr int T = WPB / 2;
    auto kern = k_cuckoo_find_stream<T, FPW, 4, WPB>;
    const int blocks = grid_blocks_warp((const void *)kern, lp, n);
    kern<<<blocks, lp.cta, 0, lp.stream>>>(ta, keys, n, status);
    return cudaGetLastError();
}

template <int WPB, int FPW0, bool LOOKUP>
static cudaError_t iceberg(const LaunchParams &lp, const TableArgs &ta, const void *keys,
                           uint64_t n, uint8_t *status) {
    constexpr int T = WPB / 2;
    if (lp.max_tiles > 0) {
        auto kern = k_iceberg<T, FPW0, LOOKUP, WPB>;
        const size_t smem = smem_bytes(lp.cta, lp.items);
        const int blocks = grid_blocks((const void *)kern, T, lp, n, smem);
        kern<<<blocks, lp.cta, smem, lp.stream>>>(ta, keys, n, status, nullptr, KVArgs{},
                                                  lp.items);
    } else {
        auto kern = k_iceberg_warp<T, FPW0, 1, LOOKUP, WPB>;
        const int blocks = grid_blocks_warp((const void *)kern, lp, n);
        kern<<<blocks, lp.cta, 0, lp.stream>>>(ta, keys, n, status);
    }
    return cudaGetLastError();
}

template <int WPB, int FPW>
static cudaError_t by_op(int op, const LaunchParams &lp, const TableArgs &ta, const void *keys,
                         uint64_t n, uint8_t *status, uint64_t *dropped) {
    switch (op) {
        case kSmallCuckooInsert: return cuckoo_insert<WPB, FPW>(lp, ta, keys, n, status, dropped);
        case kSmallCuckooFind: return cuckoo_find<WPB, FPW>(lp, ta, keys, n, status);
        case kSmallIcebergFop: return iceberg<WPB, FPW, false>(lp, ta, keys, n, status);
        case kSmallIcebergFind: return iceberg<WPB, FPW, true>(lp, ta, keys, n, status);
    }
    return cudaErrorInvalidValue;
}

template <int WPB>
static cudaError_t by_fpw(int op, int fpw, const LaunchParams &lp, const TableArgs &ta,
                          const void *keys, uint64_t n, uint8_t *status, uint64_t *dropped) {
    switch (fpw) {
        case 1: return by_op<WPB, 1>(op, lp, ta, keys, n, status, dropped);
        case 2: return by_op<WPB, 2>(op, lp, ta, keys, n, status, dropped);
        case 3: return by_op<WPB, 3>(op, lp, ta, keys, n, status, dropped);
        case 4: return by_op<WPB, 4>(op, lp, ta, keys, n, status, dropped);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_small_buckets(int op, int wpb, int fpw, const LaunchParams &lp,
                                 const TableArgs &ta, const void *keys, uint64_t n,
                                 uint8_t *status, uint64_t *dropped) {
    switch (wpb) {
        case 4: return by_fpw<4>(op, fpw, lp, ta, keys, n, status, dropped);
        case 8: return by_fpw<8>(op, fpw, lp, ta, keys, n, status, dropped);
    }
    return cudaErrorInvalidValue;
}

}  // namespace cht
