// cht_launch.h - host-side launch helpers shared by the kernel translation
// units and the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>

#include "cht_device.cuh"

namespace cht {

struct LaunchParams {
    int cta;        // threads per block
    int items;      // keys per thread per chunk
    int max_ctas;   // 0 = fill the GPU
    int max_tiles;  // 0 = unbounded
    int in_flight;  // lookups a tile keeps in flight (cuckoo lookup)
    int sms;        // multiprocessors of the device
    cudaStream_t stream;
};

// resident blocks per SM for a kernel at a given block size and shared memory
inline int occupancy(const void *kern, int cta, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, size_t>, int> cache;
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_tuple(kern, cta, smem);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, cta, smem) != cudaSuccess ||
        occ < 1)
        occ = 1;
    cache[key] = occ;
    return occ;
}

// persistent grid: enough blocks to give every chunk a tile, at most what
// fits on the GPU at once
inline int grid_blocks(const void *kern, int T, const LaunchParams &lp, uint64_t n, size_t smem) {
    const uint64_t per = (uint64_t)T * lp.items;
    uint64_t chunks = (n + per - 1) / per;
    if (lp.max_tiles > 0 && chunks > (uint64_t)lp.max_tiles) chunks = lp.max_tiles;
    const uint64_t tiles_per_block = lp.cta / T;
    uint64_t need = (chunks + tiles_per_block - 1) / tiles_per_block;
    uint64_t cap = (uint64_t)lp.sms * occupancy(kern, lp.cta, smem);
    if (lp.max_ctas > 0 && cap > (uint64_t)lp.max_ctas) cap = lp.max_ctas;
    uint64_t b = need < cap ? need : cap;
    return b < 1 ? 1 : (int)b;
}

// persistent grid for kernels that give each warp 32 keys at a time
inline int grid_blocks_warp(const void *kern, const LaunchParams &lp, uint64_t n) {
    const uint64_t warps = (n + 31) / 32;
    const uint64_t per_block = lp.cta / 32;
    uint64_t need = (warps + per_block - 1) / per_block;
    uint64_t cap = (uint64_t)lp.sms * occupancy(kern, lp.cta, 0);
    if (lp.max_ctas > 0 && cap > (uint64_t)lp.max_ctas) cap = lp.max_ctas;
    uint64_t b = need < cap ? need : cap;
    return b < 1 ? 1 : (int)b;
}

cudaError_t launch_values(bool scatter, const uint64_t *slots, uint64_t n, const void *src,
                          void *dst, int value_bytes, uint64_t nslots, int sms,
                          cudaStream_t stream);
cudaError_t launch_random_claim(void *buf, size_t buf_bytes, uint64_t n_lines, uint64_t seed,
                                unsigned long long *sink, int sms, cudaStream_t stream);
cudaError_t launch_random_read(const void *buf, size_t buf_bytes, int block_bytes,
                               uint64_t n_blocks, uint64_t seed, unsigned long long *sink,
                               int sms, cudaStream_t stream);
cudaError_t launch_cuckoo_insert(int T, int fpw, const LaunchParams &lp, const TableArgs &ta,
                                 const void *keys, uint64_t n, uint8_t *status,
                                 uint64_t *dropped);
cudaError_t launch_cuckoo_find(int T, int fpw, const LaunchParams &lp, const TableArgs &ta,
                               const void *keys, uint64_t n, uint8_t *status);
// slots (nullable): per-key slot index output of iceberg operations; kv
// (nullable): value moves of the key-value extension
cudaError_t launch_iceberg(int T, int fpw0, bool lookup, const LaunchParams &lp,
                           const TableArgs &ta, const void *keys, uint64_t n, uint8_t *status,
                           uint64_t *slots = nullptr, const KVArgs *kv = nullptr);
cudaError_t launch_iceberg_warp(int T, int fpw0, bool lookup, const LaunchParams &lp,
                                const TableArgs &ta, const void *keys, uint64_t n,
                                uint8_t *status, uint64_t *slots = nullptr,
                                const KVArgs *kv = nullptr);
// the warp-batched engine with slot outputs and value moves (one key per lane)
cudaError_t launch_iceberg_warp_slots(int T, int fpw0, bool lookup, const LaunchParams &lp,
                                      const TableArgs &ta, const void *keys, uint64_t n,
                                      uint8_t *status, uint64_t *slots, const KVArgs &kv);

// tables with 32- or 64-byte buckets (wpb = 4 or 8 words): one launcher for
// the four operations, tiles of wpb / 2 lanes
enum SmallOp { kSmallCuckooInsert, kSmallCuckooFind, kSmallIcebergFop, kSmallIcebergFind };
cudaError_t launch_small_buckets(int op, int wpb, int fpw, const LaunchParams &lp,
                                 const TableArgs &ta, const void *keys, uint64_t n,
                                 uint8_t *status, uint64_t *dropped);

struct BatchDesc;
// launch shape of the allocation-free fused find-or-put
constexpr int kStaticBatchTile = 4;
constexpr int kStaticBatchItems = 1;
// keys per lane of the warp-batched engine for an items_per_thread setting:
// 1, 2 or 4 (a warp takes chunks of 32 * I keys of one table)
inline int batch_items(int items) { return items >= 4 ? 4 : (items >= 2 ? 2 : 1); }
cudaError_t launch_iceberg_batch(int T, int fpw0, bool lookup, const LaunchParams &lp,
                                 const BatchDesc *bd, int count, uint64_t total_chunks,
                                 unsigned long long *ctr);
cudaError_t launch_iceberg_batch_noalloc(int fpw0, cudaStream_t s, int sms, const BatchDesc *bd,
                                         int count, uint64_t total_chunks);

}  // namespace cht
