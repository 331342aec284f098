// Random-access rates of this GPU's memory: the ceilings that bound every
// probe of the tables (one bucket read at a data-dependent address) and every
// put (a read, then a compare-and-swap into the same line). Each tile of
// lanes reads whole blocks at splitmix-chosen positions, four blocks in
// flight per tile, one vector load per lane per block, and folds the data
// into one word so that the loads cannot be dropped.
#include <cstdint>
#include <cuda_runtime.h>

#include "cht_device.cuh"
#include "cht_launch.h"

namespace cht {

template <int LANES, int BPL>
__global__ void __launch_bounds__(256)
    k_random_read(const uint64_t *__restrict__ buf, uint64_t blocks_mask, uint64_t n_blocks,
                  uint64_t seed, unsigned long long *__restrict__ sink) {
    constexpr int BW = LANES * BPL / 8;  // words per block
    constexpr int U = 4;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t tile = tid / LANES;
    const uint64_t ntiles = (uint64_t)gridDim.x * blockDim.x / LANES;
    const int tl = (int)(threadIdx.x % LANES);
    uint64_t acc = 0;
    for (uint64_t i0 = tile * U; i0 < n_blocks; i0 += ntiles * U) {
        uint64_t v[U][4];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool on = i0 + u < n_blocks;
            const uint64_t blk = mix64(seed + (i0 + u) * kGamma) & blocks_mask;
            const uint64_t *p = buf + blk * BW + tl * (BPL / 8);
            v[u][0] = v[u][1] = v[u][2] = v[u][3] = 0;
            if (on) {
                if constexpr (BPL == 16) {
                    asm volatile("ld.global.nc.L1::no_allocate.v2.u64 {%0, %1}, [%2];"
                                 : "=l"(v[u][0]), "=l"(v[u][1])
                                 : "l"(p));
                } else {
                    asm volatile("ld.global.nc.L1::no_allocate.v4.u64 {%0, %1, %2, %3}, [%4];"
                                 : "=l"(v[u][0]), "=l"(v[u][1]), "=l"(v[u][2]), "=l"(v[u][3])
                                 : "l"(p));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) acc ^= v[u][0] + v[u][1] + v[u][2] + v[u][3];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicXor(sink, (unsigned long long)acc);
}

// The access pattern of a put: read a random 128-byte line (eight lanes,
// one 16-byte relaxed load each, four lines in flight per tile), then
// compare-and-swap one 64-bit word of it with the value just read (the lane
// that owns the word; expected = the snapshot, as a claim does), all four
// compare-and-swaps issued before any result is read. Every line it touches
// is read once and dirtied once, so its rate is the ceiling for puts that
// claim a slot in the first bucket they probe.
__global__ void __launch_bounds__(256)
    k_random_claim(uint64_t *__restrict__ buf, uint64_t lines_mask, uint64_t n_lines,
                   uint64_t seed, unsigned long long *__restrict__ sink) {
    constexpr int U = 4;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t tile = tid / 8;
    const uint64_t ntiles = (uint64_t)gridDim.x * blockDim.x / 8;
    const int tl = (int)(threadIdx.x % 8);
    uint64_t acc = 0;
    for (uint64_t i0 = tile * U; i0 < n_lines; i0 += ntiles * U) {
        uint64_t v[U][2];
        uint64_t *p[U];
        bool on[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            on[u] = i0 + u < n_lines;
            const uint64_t h = mix64(seed + (i0 + u) * kGamma);
            p[u] = buf + (h & lines_mask) * 16 + tl * 2;
            v[u][0] = v[u][1] = 0;
            if (on[u])
                asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];"
                             : "=l"(v[u][0]), "=l"(v[u][1])
                             : "l"(p[u])
                             : "memory");
        }
        // the word to claim: one of the line's 16, chosen from the hash
        unsigned long long old[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t h = mix64(seed + (i0 + u) * kGamma);
            const int word = (int)((h >> 40) & 15);
            old[u] = 0;
            if (on[u] && tl == word / 2) {
                const uint64_t snap = (word & 1) ? v[u][1] : v[u][0];
                old[u] = atomicCAS(reinterpret_cast<unsigned long long *>(p[u] + (word & 1)),
                                   (unsigned long long)snap, (unsigned long long)(snap + 1));
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) acc ^= old[u] + v[u][0] + v[u][1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicXor(sink, (unsigned long long)acc);
}

cudaError_t launch_random_claim(void *buf, size_t buf_bytes, uint64_t n_lines, uint64_t seed,
                                unsigned long long *sink, int sms, cudaStream_t stream) {
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_random_claim, 256, 0);
    if (e != cudaSuccess) return e;
    k_random_claim<<<sms * (occ > 0 ? occ : 1), 256, 0, stream>>>(
        static_cast<uint64_t *>(buf), buf_bytes / 128 - 1, n_lines, seed, sink);
    return cudaGetLastError();
}

template <int LANES, int BPL>
static cudaError_t run(const void *buf, uint64_t nblk, uint64_t n_blocks, uint64_t seed,
                       unsigned long long *sink, int sms, cudaStream_t stream) {
    auto kern = k_random_read<LANES, BPL>;
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, 0);
    if (e != cudaSuccess) return e;
    kern<<<sms * (occ > 0 ? occ : 1), 256, 0, stream>>>(static_cast<const uint64_t *>(buf),
                                                         nblk - 1, n_blocks, seed, sink);
    return cudaGetLastError();
}

cudaError_t launch_random_read(const void *buf, size_t buf_bytes, int block_bytes,
                               uint64_t n_blocks, uint64_t seed, unsigned long long *sink,
                               int sms, cudaStream_t stream) {
    const uint64_t nblk = buf_bytes / (uint64_t)block_bytes;
    switch (block_bytes) {
        case 32: return run<2, 16>(buf, nblk, n_blocks, seed, sink, sms, stream);
        case 64: return run<4, 16>(buf, nblk, n_blocks, seed, sink, sms, stream);
        case 128: return run<8, 16>(buf, nblk, n_blocks, seed, sink, sms, stream);
        case 256: return run<8, 32>(buf, nblk, n_blocks, seed, sink, sms, stream);
    }
    return cudaErrorInvalidValue;
}

}  // namespace cht
