// cht_scan.cuh - whole-table streaming kernels: enumerate (decode every
// stored key) and clear. Included by the C ABI unit only.
#pragma once

#include "cht_kernels.cuh"

namespace cht {

// ===========================================================================
// Enumerate: decode every stored entry, k = pi_j^-1(a . r) (Section 2.4), and
// append it to the output. A streaming pass over the table: each thread reads
// 16 bytes, the warp reserves output space with one atomic.
// ===========================================================================
__device__ __forceinline__ uint64_t decode_entry(const TableArgs &ta, int kind, int level,
                                                 uint64_t a, uint64_t e) {
    const Level &L = ta.lv[level];
    if (kind == 0 || level == 1) {
        // cuckoo (r, j) or iceberg secondary (r, i): two tag bits
        const int j = (int)(e & 3) - 1;
        return ta.compact ? unquotient(L, j, a, e >> 2) : (e >> 2);
    }
    return ta.compact ? unquotient(L, 0, a, e >> 1) : (e >> 1);
}

__global__ void __launch_bounds__(256)
    k_enumerate(TableArgs ta, int kind, void *__restrict__ out, uint64_t cap,
                unsigned long long *__restrict__ count) {
    const uint64_t w0 = ta.lv[0].nb * (uint64_t)ta.wpb;
    const uint64_t w1 = (kind == 1) ? ta.lv[1].nb * (uint64_t)ta.wpb : 0;
    // the iceberg stash: whole keys after level 1, its storage rounded up
    // to whole 128-byte lines (the padding words stay zero)
    const uint64_t ws = (kind == 1) ? (ta.stash_slots + 15) / 16 * 16 : 0;
    const uint64_t npairs = (w0 + w1 + ws) / 2;  // every region holds an even word count
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < npairs; base += stride) {
        const uint64_t p = base + threadIdx.x;
        uint64_t key[8];
        int cnt = 0;
        if (p < npairs && 2 * p >= w0 + w1) {
            // a stash pair: each nonzero word is a stored key
            const ulonglong2 x = __ldcs(reinterpret_cast<const ulonglong2 *>(
                ta.lv[1].words + (2 * p - w0)));
            if (x.x) key[cnt++] = x.x;
            if (x.y) key[cnt++] = x.y;
        } else if (p < npairs) {
            const uint64_t wi = 2 * p;
            const int level = wi < w0 ? 0 : 1;
            const uint64_t lw = level ? wi - w0 : wi;
            const uint64_t *src = ta.lv[level].words + lw;
            const ulonglong2 x = __ldcs(reinterpret_cast<const ulonglong2 *>(src));
            const uint64_t a = lw / (uint64_t)ta.wpb;
            const int fpw = ta.lv[level].fpw;
            const int S = 64 / fpw;
            const uint64_t M = (S >= 64) ? ~0ull : ((1ull << S) - 1ull);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint64_t word = h ? x.y : x.x;
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    if (f < fpw) {
                        const uint64_t e = (word >> (f * S)) & M;
                        if (e) key[cnt++] = decode_entry(ta, kind, level, a, e);
                    }
                }
            }
        }
        // warp prefix sum of counts, one atomic per warp
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long wbase = 0;
        if (lane == 31 && total) wbase = atomicAdd(count, (unsigned long long)total);
        wbase = __shfl_sync(0xffffffffu, wbase, 31);
        uint64_t pos = wbase + (uint64_t)(incl - cnt);
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (i < cnt && pos + i < cap) store_key(out, ta.key_bytes, pos + i, key[i]);
    }
}

__global__ void k_zero_u64(unsigned long long *p) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *p = 0ull;
}

// zero the storage (header and both levels) of every table of a batch: the
// whole grid sweeps one table after another
__global__ void __launch_bounds__(256) k_clear_batch(const BatchDesc *__restrict__ bd, int count) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (int t = 0; t < count; ++t) {
        const TableArgs &ta = bd[t].ta;
        ulonglong2 *p = reinterpret_cast<ulonglong2 *>(ta.err);  // header start
        const uint64_t nb = ta.lv[0].nb + ta.lv[1].nb;  // lv[1].nb is 0 for cuckoo
        const uint64_t stash_bytes = (ta.stash_slots + 15) / 16 * 128;
        const uint64_t n16 = (256 + nb * 8 * (uint64_t)ta.wpb + stash_bytes) / 16;
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride)
            __stcs(p + i, make_ulonglong2(0ull, 0ull));
    }
}

// batch descriptors carried to the device as kernel parameters: the upload is
// then an ordinary asynchronous launch, with no host buffer to keep alive
constexpr int kDescPerLaunch = 64;
struct DescBlock {
    BatchDesc d[kDescPerLaunch];
};
__global__ void __launch_bounds__(128) k_write_desc(BatchDesc *__restrict__ dst, DescBlock blk,
                                                    int count) {
    const uint64_t *src = reinterpret_cast<const uint64_t *>(blk.d);
    uint64_t *out = reinterpret_cast<uint64_t *>(dst);
    const int words = count * (int)(sizeof(BatchDesc) / 8);
    for (int i = threadIdx.x; i < words; i += blockDim.x) out[i] = src[i];
}

// zero n16 16-byte units starting at p (16-byte aligned)
__global__ void __launch_bounds__(256) k_clear(ulonglong2 *p, uint64_t n16) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride)
        __stcs(p + i, make_ulonglong2(0ull, 0ull));
}

}  // namespace cht
