// keygen.cu - device generator of the served benchmark's request keys.
//
// Input generation only: none of the hash tables' arithmetic is here. Key
// number i of a table's sequence is G_s(i'), a 4-round balanced Feistel
// bijection on w-bit integers (cycle-walking for odd w) whose round function
// is the splitmix64 finaliser (Steele, Lea and Flood 2014), with i' = i + 1
// for i at or past the one index that maps to 0. This is the definition the
// package's workloads module implements with torch; the two must agree bit
// for bit (a test checks it). A request's keys are n_fresh keys at
// consecutive indices from fresh_base, then n - n_fresh re-queries at indices
// floor(h * re_hi / 2^64) with h = splitmix64(re_seed, j) for the j-th
// re-query, or, when re_hi is 0, at consecutive indices from miss_base.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

struct GenReq {
    unsigned long long out_off;     // first output position of the request
    unsigned long long n;           // keys of the request
    unsigned long long n_fresh;     // leading keys at consecutive indices
    unsigned long long fresh_base;  // their first index
    unsigned long long re_hi;       // re-queries: indices uniform in [0, re_hi)
    unsigned long long re_seed;
    unsigned long long miss_base;   // when re_hi == 0: consecutive indices from here
    unsigned long long rk[4];       // round keys of the table's key sequence
    unsigned long long skip;        // the index whose image is 0 (skipped)
    int key_bits;
    int pad;
};

constexpr int kReqPerLaunch = 128;
struct GenBlock {
    GenReq r[kReqPerLaunch];
};

constexpr unsigned long long kGamma = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ unsigned long long mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long feistel(unsigned long long x, int bits,
                                                      const unsigned long long (&rk)[4]) {
    const int h = bits / 2;
    const unsigned long long m = (1ull << h) - 1ull;
    unsigned long long L = x >> h, R = x & m;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const unsigned long long nl = R;
        R = L ^ (mix(R + rk[r]) & m);
        L = nl;
    }
    return (L << h) | R;
}

__global__ void __launch_bounds__(256)
    k_request_keys(GenBlock blk, int count, unsigned long long total,
                   unsigned long long *__restrict__ out) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long p = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
         p < total; p += stride) {
        // the request holding output position p (offsets ascend)
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (blk.r[mid].out_off <= p)
                lo = mid;
            else
                hi = mid - 1;
        }
        const GenReq &q = blk.r[lo];
        const unsigned long long i = p - q.out_off;
        if (i >= q.n) continue;  // a gap between requests: nothing to write
        unsigned long long idx;
        if (i < q.n_fresh) {
            idx = q.fresh_base + i;
        } else if (q.re_hi) {
            idx = __umul64hi(mix(q.re_seed + (i - q.n_fresh + 1) * kGamma), q.re_hi);
        } else {
            idx = q.miss_base + (i - q.n_fresh);
        }
        idx += idx >= q.skip ? 1ull : 0ull;
        const int w = q.key_bits;
        const int bits = w + (w & 1);
        unsigned long long y = feistel(idx, bits, q.rk);
        while (y >> w) y = feistel(y, bits, q.rk);  // cycle-walk for odd w
        out[p] = y;
    }
}

}  // namespace

extern "C" {

// Bytes of one request descriptor (the binding checks its layout).
int keygen_req_bytes(void) { return (int)sizeof(GenReq); }
int keygen_req_per_launch(void) { return kReqPerLaunch; }

// Write the keys of count requests (descriptors in host memory, out_off
// ascending) into d_out (total positions, device int64), on stream. Returns
// 0 or a CUDA error code.
int keygen_request_keys(const void *reqs, int count, unsigned long long total, void *d_out,
                        int sms, void *stream) {
    if (count < 1 || count > kReqPerLaunch || !reqs || !d_out) return (int)cudaErrorInvalidValue;
    GenBlock blk;
    const GenReq *r = static_cast<const GenReq *>(reqs);
    for (int i = 0; i < count; ++i) blk.r[i] = r[i];
    unsigned long long blocks = (total + 255) / 256;
    const unsigned long long cap = (unsigned long long)(sms > 0 ? sms : 1) * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_request_keys<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        blk, count, total, static_cast<unsigned long long *>(d_out));
    return (int)cudaGetLastError();
}

}  // extern "C"
