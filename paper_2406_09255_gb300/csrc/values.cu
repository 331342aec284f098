// Value array moves for the key-value extension: values live in a caller
// array indexed by the stable slot of their key (iceberg tables), so a put is
// find-or-put plus a scatter to the returned slots and a get is a lookup plus
// a gather from them.
#include <cstdint>
#include <cuda_runtime.h>

#include "cht_launch.h"

namespace cht {

template <typename V>
__global__ void __launch_bounds__(256)
    k_values_scatter(const uint64_t *__restrict__ slots, uint64_t n, const V *__restrict__ vals,
                     V *__restrict__ store, uint64_t nslots) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t s = slots[i];
        if (s < nslots) store[s] = vals[i];
    }
}

template <typename V>
__global__ void __launch_bounds__(256)
    k_values_gather(const uint64_t *__restrict__ slots, uint64_t n, const V *__restrict__ store,
                    V *__restrict__ out, uint64_t nslots) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t s = slots[i];
        V v{};
        if (s < nslots) v = store[s];
        out[i] = v;
    }
}

static int blocks_for(uint64_t n, int sms) {
    const uint64_t need = (n + 255) / 256;
    const uint64_t cap = (uint64_t)sms * 8;
    return (int)(need < cap ? (need ? need : 1) : cap);
}

cudaError_t launch_values(bool scatter, const uint64_t *slots, uint64_t n, const void *src,
                          void *dst, int value_bytes, uint64_t nslots, int sms,
                          cudaStream_t stream) {
    const int b = blocks_for(n, sms);
    switch (value_bytes) {
        case 4:
            if (scatter)
                k_values_scatter<uint32_t><<<b, 256, 0, stream>>>(
                    slots, n, static_cast<const uint32_t *>(src), static_cast<uint32_t *>(dst), nslots);
            else
                k_values_gather<uint32_t><<<b, 256, 0, stream>>>(
                    slots, n, static_cast<const uint32_t *>(src), static_cast<uint32_t *>(dst), nslots);
            break;
        case 8:
            if (scatter)
                k_values_scatter<uint64_t><<<b, 256, 0, stream>>>(
                    slots, n, static_cast<const uint64_t *>(src), static_cast<uint64_t *>(dst), nslots);
            else
                k_values_gather<uint64_t><<<b, 256, 0, stream>>>(
                    slots, n, static_cast<const uint64_t *>(src), static_cast<uint64_t *>(dst), nslots);
            break;
        case 16:
            if (scatter)
                k_values_scatter<ulonglong2><<<b, 256, 0, stream>>>(
                    slots, n, static_cast<const ulonglong2 *>(src), static_cast<ulonglong2 *>(dst), nslots);
            else
                k_values_gather<ulonglong2><<<b, 256, 0, stream>>>(
                    slots, n, static_cast<const ulonglong2 *>(src), static_cast<ulonglong2 *>(dst), nslots);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace cht
