// Device-side block copy shared by the copy engine and the batched plan.
#pragma once
#include <stdint.h>

namespace phos {

// Copy len bytes with the whole CTA, using unit-sized accesses on a
// region whose src and dst are both unit-aligned.
template <typename U>
__device__ __forceinline__ void copy_units(uint8_t *dst, const uint8_t *src, uint64_t nunits) {
    const U *s = reinterpret_cast<const U *>(src);
    U *d = reinterpret_cast<U *>(dst);
    const uint64_t stride = blockDim.x;
    uint64_t i = threadIdx.x;
    for (; i + 3 * stride < nunits; i += 4 * stride) {
        U v0 = s[i], v1 = s[i + stride], v2 = s[i + 2 * stride], v3 = s[i + 3 * stride];
        d[i] = v0;
        d[i + stride] = v1;
        d[i + 2 * stride] = v2;
        d[i + 3 * stride] = v3;
    }
    for (; i < nunits; i += stride) d[i] = s[i];
}

__device__ __forceinline__ void copy_vec16(uint8_t *dst, const uint8_t *src, uint64_t nvec) {
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    const uint64_t stride = blockDim.x;
    uint64_t i = threadIdx.x;
    for (; i + 3 * stride < nvec; i += 4 * stride) {
        uint4 v0 = __ldcs(s + i), v1 = __ldcs(s + i + stride), v2 = __ldcs(s + i + 2 * stride),
              v3 = __ldcs(s + i + 3 * stride);
        __stcs(d + i, v0);
        __stcs(d + i + stride, v1);
        __stcs(d + i + 2 * stride, v2);
        __stcs(d + i + 3 * stride, v3);
    }
    for (; i < nvec; i += stride) __stcs(d + i, __ldcs(s + i));
}

__device__ __forceinline__ void copy_block(uint8_t *dst, const uint8_t *src, uint64_t len) {
    const uint64_t x = ((uintptr_t)src ^ (uintptr_t)dst) | 16;
    const uint32_t unit = (uint32_t)(x & (~x + 1));  // lowest set bit, <= 16
    const uint64_t head = min(len, (uint64_t)((unit - ((uintptr_t)src & (unit - 1))) & (unit - 1)));
    for (uint64_t i = threadIdx.x; i < head; i += blockDim.x) dst[i] = src[i];
    const uint64_t body = (len - head) / unit;
    uint8_t *d = dst + head;
    const uint8_t *s = src + head;
    switch (unit) {
        case 16: copy_vec16(d, s, body); break;
        case 8: copy_units<uint64_t>(d, s, body); break;
        case 4: copy_units<uint32_t>(d, s, body); break;
        case 2: copy_units<uint16_t>(d, s, body); break;
        default: copy_units<uint8_t>(d, s, body); break;
    }
    const uint64_t done = head + body * unit;
    for (uint64_t i = done + threadIdx.x; i < len; i += blockDim.x) dst[i] = src[i];
}

}  // namespace phos
