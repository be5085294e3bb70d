// Device-side block copy shared by the copy engine and the batched plan.
#pragma once
#include <stdint.h>

namespace phos {

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

template <typename T>
__device__ __forceinline__ void copy_units(uint8_t *dst, const uint8_t *src, uint64_t nunits) {
    const T *s = reinterpret_cast<const T *>(src);
    T *d = reinterpret_cast<T *>(dst);
    const uint64_t stride = blockDim.x;
    uint64_t i = threadIdx.x;
    for (; i + 3 * stride < nunits; i += 4 * stride) {
        T v0 = s[i], v1 = s[i + stride], v2 = s[i + 2 * stride], v3 = s[i + 3 * stride];
        d[i] = v0;
        d[i + stride] = v1;
        d[i + 2 * stride] = v2;
        d[i + 3 * stride] = v3;
    }
    for (; i < nunits; i += stride) d[i] = s[i];
}

// Bytes K .. K+15 of the 32-byte little-endian concatenation a|b.
template <uint32_t K>
__device__ __forceinline__ uint4 bytes_from(uint4 a, uint4 b) {
    constexpr uint32_t q = K >> 2, r = (K & 3) * 8;
    const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    if constexpr (r == 0) {
        return make_uint4(w[q], w[q + 1], w[q + 2], w[q + 3]);
    } else {
        return make_uint4(__funnelshift_r(w[q], w[q + 1], r), __funnelshift_r(w[q + 1], w[q + 2], r),
                          __funnelshift_r(w[q + 2], w[q + 3], r),
                          __funnelshift_r(w[q + 3], w[q + 4], r));
    }
}

// nvec 16-byte vectors to a 16-byte aligned dst from a src that is K bytes
// past a 16-byte boundary (0 < K < 16).  Each lane loads one aligned source
// vector and takes the words it needs of the next one from its neighbour
// lane (lane 31 from lane 0's vector of the next chunk), so every source
// vector is loaded once, plus one per 128 that lane 0 loads ahead; an
// aligned vector that holds at least one byte of the region never leaves
// the region's allocation.  Four 32-vector chunks in flight per warp.
template <uint32_t K>
__device__ __forceinline__ void copy_shifted(uint8_t *dst, const uint8_t *src, uint64_t nvec) {
    constexpr uint32_t nb = (K >> 2) + ((K & 3) ? 1 : 0);   // words of the next vector used
    const uint4 *s = reinterpret_cast<const uint4 *>(src - K);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t from = (lane + 1) & 31;
    const uint64_t warps = blockDim.x >> 5;
    const uint64_t w = threadIdx.x >> 5;
    const uint4 z = make_uint4(0, 0, 0, 0);
    for (uint64_t v0 = w * 128; v0 < nvec; v0 += warps * 128) {
        uint4 a[5];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t i = v0 + 32 * u + lane;
            a[u] = i <= nvec ? __ldcs(s + i) : z;
        }
        a[4] = (lane == 0 && v0 + 128 <= nvec) ? __ldcs(s + v0 + 128) : z;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t i = v0 + 32 * u + lane;
            const uint4 nx = lane == 0 ? a[u + 1] : a[u];   // what lane - 1 reads here
            uint4 b = z;
            b.x = __shfl_sync(0xffffffffu, nx.x, from);
            if constexpr (nb > 1) b.y = __shfl_sync(0xffffffffu, nx.y, from);
            if constexpr (nb > 2) b.z = __shfl_sync(0xffffffffu, nx.z, from);
            if constexpr (nb > 3) b.w = __shfl_sync(0xffffffffu, nx.w, from);
            if (i < nvec) __stcs(d + i, bytes_from<K>(a[u], b));
        }
    }
}

__device__ __forceinline__ void copy_block(uint8_t *dst, const uint8_t *src, uint64_t len) {
    if ((((uintptr_t)src ^ (uintptr_t)dst) & 15) == 0) {
        // common 16-byte alignment: byte head, 16-byte vectors, byte tail
        const uint64_t head = min(len, (uint64_t)((16 - ((uintptr_t)src & 15)) & 15));
        for (uint64_t i = threadIdx.x; i < head; i += blockDim.x) dst[i] = src[i];
        const uint64_t body = (len - head) / 16;
        copy_vec16(dst + head, src + head, body);
        for (uint64_t i = head + body * 16 + threadIdx.x; i < len; i += blockDim.x)
            dst[i] = src[i];
        return;
    }
    if ((((uintptr_t)src ^ (uintptr_t)dst) & 7) == 0) {
        // common 8-byte alignment: 8-byte units
        const uint64_t head = min(len, (uint64_t)((8 - ((uintptr_t)src & 7)) & 7));
        for (uint64_t i = threadIdx.x; i < head; i += blockDim.x) dst[i] = src[i];
        const uint64_t body = (len - head) / 8;
        copy_units<uint64_t>(dst + head, src + head, body);
        for (uint64_t i = head + body * 8 + threadIdx.x; i < len; i += blockDim.x)
            dst[i] = src[i];
        return;
    }
    // otherwise: bytes up to a 16-byte boundary of dst, then aligned 16-byte
    // stores whose bytes come out of two aligned source vectors, then the
    // byte tail
    const uint64_t head = min(len, (uint64_t)((16 - ((uintptr_t)dst & 15)) & 15));
    for (uint64_t i = threadIdx.x; i < head; i += blockDim.x) dst[i] = src[i];
    const uint64_t body = (len - head) / 16;
    const uint8_t *s = src + head;
    uint8_t *d = dst + head;
    if (body) {
        switch ((uintptr_t)s & 15) {
            case 1: copy_shifted<1>(d, s, body); break;
            case 2: copy_shifted<2>(d, s, body); break;
            case 3: copy_shifted<3>(d, s, body); break;
            case 4: copy_shifted<4>(d, s, body); break;
            case 5: copy_shifted<5>(d, s, body); break;
            case 6: copy_shifted<6>(d, s, body); break;
            case 7: copy_shifted<7>(d, s, body); break;
            case 9: copy_shifted<9>(d, s, body); break;
            case 10: copy_shifted<10>(d, s, body); break;
            case 11: copy_shifted<11>(d, s, body); break;
            case 12: copy_shifted<12>(d, s, body); break;
            case 13: copy_shifted<13>(d, s, body); break;
            case 14: copy_shifted<14>(d, s, body); break;
            default: copy_shifted<15>(d, s, body); break;
        }
    }
    for (uint64_t i = head + body * 16 + threadIdx.x; i < len; i += blockDim.x) dst[i] = src[i];
}

}  // namespace phos
