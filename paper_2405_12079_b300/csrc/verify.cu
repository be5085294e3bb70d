// Image integrity for restore (the failure list of a C/R system includes a
// checkpoint image that comes back corrupted or truncated; PhoenixOS Sec. 7
// restores the latest checkpoint after a failure, so a damaged one must be
// caught, not replayed).  A manifest holds one 64-bit digest per buffer of
// the image (the order-independent digest of include/phos_harness.h);
// phos_image_manifest computes it over an image, and a restore session
// given one digests every buffer on the device the moment its last byte
// lands in live memory, before any kernel can touch it, and compares.
//
// The digest is a sum of per-word terms mod 2^64, so CTAs take 256 KiB
// tiles of any buffer and add their partial sums with one 64-bit atomic
// each; in a verification the last tile of a buffer (a per-buffer tile
// counter) compares the sum with the manifest and resets both words, so a
// buffer restored again (a rollback) is verified again.
#include <limits.h>

#include <algorithm>
#include <vector>

#include "digest_dev.cuh"
#include "internal.h"

namespace phos {

constexpr uint64_t kVTile = 256 * 1024;
// Regions per launch: a batch travels as the kernel's parameters, 64
// regions (2 KB) for the short lists of a restore's sub-batches, 1,000
// (32 KB, near the 32,764-byte parameter limit) for a whole table, so a
// table of up to 1,000 buffers is one launch whose tiles spread over the
// whole grid (with 64 regions per launch a 2 GB manifest took 17 thin
// launches and 0.65 ms).
constexpr int kVSmall = 64;
constexpr int kVLarge = 1000;

struct VEnt {
    uint64_t ptr, len;
    uint32_t tile0, tiles, buf, pad;
};

template <int N>
struct VBatch {
    VEnt e[N];
    uint32_t count, tiles;
};
static_assert(sizeof(VBatch<kVLarge>) + 5 * sizeof(void *) <= 32764,
              "k_verify's parameters exceed the launch limit");

template <int N>
__global__ void __launch_bounds__(512) k_verify(const __grid_constant__ VBatch<N> b,
                                                unsigned long long *acc, uint32_t *cnt,
                                                const uint64_t *manifest, uint32_t *status,
                                                int *bad) {
    __shared__ unsigned long long s_acc;
    if (threadIdx.x == 0) s_acc = 0;
    __syncthreads();
    for (uint32_t t = blockIdx.x; t < b.tiles; t += gridDim.x) {
        // the entry holding tile t: the last one whose first tile is <= t
        int lo = 0, hi = (int)b.count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (b.e[mid].tile0 <= t)
                lo = mid;
            else
                hi = mid - 1;
        }
        const VEnt &e = b.e[lo];
        const uint64_t off = (uint64_t)(t - e.tile0) * kVTile;
        const uint64_t end = min(off + kVTile, e.len);
        const unsigned long long part = digest_range(reinterpret_cast<const uint8_t *>(e.ptr),
                                                     e.len, off, end);
        if ((threadIdx.x & 31) == 0 && part) atomicAdd(&s_acc, part);
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned long long v = s_acc;
            s_acc = 0;
            if (v) atomicAdd(acc + e.buf, v);
            if (manifest) {
                __threadfence();
                if (atomicAdd(cnt + e.buf, 1u) == e.tiles - 1) {
                    // every tile of this buffer has added its part
                    __threadfence();
                    const unsigned long long d = atomicAdd(acc + e.buf, 0ull);
                    if (d != (unsigned long long)manifest[e.buf]) {
                        atomicCAS(status, 0u, (uint32_t)PHOS_ECORRUPT);
                        atomicMin(bad, (int)e.buf);
                    }
                    acc[e.buf] = 0;
                    cnt[e.buf] = 0;
                }
            }
        }
        __syncthreads();
    }
}

__global__ void k_vzero(unsigned long long *p, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        p[i] = 0;
}

// Digest regions [ptrs[k], +lens[k]) into acc[bufs[k]] (manifest == NULL),
// or verify them against manifest[bufs[k]] (see k_verify).
template <int N>
static phos_status digest_regions_n(const std::vector<uint64_t> &ptrs,
                                    const std::vector<uint64_t> &lens,
                                    const std::vector<uint32_t> &bufs, unsigned long long *acc,
                                    uint32_t *cnt, const uint64_t *manifest, uint32_t *status,
                                    int *bad, cudaStream_t s) {
    for (size_t b0 = 0; b0 < ptrs.size(); b0 += N) {
        VBatch<N> b;
        memset(&b, 0, sizeof b);
        uint32_t tiles = 0;
        b.count = (uint32_t)std::min<size_t>(N, ptrs.size() - b0);
        for (uint32_t q = 0; q < b.count; ++q) {
            VEnt &e = b.e[q];
            e.ptr = ptrs[b0 + q];
            e.len = lens[b0 + q];
            e.buf = bufs[b0 + q];
            e.tile0 = tiles;
            e.tiles = (uint32_t)std::max<uint64_t>(1, (e.len + kVTile - 1) / kVTile);
            tiles += e.tiles;
        }
        b.tiles = tiles;
        const unsigned grid = (unsigned)std::max<uint32_t>(1, std::min<uint32_t>(tiles, 148 * 4));
        k_verify<N><<<grid, 512, 0, s>>>(b, acc, cnt, manifest, status, bad);
        count_launch();
        PHOS_CUDA(cudaGetLastError());
    }
    return PHOS_OK;
}

static phos_status digest_regions(const std::vector<uint64_t> &ptrs,
                                  const std::vector<uint64_t> &lens,
                                  const std::vector<uint32_t> &bufs, unsigned long long *acc,
                                  uint32_t *cnt, const uint64_t *manifest, uint32_t *status,
                                  int *bad, cudaStream_t s) {
    if (ptrs.size() <= (size_t)kVSmall)
        return digest_regions_n<kVSmall>(ptrs, lens, bufs, acc, cnt, manifest, status, bad, s);
    return digest_regions_n<kVLarge>(ptrs, lens, bufs, acc, cnt, manifest, status, bad, s);
}

phos_status verify_buffers(const phos_table *t, const std::vector<uint32_t> &bufs,
                           const uint64_t *d_manifest, unsigned long long *d_acc,
                           uint32_t *d_cnt, uint32_t *d_status, int *d_bad, cudaStream_t s) {
    if (bufs.empty()) return PHOS_OK;
    std::vector<uint64_t> ptrs(bufs.size()), lens(bufs.size());
    for (size_t k = 0; k < bufs.size(); ++k) {
        ptrs[k] = t->base[bufs[k]];
        lens[k] = t->size[bufs[k]];
    }
    return digest_regions(ptrs, lens, bufs, d_acc, d_cnt, d_manifest, d_status, d_bad, s);
}

}  // namespace phos

using namespace phos;

extern "C" phos_status phos_image_manifest(const phos_table_t *t, const void *image,
                                           uint64_t image_bytes, uint64_t *d_digest,
                                           phos_stream_t stream) {
    if (!t || !d_digest || (!image && t->n)) return fail(PHOS_EINVAL, "image_manifest: NULL argument");
    if (image_bytes < t->image_bytes)
        return fail(PHOS_ECORRUPT, "image_manifest: image truncated (%llu of %llu bytes)",
                    (unsigned long long)image_bytes, (unsigned long long)t->image_bytes);
    if (!t->n) return PHOS_OK;
    void *dv = nullptr;
    phos_status r = device_view(image, &dv);
    if (r) return r;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long *out = reinterpret_cast<unsigned long long *>(d_digest);
    k_vzero<<<(t->n + 255) / 256, 256, 0, s>>>(out, t->n);
    count_launch();
    PHOS_CUDA(cudaGetLastError());
    std::vector<uint64_t> ptrs(t->n), lens(t->n);
    std::vector<uint32_t> bufs(t->n);
    for (uint32_t i = 0; i < t->n; ++i) {
        ptrs[i] = reinterpret_cast<uint64_t>(dv) + t->img_off[i];
        lens[i] = t->size[i];
        bufs[i] = i;
    }
    return digest_regions(ptrs, lens, bufs, out, nullptr, nullptr, nullptr, nullptr, s);
}
