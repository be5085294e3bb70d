// The copy engine behind soft copy-on-write (PhoenixOS Sec. 4.2), soft
// recopy (Sec. 4.3, chunked as in Sec. 5) and soft on-demand restore
// (Sec. 6): batched gather-copies of (buffer, offset, len) regions between
// live device memory, a device staging area and the image (pinned host
// memory reached through its mapped address, or device memory).
//
// B300 design
//   * Two launches per batch.  A one-CTA prologue validates and resolves
//     every descriptor to (src, dst, len) and scans the per-descriptor tile
//     counts; the main kernel is a persistent grid (SMs x CTAs-per-SM) that
//     walks global tile ids, finds each tile's descriptor by binary search
//     over the scan, and copies it with the whole CTA.  No host round trip
//     and no per-descriptor launch, so thousands of small regions cost the
//     same launch overhead as one.
//   * The copy is SM-driven: 16-byte vector loads/stores with four loads in
//     flight per thread, streaming cache hints (evict-first) because a
//     checkpoint touches each byte once.  Device->host and host->device
//     legs are the same kernel with the image end in mapped pinned memory:
//     plain stores post straight onto PCIe, and loads from host memory are
//     hidden behind the grid's bytes in flight.
//   * Regions whose source and destination share 16-byte alignment take the
//     vector path with a byte head and tail; otherwise the destination is
//     brought to a 16-byte boundary and each aligned 16-byte store takes its
//     bytes out of two aligned source vectors with funnel shifts (the
//     neighbouring vector comes from the next lane by a shuffle, so every
//     source vector is loaded once).
//   * Present bits (restore) are set by the CTA that finishes a
//     descriptor's last tile, after a device-wide fence, so a stream-ordered
//     reader never sees a bit before its bytes.
#include <string.h>

#include <algorithm>

#include "copy_dev.cuh"
#include "internal.h"

namespace phos {

struct CopyRes {
    const uint8_t *src;
    uint8_t *dst;
    uint64_t len;
    uint64_t ntiles;
    uint32_t buf;
    uint32_t flags;
};

struct CopyArgs {
    const phos_copy_t *list;
    uint32_t n;            // descriptors (the capacity when n_dev is set)
    const uint32_t *n_dev; // optional: the count, read on the device (<= n)
    TableDev tab;
    uint8_t *staging;
    uint64_t staging_bytes;
    uint8_t *image;
    uint64_t image_bytes;
    uint32_t *present;
    uint32_t *status;
    uint32_t allow;        // bit k set: direction k allowed
    uint64_t tile;
    // scratch
    uint64_t *prefix;      // [n + 1]
    CopyRes *res;          // [n]
    uint32_t *done;        // [n]
};

__device__ __forceinline__ uint32_t copy_count(const CopyArgs &a) {
    return a.n_dev ? min(*a.n_dev, a.n) : a.n;
}

__global__ void __launch_bounds__(1024) k_copy_prep(const CopyArgs a) {
    __shared__ unsigned long long s_warp[32];
    __shared__ unsigned long long s_carry;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t N = copy_count(a);
    if (tid == 0) {
        s_carry = 0;
        a.prefix[0] = 0;
    }
    __syncthreads();
    for (uint32_t b0 = 0; b0 < N; b0 += blockDim.x) {
        const uint32_t d = b0 + tid;
        unsigned long long nt = 0;
        if (d < N) {
            const phos_copy_t c = a.list[d];
            const uint32_t dir = c.flags & PHOS_COPY_DIR_MASK;
            bool ok = (c.flags & ~(uint32_t)(PHOS_COPY_DIR_MASK | PHOS_COPY_MARK_PRESENT)) == 0 &&
                      dir >= 1 && dir <= 4 && ((a.allow >> dir) & 1);
            const uint8_t *src = nullptr;
            uint8_t *dst = nullptr;
            auto live_ok = [&](uint64_t off) {
                return c.buf < a.tab.n && off <= a.tab.size[c.buf] &&
                       c.len <= a.tab.size[c.buf] - off;
            };
            auto area_ok = [&](const uint8_t *p, uint64_t bytes, uint64_t off) {
                return p != nullptr && off <= bytes && c.len <= bytes - off;
            };
            if (ok) {
                switch (dir) {
                    case PHOS_COPY_LIVE_TO_STAGING:
                        ok = live_ok(c.src_off) && area_ok(a.staging, a.staging_bytes, c.dst_off);
                        if (ok) {
                            src = (const uint8_t *)(a.tab.base[c.buf] + c.src_off);
                            dst = a.staging + c.dst_off;
                        }
                        break;
                    case PHOS_COPY_LIVE_TO_IMAGE:
                        ok = live_ok(c.src_off) && area_ok(a.image, a.image_bytes, c.dst_off);
                        if (ok) {
                            src = (const uint8_t *)(a.tab.base[c.buf] + c.src_off);
                            dst = a.image + c.dst_off;
                        }
                        break;
                    case PHOS_COPY_STAGING_TO_IMAGE:
                        ok = area_ok(a.staging, a.staging_bytes, c.src_off) &&
                             area_ok(a.image, a.image_bytes, c.dst_off);
                        if (ok) {
                            src = a.staging + c.src_off;
                            dst = a.image + c.dst_off;
                        }
                        break;
                    default:  // IMAGE_TO_LIVE
                        ok = area_ok(a.image, a.image_bytes, c.src_off) && live_ok(c.dst_off);
                        if (ok) {
                            src = a.image + c.src_off;
                            dst = (uint8_t *)(a.tab.base[c.buf] + c.dst_off);
                        }
                        break;
                }
            }
            if (ok && (c.flags & PHOS_COPY_MARK_PRESENT) && (!a.present || c.buf >= a.tab.n))
                ok = false;
            if (ok) {
                nt = (c.len + a.tile - 1) / a.tile;
                if (nt == 0 && (c.flags & PHOS_COPY_MARK_PRESENT)) nt = 1;
            } else {
                set_status(a.status, PHOS_EINVAL);
            }
            CopyRes r;
            r.src = src;
            r.dst = dst;
            r.len = ok ? c.len : 0;
            r.ntiles = nt;
            r.buf = c.buf;
            r.flags = ok ? c.flags : 0;
            a.res[d] = r;
            a.done[d] = 0;
        }
        // block inclusive scan of nt
        unsigned long long incl = nt;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        unsigned long long woff = 0, total = 0;
        for (uint32_t q = 0; q < (blockDim.x >> 5); ++q) {
            if (q < warp) woff += s_warp[q];
            total += s_warp[q];
        }
        const unsigned long long carry = s_carry;
        if (d < N) a.prefix[d + 1] = carry + woff + incl;
        __syncthreads();
        if (tid == 0) s_carry = carry + total;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(512, 3) k_copy_main(const CopyArgs a) {
    __shared__ uint32_t s_d;
    __shared__ uint32_t s_last;
    const uint32_t N = copy_count(a);
    const uint64_t total = a.prefix[N];
    for (uint64_t t = blockIdx.x; t < total; t += gridDim.x) {
        if (threadIdx.x == 0) {
            // last descriptor whose prefix <= t
            uint32_t lo = 0, cnt = N + 1;
            while (cnt > 0) {
                uint32_t half = cnt >> 1;
                if (a.prefix[lo + half] <= t) {
                    lo += half + 1;
                    cnt -= half + 1;
                } else {
                    cnt = half;
                }
            }
            s_d = lo - 1;
        }
        __syncthreads();
        const uint32_t d = s_d;
        const CopyRes r = a.res[d];
        const uint64_t off = (t - a.prefix[d]) * a.tile;
        const uint64_t len = off < r.len ? min(a.tile, r.len - off) : 0;
        copy_block(r.dst + off, r.src + off, len);
        if (r.flags & PHOS_COPY_MARK_PRESENT) {
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) {
                s_last = (atomicAdd(&a.done[d], 1u) + 1 == (uint32_t)r.ntiles) ? 1u : 0u;
                if (s_last) {
                    __threadfence();
                    atomicOr(&a.present[r.buf >> 5], 1u << (r.buf & 31));
                }
            }
        }
        __syncthreads();
    }
}

size_t copy_scratch_bytes(uint32_t n) {
    const size_t off_res = align_up(8ull * (n + 1), 256);
    const size_t off_done = align_up(off_res + sizeof(CopyRes) * (size_t)n, 256);
    return off_done + 4ull * n;
}

static uint64_t g_tile = 1ull << 16;  // 64 KiB per CTA work item
static uint32_t g_ctas_per_sm = 3;

static phos_status launch_copy(const phos_table_t *t, const phos_copy_t *d_list, uint32_t n,
                               void *staging, uint64_t staging_bytes, const void *image,
                               uint64_t image_bytes, uint32_t *d_present, uint32_t *d_status,
                               uint32_t allow, phos_stream_t stream, const char *who,
                               const uint32_t *d_n = nullptr) {
    if (!t) return fail(PHOS_EINVAL, "%s: table is NULL", who);
    if (n == 0) return PHOS_OK;
    if (!d_list) return fail(PHOS_EINVAL, "%s: d_list is NULL", who);
    void *img = nullptr, *stg = nullptr;
    phos_status r = device_view(image, &img);
    if (r) return r;
    r = device_view(staging, &stg);
    if (r) return r;
    phos_table *T = const_cast<phos_table *>(t);
    const size_t off_res = align_up(8ull * (n + 1), 256);
    const size_t off_done = align_up(off_res + sizeof(CopyRes) * (size_t)n, 256);
    const size_t need = copy_scratch_bytes(n);
    {
        std::lock_guard<std::mutex> g(T->mu);
        r = T->copy_scratch.reserve(need);
        if (r) return r;
    }
    uint8_t *sc = static_cast<uint8_t *>(T->copy_scratch.ptr);
    CopyArgs a;
    a.list = d_list;
    a.n = n;
    a.n_dev = d_n;
    a.tab = t->view;
    a.staging = static_cast<uint8_t *>(stg);
    a.staging_bytes = stg ? staging_bytes : 0;
    a.image = static_cast<uint8_t *>(img);
    a.image_bytes = img ? image_bytes : 0;
    a.present = d_present;
    a.status = d_status;
    a.allow = allow;
    a.tile = g_tile;
    a.prefix = reinterpret_cast<uint64_t *>(sc);
    a.res = reinterpret_cast<CopyRes *>(sc + off_res);
    a.done = reinterpret_cast<uint32_t *>(sc + off_done);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_copy_prep<<<1, 1024, 0, s>>>(a);
    count_launch();
    PHOS_CUDA(cudaGetLastError());
    const unsigned G = (unsigned)(sm_count(T->device) * g_ctas_per_sm);
    k_copy_main<<<G, 512, 0, s>>>(a);
    count_launch();
    PHOS_CUDA(cudaGetLastError());
    return PHOS_OK;
}

// Small host -> device uploads without a device-side read of host memory.
// While the copier's device -> host DMA copies fill the link, anything the
// device has to fetch from host memory at run time waits behind them: a
// cudaMemcpyAsync of 2 KB took ~60 us on B300 (~3 us idle), and SM loads
// from mapped pinned memory stalled the same way.  Kernel parameters travel
// with the launch, which the front end fetches ahead of execution, so
// bytes up to a parameter block go as the parameters of k_put; larger
// uploads fall back to k_pull (SM loads from the mapped arena).
template <uint32_t kData>
struct PutArgs {
    uint8_t *dst;
    uint64_t len;
    uint8_t data[kData];
};

template <uint32_t kData>
__global__ void __launch_bounds__(256) k_put(const __grid_constant__ PutArgs<kData> a) {
    const uint64_t n = a.len;
    uint64_t done = 0;
    // 8-byte units (data sits 16 bytes into a block of 8-byte alignment)
    if (((uintptr_t)a.dst & 7) == 0) {
        const uint64_t nv = n / 8;
        const uint64_t *s = reinterpret_cast<const uint64_t *>(a.data);
        uint64_t *d = reinterpret_cast<uint64_t *>(a.dst);
        for (uint64_t i = threadIdx.x; i < nv; i += blockDim.x) d[i] = s[i];
        done = nv * 8;
    }
    for (uint64_t i = done + threadIdx.x; i < n; i += blockDim.x) a.dst[i] = a.data[i];
}

__global__ void __launch_bounds__(256) k_pull(uint8_t *dst, const uint8_t *src, uint64_t n) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    uint64_t done = 0;
    if ((((uintptr_t)dst | (uintptr_t)src) & 15) == 0) {
        const uint64_t nv = n / 16;
        const uint4 *s = reinterpret_cast<const uint4 *>(src);
        uint4 *d = reinterpret_cast<uint4 *>(dst);
        // volatile loads: a line of host memory seen before is fetched again
        for (uint64_t i = tid; i < nv; i += nt) d[i] = __ldcv(s + i);
        done = nv * 16;
    }
    for (uint64_t i = done + tid; i < n; i += nt) dst[i] = (uint8_t)__ldcv(src + i);
}

// The parameter blocks: 4 KB (the classic limit) and 32 KB (the limit of
// CUDA 12.1 and later), less the header.
constexpr uint32_t kPutSmall = 4096 - 16, kPutLarge = 32752 - 16;

template <uint32_t kData>
static phos_status put_launch(void *d_dst, const void *h_src, uint64_t bytes, cudaStream_t s) {
    PutArgs<kData> a;
    a.dst = static_cast<uint8_t *>(d_dst);
    a.len = bytes;
    memcpy(a.data, h_src, bytes);
    k_put<kData><<<1, 256, 0, s>>>(a);
    count_launch();
    PHOS_CUDA(cudaGetLastError());
    return PHOS_OK;
}

phos_status push_small(void *d_dst, const void *h_src, const void *h_src_dev, uint64_t bytes,
                       cudaStream_t s) {
    if (!bytes) return PHOS_OK;
    if (bytes <= kPutSmall) return put_launch<kPutSmall>(d_dst, h_src, bytes, s);
    if (bytes <= kPutLarge) return put_launch<kPutLarge>(d_dst, h_src, bytes, s);
    const uint64_t ctas = std::min<uint64_t>((bytes + 16 * 256 * 4 - 1) / (16 * 256 * 4), 64);
    k_pull<<<(unsigned)ctas, 256, 0, s>>>(static_cast<uint8_t *>(d_dst),
                                           static_cast<const uint8_t *>(h_src_dev), bytes);
    count_launch();
    PHOS_CUDA(cudaGetLastError());
    return PHOS_OK;
}

phos_status copy_device_count(const phos_table_t *t, const phos_copy_t *d_list, uint32_t cap,
                              const uint32_t *d_n, void *staging, uint64_t staging_bytes,
                              const void *image, uint64_t image_bytes, uint32_t *d_present,
                              uint32_t *d_status, phos_stream_t stream) {
    if (!d_n) return fail(PHOS_EINVAL, "copy_device_count: NULL count");
    return launch_copy(t, d_list, cap, staging, staging_bytes, image, image_bytes, d_present,
                       d_status, 0x1Eu, stream, "copy_device_count", d_n);
}

}  // namespace phos

using namespace phos;

extern "C" phos_status phos_copy_config(uint64_t tile_bytes, uint32_t ctas_per_sm) {
    if (tile_bytes) {
        if (tile_bytes % 4096 || tile_bytes < 4096 || tile_bytes > (16ull << 20))
            return fail(PHOS_EINVAL, "copy_config: tile_bytes %llu", (unsigned long long)tile_bytes);
        g_tile = tile_bytes;
    }
    if (ctas_per_sm) {
        if (ctas_per_sm > 8) return fail(PHOS_EINVAL, "copy_config: ctas_per_sm %u", ctas_per_sm);
        g_ctas_per_sm = ctas_per_sm;
    }
    return PHOS_OK;
}

extern "C" phos_status phos_cow_copy(const phos_table_t *t, const phos_copy_t *d_list, uint32_t n,
                                     void *d_staging, uint64_t staging_bytes, uint32_t *d_status,
                                     phos_stream_t stream) {
    return launch_copy(t, d_list, n, d_staging, staging_bytes, nullptr, 0, nullptr, d_status,
                       1u << PHOS_COPY_LIVE_TO_STAGING, stream, "cow_copy");
}

extern "C" phos_status phos_recopy(const phos_table_t *t, const phos_copy_t *d_list, uint32_t n,
                                   void *image, uint64_t image_bytes, uint32_t *d_status,
                                   phos_stream_t stream) {
    return launch_copy(t, d_list, n, nullptr, 0, image, image_bytes, nullptr, d_status,
                       1u << PHOS_COPY_LIVE_TO_IMAGE, stream, "recopy");
}

extern "C" phos_status phos_restore_on_demand(const phos_table_t *t, const phos_copy_t *d_list,
                                              uint32_t n, const void *image,
                                              uint64_t image_bytes, uint32_t *d_present,
                                              uint32_t *d_status, phos_stream_t stream) {
    return launch_copy(t, d_list, n, nullptr, 0, image, image_bytes, d_present, d_status,
                       1u << PHOS_COPY_IMAGE_TO_LIVE, stream, "restore_on_demand");
}

extern "C" phos_status phos_copy(const phos_table_t *t, const phos_copy_t *d_list, uint32_t n,
                                 void *d_staging, uint64_t staging_bytes, void *image,
                                 uint64_t image_bytes, uint32_t *d_present, uint32_t *d_status,
                                 phos_stream_t stream) {
    return launch_copy(t, d_list, n, d_staging, staging_bytes, image, image_bytes, d_present,
                       d_status, 0x1Eu, stream, "copy");
}
