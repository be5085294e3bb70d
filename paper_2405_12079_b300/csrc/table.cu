// Buffer table, speculation (host side), error reporting and shared
// host utilities of the C ABI.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <set>
#include <utility>

#include "internal.h"

namespace phos {

static std::atomic<uint64_t> g_launches{0};
void count_launch(uint32_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

static thread_local std::string g_last_error;

phos_status fail(phos_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

phos_status cuda_fail(cudaError_t e, const char *what) {
    return fail(PHOS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

phos_status Scratch::reserve(size_t need) {
    if (need <= bytes) return PHOS_OK;
    size_t nb = std::max(need, bytes * 2);
    nb = align_up(nb, 4096);
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, nb);
    if (e != cudaSuccess) return fail(PHOS_ENOMEM, "scratch cudaMalloc(%zu): %s", nb,
                                      cudaGetErrorString(e));
    // zero so that self-cleaning accumulators start from a known state;
    // the device-wide sync orders the memset before work on any stream and
    // retires work still using the old allocation
    e = cudaMemset(p, 0, nb);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(p);
        return cuda_fail(e, "scratch zeroing");
    }
    if (ptr) cudaFree(ptr);
    ptr = p;
    bytes = nb;
    return PHOS_OK;
}

Scratch::~Scratch() {
    if (ptr) cudaFree(ptr);
}

phos_status smem_optin_once(const void *fn) {
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    int dev = 0;
    PHOS_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> g(mu);
    if (done.count({fn, dev})) return PHOS_OK;
    PHOS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    done.insert({fn, dev});
    return PHOS_OK;
}

int sm_count(int device) {
    static int cached[64] = {0};
    if (device < 0 || device >= 64) return 148;
    if (!cached[device]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
        cached[device] = v > 0 ? v : 148;
    }
    return cached[device];
}

phos_status device_view(const void *p, void **out) {
    if (!p) {
        *out = nullptr;
        return PHOS_OK;
    }
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) return cuda_fail(e, "cudaPointerGetAttributes(image)");
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
        *out = const_cast<void *>(p);
        return PHOS_OK;
    }
    if (a.type == cudaMemoryTypeHost && a.devicePointer) {
        *out = a.devicePointer;
        return PHOS_OK;
    }
    return fail(PHOS_EINVAL, "image %p is pageable host memory; pin or register it", p);
}

}  // namespace phos

using namespace phos;

extern "C" const char *phos_last_error(void) { return g_last_error.c_str(); }

extern "C" uint64_t phos_launch_count(void) { return g_launches.load(); }

extern "C" const char *phos_status_name(phos_status s) {
    switch (s) {
        case PHOS_OK: return "PHOS_OK";
        case PHOS_EINVAL: return "PHOS_EINVAL";
        case PHOS_ENOMEM: return "PHOS_ENOMEM";
        case PHOS_EBUDGET: return "PHOS_EBUDGET";
        case PHOS_ECUDA: return "PHOS_ECUDA";
        case PHOS_ETIMEDOUT: return "PHOS_ETIMEDOUT";
        case PHOS_ECORRUPT: return "PHOS_ECORRUPT";
        case PHOS_EMISSPEC: return "PHOS_EMISSPEC";
        default: return "PHOS_E?";
    }
}

extern "C" phos_status phos_table_create(const phos_buf_t *bufs, uint32_t n,
                                         phos_table_t **out) {
    if (!out) return fail(PHOS_EINVAL, "table_create: out is NULL");
    *out = nullptr;
    if (n && !bufs) return fail(PHOS_EINVAL, "table_create: bufs is NULL");
    if (n > kMaxTable) return fail(PHOS_EINVAL, "table_create: %u buffers > %u", n, kMaxTable);
    for (uint32_t i = 0; i < n; ++i) {
        const uint64_t b = bufs[i].base, s = bufs[i].size;
        if (s == 0) return fail(PHOS_EINVAL, "table_create: buffer %u has size 0", i);
        if (b > PHOS_REC_ADDR_MASK || s > PHOS_REC_ADDR_MASK + 1 - b)
            return fail(PHOS_EINVAL, "table_create: buffer %u leaves the 57-bit space", i);
        if (i && bufs[i - 1].base + bufs[i - 1].size > b)
            return fail(PHOS_EINVAL, "table_create: buffers %u and %u unsorted or overlapping",
                        i - 1, i);
    }
    phos_table *t = new phos_table();
    cudaGetDevice(&t->device);
    t->n = n;
    t->base.resize(n);
    t->size.resize(n);
    t->img_off.resize(n);
    uint64_t acc = 0;
    for (uint32_t i = 0; i < n; ++i) {
        t->base[i] = bufs[i].base;
        t->size[i] = bufs[i].size;
        t->img_off[i] = acc;
        acc += align_up(bufs[i].size, 256);
    }
    t->image_bytes = acc;
    const uint32_t nf1 = (n + 31) / 32, nf2 = (n + 1023) / 1024;
    const size_t words = 2 * (size_t)std::max(n, 1u) + std::max(nf1, 1u) + std::max(nf2, 1u);
    std::vector<uint64_t> h(words, 0);
    uint64_t *hb = h.data(), *hs = hb + std::max(n, 1u), *hf1 = hs + std::max(n, 1u),
             *hf2 = hf1 + std::max(nf1, 1u);
    for (uint32_t i = 0; i < n; ++i) {
        hb[i] = bufs[i].base;
        hs[i] = bufs[i].size;
    }
    for (uint32_t j = 0; j < nf1; ++j) hf1[j] = bufs[32 * j].base;
    for (uint32_t j = 0; j < nf2; ++j) hf2[j] = bufs[1024 * j].base;
    cudaError_t e = cudaMalloc(&t->dev, words * 8);
    if (e != cudaSuccess) {
        delete t;
        return fail(PHOS_ENOMEM, "table_create: cudaMalloc: %s", cudaGetErrorString(e));
    }
    e = cudaMemcpy(t->dev, h.data(), words * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(t->dev);
        delete t;
        return cuda_fail(e, "table_create: cudaMemcpy");
    }
    uint64_t *d = static_cast<uint64_t *>(t->dev);
    t->view.base = d;
    t->view.size = d + std::max(n, 1u);
    t->view.fence1 = d + 2 * std::max(n, 1u);
    t->view.fence2 = t->view.fence1 + std::max(nf1, 1u);
    t->view.n = n;
    // the copy engine's scratch for up to max(n, 1024) descriptors now, so
    // that copies on this table (a server admitting it, a session's rounds)
    // never grow it -- growth synchronises the whole device
    phos_status r = t->copy_scratch.reserve(copy_scratch_bytes(std::max(n, kCopyReserve)));
    if (r) {
        phos_table_destroy(t);
        return r;
    }
    *out = t;
    return PHOS_OK;
}

extern "C" phos_status phos_table_destroy(phos_table_t *t) {
    if (!t) return PHOS_OK;
    if (t->dev) cudaFree(t->dev);
    delete t;
    return PHOS_OK;
}

extern "C" uint32_t phos_table_size(const phos_table_t *t) { return t ? t->n : 0; }

// index of the buffer containing v (base <= v < base + size), or -1
static long find_buf(const phos_table *t, uint64_t v) {
    auto it = std::upper_bound(t->base.begin(), t->base.end(), v);
    if (it == t->base.begin()) return -1;
    long i = (long)(it - t->base.begin()) - 1;
    return v - t->base[i] < t->size[i] ? i : -1;
}

extern "C" phos_status phos_speculate(const phos_table_t *t, const void *const *args,
                                      const uint32_t *arg_size, const uint8_t *kind,
                                      uint32_t nargs, uint8_t *perm_out) {
    if (!t || !perm_out || (nargs && (!args || !arg_size || !kind)))
        return fail(PHOS_EINVAL, "speculate: NULL argument");
    for (uint32_t j = 0; j < nargs; ++j) {
        const uint8_t *b = static_cast<const uint8_t *>(args[j]);
        if (kind[j] > PHOS_ARG_STRUCT) return fail(PHOS_EINVAL, "speculate: bad kind %u", kind[j]);
        if (kind[j] == PHOS_ARG_SCALAR) continue;
        if (!b && arg_size[j]) return fail(PHOS_EINVAL, "speculate: args[%u] is NULL", j);
        if (kind[j] == PHOS_ARG_STRUCT) {
            for (uint32_t off = 0; off + 8 <= arg_size[j]; off += 8) {
                uint64_t v;
                memcpy(&v, b + off, 8);
                long i = find_buf(t, v);
                if (i >= 0) perm_out[i] |= PHOS_PERM_RW;
            }
        } else {
            uint64_t v = 0;
            memcpy(&v, b, std::min<uint32_t>(arg_size[j], 8));
            long i = find_buf(t, v);
            if (i >= 0) perm_out[i] |= (kind[j] == PHOS_ARG_CONST_PTR) ? PHOS_PERM_R : PHOS_PERM_RW;
        }
    }
    return PHOS_OK;
}

// Device speculation: one warp per launch.  Lanes look up 32 argument words
// at a time (binary search over the device table); the hits are then
// OR-ed into the launch's perm row one lane after another, so no two lanes
// update a byte at once and no atomics are needed (each row belongs to
// one warp).
__global__ void k_speculate(phos::TableDev tab, const uint64_t *words, const uint8_t *kind,
                            const uint64_t *off, uint32_t n_launch, uint8_t *perm,
                            uint32_t *status) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t l = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (l >= n_launch) return;
    const uint64_t j0 = off[l], j1 = off[l + 1];
    uint8_t *row = perm + l * (uint64_t)tab.n;
    if (j1 < j0) {
        if (lane == 0) phos::set_status(status, PHOS_EINVAL);
        return;
    }
    for (uint64_t jb = j0; jb < j1; jb += 32) {
        const uint64_t j = jb + lane;
        int hit = -1;
        uint8_t pm = 0;
        if (j < j1) {
            const uint8_t k = kind[j];
            if (k > PHOS_ARG_STRUCT) phos::set_status(status, PHOS_EINVAL);
            if (k == PHOS_ARG_CONST_PTR || k == PHOS_ARG_MUT_PTR || k == PHOS_ARG_STRUCT) {
                const uint64_t v = words[j];
                uint32_t lo = 0, cnt = tab.n;       // last base <= v
                while (cnt > 0) {
                    const uint32_t half = cnt >> 1;
                    if (tab.base[lo + half] <= v) {
                        lo += half + 1;
                        cnt -= half + 1;
                    } else {
                        cnt = half;
                    }
                }
                if (lo > 0 && v - tab.base[lo - 1] < tab.size[lo - 1]) {
                    hit = (int)lo - 1;
                    pm = k == PHOS_ARG_CONST_PTR ? PHOS_PERM_R : PHOS_PERM_RW;
                }
            }
        }
        for (uint32_t q = 0; q < 32; ++q) {
            if (lane == q && hit >= 0) row[hit] |= pm;
            __syncwarp();
        }
    }
}

extern "C" phos_status phos_speculate_device(const phos_table_t *t, const uint64_t *d_words,
                                             const uint8_t *d_kind, const uint64_t *d_launch_off,
                                             uint32_t n_launch, uint8_t *d_perm,
                                             uint32_t *d_status, phos_stream_t stream) {
    if (!t || (n_launch && (!d_launch_off || !d_perm)))
        return fail(PHOS_EINVAL, "speculate_device: NULL argument");
    if (n_launch == 0 || t->n == 0) return PHOS_OK;
    const uint32_t warps = 8;
    const unsigned grid = (unsigned)((n_launch + warps - 1) / warps);
    k_speculate<<<grid, 32 * warps, 0, static_cast<cudaStream_t>(stream)>>>(
        t->view, d_words, d_kind, d_launch_off, n_launch, d_perm, d_status);
    count_launch();
    PHOS_CUDA(cudaGetLastError());
    return PHOS_OK;
}

extern "C" phos_status phos_speculate_region(const phos_table_t *t, uint64_t addr, uint64_t len,
                                             uint8_t perm, uint8_t *perm_out) {
    if (!t || !perm_out) return fail(PHOS_EINVAL, "speculate_region: NULL argument");
    if (len == 0) return PHOS_OK;
    // first buffer whose end is above addr
    auto it = std::upper_bound(t->base.begin(), t->base.end(), addr);
    size_t i = (it == t->base.begin()) ? 0 : (size_t)(it - t->base.begin()) - 1;
    for (; i < t->n && t->base[i] < addr + len; ++i)
        if (addr < t->base[i] + t->size[i]) perm_out[i] |= perm;
    return PHOS_OK;
}

extern "C" uint64_t phos_image_bytes(const phos_table_t *t) { return t ? t->image_bytes : 0; }

extern "C" phos_status phos_image_offsets(const phos_table_t *t, uint64_t *out) {
    if (!t || (!out && t->n)) return fail(PHOS_EINVAL, "image_offsets: NULL argument");
    for (uint32_t i = 0; i < t->n; ++i) out[i] = t->img_off[i];
    return PHOS_OK;
}
