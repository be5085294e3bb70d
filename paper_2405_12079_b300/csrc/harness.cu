// Harness kernels: digest, mutator and fill (see include/phos_harness.h).
// They stand in for the application and fingerprint memory; they are not
// part of the checkpoint/restore method.
#include <algorithm>
#include <vector>

#include "../../include/phos_harness.h"
#include "digest_dev.cuh"
#include "internal.h"

namespace phos {

constexpr uint64_t kHTile = 256 * 1024;  // bytes per CTA work item
constexpr int kMaxEnt = 64;

struct Ent {
    uint64_t ptr, len;
    uint64_t key;      // fill: key of the region's words
    uint64_t jbase;    // fill: word index of the entry's first byte
    uint32_t tile0;    // first global tile of this entry
    uint32_t id;       // digest: output slot; mutate: written buffer index
};

struct EntBatch {
    Ent e[kMaxEnt];
    uint32_t count;
    uint32_t tiles;
};

__device__ __forceinline__ int find_ent(const EntBatch &b, uint32_t t) {
    int lo = 0;
    for (int q = 1; q < (int)b.count; ++q)
        if (b.e[q].tile0 <= t) lo = q;
    return lo;
}

__global__ void __launch_bounds__(512) k_digest(const __grid_constant__ EntBatch b,
                                                unsigned long long *out) {
    __shared__ unsigned long long s_acc;
    if (threadIdx.x == 0) s_acc = 0;
    __syncthreads();
    for (uint32_t t = blockIdx.x; t < b.tiles; t += gridDim.x) {
        const Ent &e = b.e[find_ent(b, t)];
        const uint64_t off = (uint64_t)(t - e.tile0) * kHTile;
        const uint64_t end = min(off + kHTile, e.len);
        const unsigned long long acc =
            digest_range(reinterpret_cast<const uint8_t *>(e.ptr), e.len, off, end);
        if ((threadIdx.x & 31) == 0 && acc) atomicAdd(&s_acc, acc);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_acc) atomicAdd(out + e.id, s_acc);
            s_acc = 0;
        }
        __syncthreads();
    }
}

__global__ void k_zero64(unsigned long long *p, uint32_t n) {
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) p[i] = 0;
}

// word j of a region = sm(key ^ j); key fixed per entry, or derived from
// the mutator seed when dig != nullptr.
__global__ void __launch_bounds__(512) k_fill(const __grid_constant__ EntBatch b,
                                              const unsigned long long *dig, uint32_t nr,
                                              uint64_t seed, uint64_t k) {
    __shared__ uint64_t s_sk;
    if (dig) {
        if (threadIdx.x == 0) {
            uint64_t s = sm64(seed ^ sm64(k));
            for (uint32_t q = 0; q < nr; ++q) s = sm64(s ^ dig[q]);
            s_sk = s;
        }
        __syncthreads();
    }
    for (uint32_t t = blockIdx.x; t < b.tiles; t += gridDim.x) {
        const Ent &e = b.e[find_ent(b, t)];
        const uint64_t key = dig ? sm64(s_sk ^ sm64((uint64_t)e.id)) : e.key;
        const uint64_t off = (uint64_t)(t - e.tile0) * kHTile;
        const uint64_t end = min(off + kHTile, e.len);
        uint8_t *p = reinterpret_cast<uint8_t *>(e.ptr);
        const uint64_t j0 = e.jbase + off / 8;
        if (((uintptr_t)(p + off) & 15) == 0) {
            const uint64_t full = (end - off) / 16;
            uint4 *q = reinterpret_cast<uint4 *>(p + off);
            for (uint64_t i = threadIdx.x; i < full; i += blockDim.x) {
                const uint64_t j = j0 + 2 * i;
                const uint64_t w0 = sm64(key ^ j), w1 = sm64(key ^ (j + 1));
                q[i] = make_uint4((uint32_t)w0, (uint32_t)(w0 >> 32), (uint32_t)w1,
                                  (uint32_t)(w1 >> 32));
            }
            for (uint64_t bb = off + 16 * full + threadIdx.x; bb < end; bb += blockDim.x)
                p[bb] = (uint8_t)(sm64(key ^ (e.jbase + bb / 8)) >> (8 * (bb & 7)));
        } else {
            for (uint64_t bb = off + threadIdx.x; bb < end; bb += blockDim.x)
                p[bb] = (uint8_t)(sm64(key ^ (e.jbase + bb / 8)) >> (8 * (bb & 7)));
        }
    }
}

__global__ void k_strays(const uint64_t *strays, uint32_t ns, uint64_t seed, uint64_t k) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const uint64_t kk = sm64(seed ^ k);
    for (uint32_t q = 0; q < ns; ++q) {
        const uint64_t r = strays[2 * q], a = strays[2 * q + 1];
        const uint32_t v = (uint32_t)sm64(kk ^ r);
        uint8_t *p = reinterpret_cast<uint8_t *>(a);
        for (int t = 0; t < 4; ++t) p[t] = (uint8_t)(v >> (8 * t));
    }
}

// Split (ptr, len, id, key) entries into batches of kMaxEnt and launch.
template <typename F>
static phos_status batched(const std::vector<Ent> &ents, F launch) {
    for (size_t b0 = 0; b0 < ents.size(); b0 += kMaxEnt) {
        EntBatch b{};
        uint32_t tiles = 0;
        b.count = (uint32_t)std::min<size_t>(kMaxEnt, ents.size() - b0);
        for (uint32_t q = 0; q < b.count; ++q) {
            b.e[q] = ents[b0 + q];
            b.e[q].tile0 = tiles;
            tiles += (uint32_t)std::max<uint64_t>(1, (b.e[q].len + kHTile - 1) / kHTile);
        }
        b.tiles = tiles;
        phos_status r = launch(b);
        if (r) return r;
    }
    return PHOS_OK;
}

static unsigned grid_for(uint32_t tiles) {
    return (unsigned)std::max<uint32_t>(1, std::min<uint32_t>(tiles, 148 * 4));
}

}  // namespace phos

using namespace phos;

extern "C" phos_status phos_harness_digest(const uint64_t *ptrs, const uint64_t *lens, uint32_t n,
                                           uint64_t *d_out, phos_stream_t stream) {
    if (n == 0) return PHOS_OK;
    if (!ptrs || !lens || !d_out) return fail(PHOS_EINVAL, "harness_digest: NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<Ent> ents(n);
    for (uint32_t j = 0; j < n; ++j) {
        void *dp = nullptr;
        phos_status r = device_view(reinterpret_cast<void *>(ptrs[j]), &dp);
        if (r) return r;
        ents[j] = Ent{(uint64_t)dp, lens[j], 0, 0, 0, j};
    }
    unsigned long long *out = reinterpret_cast<unsigned long long *>(d_out);
    k_zero64<<<1, 256, 0, s>>>(out, n);
    count_launch();
    PHOS_CUDA(cudaGetLastError());
    return batched(ents, [&](const EntBatch &b) -> phos_status {
        k_digest<<<grid_for(b.tiles), 512, 0, s>>>(b, out);
        count_launch();
        PHOS_CUDA(cudaGetLastError());
        return PHOS_OK;
    });
}

extern "C" phos_status phos_harness_mutate(const phos_table_t *t, uint64_t seed, uint64_t k,
                                           const uint32_t *reads, uint32_t nr,
                                           const uint32_t *writes, uint32_t nw,
                                           const uint64_t *d_strays, uint32_t ns,
                                           phos_stream_t stream) {
    if (!t) return fail(PHOS_EINVAL, "harness_mutate: table is NULL");
    if ((nr && !reads) || (nw && !writes) || (ns && !d_strays))
        return fail(PHOS_EINVAL, "harness_mutate: NULL argument");
    for (uint32_t q = 0; q < nr; ++q)
        if (reads[q] >= t->n || (q && reads[q] <= reads[q - 1]))
            return fail(PHOS_EINVAL, "harness_mutate: reads must be ascending table indices");
    for (uint32_t q = 0; q < nw; ++q)
        if (writes[q] >= t->n) return fail(PHOS_EINVAL, "harness_mutate: bad write index");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    phos_table *T = const_cast<phos_table *>(t);
    {
        std::lock_guard<std::mutex> g(T->mu);
        phos_status r = T->harness_scratch.reserve(8ull * std::max(nr, 1u));
        if (r) return r;
    }
    unsigned long long *dig = static_cast<unsigned long long *>(T->harness_scratch.ptr);
    std::vector<Ent> ents;
    for (uint32_t q = 0; q < nr; ++q)
        ents.push_back(Ent{t->base[reads[q]], t->size[reads[q]], 0, 0, 0, q});
    if (nr) {
        k_zero64<<<1, 256, 0, s>>>(dig, nr);
        count_launch();
        PHOS_CUDA(cudaGetLastError());
        phos_status r = batched(ents, [&](const EntBatch &b) -> phos_status {
            k_digest<<<grid_for(b.tiles), 512, 0, s>>>(b, dig);
            count_launch();
            PHOS_CUDA(cudaGetLastError());
            return PHOS_OK;
        });
        if (r) return r;
    }
    ents.clear();
    for (uint32_t q = 0; q < nw; ++q)
        ents.push_back(Ent{t->base[writes[q]], t->size[writes[q]], 0, 0, 0, writes[q]});
    phos_status r = batched(ents, [&](const EntBatch &b) -> phos_status {
        k_fill<<<grid_for(b.tiles), 512, 0, s>>>(b, dig, nr, seed, k);
        count_launch();
        PHOS_CUDA(cudaGetLastError());
        return PHOS_OK;
    });
    if (r) return r;
    if (ns) {
        k_strays<<<1, 32, 0, s>>>(d_strays, ns, seed, k);
        count_launch();
        PHOS_CUDA(cudaGetLastError());
    }
    return PHOS_OK;
}

extern "C" phos_status phos_harness_fill(uint64_t ptr, uint64_t len, uint64_t key,
                                         phos_stream_t stream) {
    if (len == 0) return PHOS_OK;
    if (!ptr) return fail(PHOS_EINVAL, "harness_fill: NULL pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // 1 GiB pieces keep a batch's tile count within 32 bits; word indices
    // continue across pieces (jbase)
    std::vector<Ent> ents;
    const uint64_t piece = 1ull << 30;
    for (uint64_t o = 0; o < len; o += piece)
        ents.push_back(Ent{ptr + o, std::min(piece, len - o), key, o / 8, 0, 0});
    return batched(ents, [&](const EntBatch &b) -> phos_status {
        k_fill<<<grid_for(b.tiles), 512, 0, s>>>(b, nullptr, 0, 0, 0);
        count_launch();
        PHOS_CUDA(cudaGetLastError());
        return PHOS_OK;
    });
}

extern "C" phos_status phos_harness_drive_ckpt(phos_ckpt_t *c, const phos_table_t *t,
                                               uint64_t seed, uint64_t quota,
                                               const phos_harness_kernel_t *ks, uint32_t n,
                                               phos_stream_t stream, uint32_t *kernels_run) {
    if (!c || !t || (n && !ks)) return fail(PHOS_EINVAL, "harness_drive_ckpt: NULL argument");
    std::vector<uint8_t> perm(std::max(t->n, 1u));
    uint32_t k = 0;
    phos_status r = PHOS_OK;
    while (k < n) {
        int done = 0, mis = 0;
        if ((r = phos_ckpt_advance(c, quota, &done))) break;
        if (done) break;
        const phos_harness_kernel_t &K = ks[k];
        std::fill(perm.begin(), perm.end(), 0);
        if ((r = phos_speculate(t, K.args, K.arg_size, K.kind, K.nargs, perm.data()))) break;
        if ((r = phos_ckpt_before_kernel(c, perm.data()))) break;
        if ((r = phos_harness_mutate(t, seed, k, K.reads, K.nr, K.writes, K.nw, K.d_strays, K.ns,
                                     stream)))
            break;
        if ((r = phos_ckpt_after_kernel(c, K.d_trace, K.n_rec, &mis))) break;
        ++k;
        if (mis) break;
    }
    if (kernels_run) *kernels_run = k;
    return r;
}

// Test hooks on a table handle (see phos_harness.h).
extern "C" phos_status phos_harness_table_rebind(phos_table_t *t, int device, int *old_device) {
    if (!t) return fail(PHOS_EINVAL, "harness_table_rebind: table is NULL");
    if (old_device) *old_device = t->device;
    t->device = device;
    return PHOS_OK;
}

extern "C" phos_status phos_harness_table_scratch(const phos_table_t *t, uint64_t *val_bytes) {
    if (!t || !val_bytes) return fail(PHOS_EINVAL, "harness_table_scratch: NULL argument");
    phos_table *T = const_cast<phos_table *>(t);
    std::lock_guard<std::mutex> g(T->mu);
    *val_bytes = T->val_scratch.bytes;
    return PHOS_OK;
}

// Deferred validation launch, as sessions run it (see phos_harness.h).
extern "C" phos_status phos_harness_validate_rounds(const phos_table_t *t,
                                                   const phos_harness_round_t *rounds, uint32_t k,
                                                   uint32_t access_bytes, uint32_t rule,
                                                   uint8_t *d_dirty, uint64_t *d_acc,
                                                   int64_t *d_flag, uint32_t *d_status,
                                                   void *d_scratch, phos_stream_t stream) {
    if (!t || (k && !rounds) || !d_acc || !d_flag || !d_scratch)
        return fail(PHOS_EINVAL, "harness_validate_rounds: NULL argument");
    if (rule < 1 || rule > 3) return fail(PHOS_EINVAL, "harness_validate_rounds: rule %u", rule);
    if (rule == 1 && !d_dirty) return fail(PHOS_EINVAL, "harness_validate_rounds: NULL d_dirty");
    if (access_bytes == 0) return fail(PHOS_EINVAL, "harness_validate_rounds: access_bytes is 0");
    const uint32_t cap = rounds_cap(t->n, t->device);
    if (k > cap)
        return fail(PHOS_EINVAL, "harness_validate_rounds: %u rounds, at most %u for %u buffers", k,
                    cap, t->n);
    std::vector<RoundSeg> seg(k);
    for (uint32_t i = 0; i < k; ++i) {
        const phos_harness_round_t &R = rounds[i];
        if (R.n_rec && (!R.d_trace || ((uintptr_t)R.d_trace & 15)))
            return fail(PHOS_EINVAL, "harness_validate_rounds: round %u trace NULL or unaligned", i);
        if (t->n && (!R.d_perm || !R.d_flags))
            return fail(PHOS_EINVAL, "harness_validate_rounds: round %u perm or flags NULL", i);
        seg[i] = RoundSeg{R.d_trace, R.n_rec, R.d_perm, R.d_flags, R.round};
    }
    return validate_rounds(t, seg.data(), k, access_bytes, rule, d_dirty, d_acc, d_flag, d_status,
                           d_scratch, static_cast<cudaStream_t>(stream));
}

extern "C" phos_status phos_harness_rounds_scratch(const phos_table_t *t, uint64_t *bytes,
                                                  uint32_t *max_rounds) {
    if (!t || !bytes) return fail(PHOS_EINVAL, "harness_rounds_scratch: NULL argument");
    *bytes = rounds_scratch_bytes(t->n, kMaxRounds);
    if (max_rounds) *max_rounds = rounds_cap(t->n, t->device);
    return PHOS_OK;
}
