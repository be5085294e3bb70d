// Device-decided protocol rounds (PHOS_CKPT_DEVICE): the per-round decisions
// of soft copy-on-write (PhoenixOS Sec. 4.2) and soft on-demand restore
// (Sec. 6) taken on the GPU from device-resident state, so that the host
// only enqueues work and a round needs no host data at all when the
// speculated permissions are on the device too (phos_speculate_device).
//
// State per buffer (device arrays): copier state (pending / in flight /
// done), bytes copied, the CoW shadow's staging offset, and the flags the
// validation rule reads (CoW: done or shadowed; restore: restored).  Per
// round, in stream order on the caller's stream:
//   k_dr_copier   one thread walks the copier cursor exactly as the host
//                 copier does (ascending index, pieces of at most `chunk`
//                 that never cross a buffer, cut at the quota left, each
//                 charging align256(len); restore skips restored buffers;
//                 a CoW drain from a shadow releases its staging extent) and
//                 writes the round's descriptors and log rows
//   copy engine   with the descriptor count read on the device
//   k_dr_need     restore: every buffer with perm != 0 not yet restored, in
//                 ascending order (block-wide scan), gets its remaining
//                 bytes as an on-demand copy and is marked restored
//   k_dr_cow      CoW: the candidates (perm has W, not done, not shadowed)
//                 are compacted in ascending order, then one thread
//                 allocates staging first fit for each (or copies its
//                 remaining bytes straight to the image when staging is
//                 full), and the rule flags are set
//   copy engine, the application kernel, the validation with its rule.
// The staging allocator is the host's first fit over free extents (sorted
// by offset, coalesced on release), kept in a device array.  Logs of every
// piece and every CoW / on-demand copy are kept on the device and read back
// at finish; their capacity is fixed at begin (an overflow is reported).
#include <algorithm>
#include <vector>

#include "internal.h"

namespace phos {

enum : uint8_t { kDrPending = 0, kDrInflight = 1, kDrDone = 2 };

struct DrDev {
    uint32_t n;
    uint32_t mode;          // 1 restore, 2 CoW
    uint64_t chunk;
    uint64_t staging_bytes;
    const uint64_t *size;   // table sizes (device)
    const uint64_t *img_off;
    uint8_t *state;
    uint64_t *copied;
    uint64_t *shadow;       // staging offset + 1, 0 = none
    uint8_t *flags;
    uint64_t *ext;          // free extents (off, len), sorted by off
    uint32_t *cand;         // [n] CoW candidates of a round
    phos_copy_t *lc;        // copier descriptors [cap_c]
    phos_copy_t *la;        // action descriptors [n]
    uint32_t *cnt;          // [0] copier descs, [1] action descs, [2] cursor, [3] extents,
                            // [4] overflow
    uint64_t *log_c;        // copier log rows (round, buf, off, len, shadow)
    uint64_t *log_a;        // CoW rows (round, buf, 1 staging | 2 image, off, len) or
                            // on-demand rows (round, buf, off, len, 0)
    unsigned long long *ctr;  // [0] copier rows, [1] action rows, [2] copier bytes,
                              // [3] CoW bytes, [4] direct bytes, [5] on-demand bytes
    uint32_t cap_c;
    uint64_t cap_lc;
    uint32_t mark_present;
};

__device__ __forceinline__ uint64_t a256(uint64_t x) { return (x + 255) & ~255ull; }

// First fit (one thread).  Returns false when no extent holds `need`.
__device__ bool dr_alloc(const DrDev &D, uint64_t need, uint64_t *off) {
    const uint32_t m = D.cnt[3];
    for (uint32_t j = 0; j < m; ++j) {
        const uint64_t o = D.ext[2 * j], l = D.ext[2 * j + 1];
        if (l >= need) {
            *off = o;
            if (l == need) {
                for (uint32_t q = j; q + 1 < m; ++q) {
                    D.ext[2 * q] = D.ext[2 * q + 2];
                    D.ext[2 * q + 1] = D.ext[2 * q + 3];
                }
                D.cnt[3] = m - 1;
            } else {
                D.ext[2 * j] = o + need;
                D.ext[2 * j + 1] = l - need;
            }
            return true;
        }
    }
    return false;
}

// Release with coalescing (one thread).
__device__ void dr_release(const DrDev &D, uint64_t off, uint64_t len) {
    uint32_t m = D.cnt[3];
    uint32_t j = 0;
    while (j < m && D.ext[2 * j] < off) ++j;
    for (uint32_t q = m; q > j; --q) {
        D.ext[2 * q] = D.ext[2 * q - 2];
        D.ext[2 * q + 1] = D.ext[2 * q - 1];
    }
    D.ext[2 * j] = off;
    D.ext[2 * j + 1] = len;
    ++m;
    if (j + 1 < m && D.ext[2 * j] + D.ext[2 * j + 1] == D.ext[2 * j + 2]) {
        D.ext[2 * j + 1] += D.ext[2 * j + 3];
        for (uint32_t q = j + 1; q + 1 < m; ++q) {
            D.ext[2 * q] = D.ext[2 * q + 2];
            D.ext[2 * q + 1] = D.ext[2 * q + 3];
        }
        --m;
    }
    if (j > 0 && D.ext[2 * j - 2] + D.ext[2 * j - 1] == D.ext[2 * j]) {
        D.ext[2 * j - 1] += D.ext[2 * j + 1];
        for (uint32_t q = j; q + 1 < m; ++q) {
            D.ext[2 * q] = D.ext[2 * q + 2];
            D.ext[2 * q + 1] = D.ext[2 * q + 3];
        }
        --m;
    }
    D.cnt[3] = m;
}

__device__ __forceinline__ void dr_log(uint64_t *log, unsigned long long *row, uint64_t cap,
                                       uint32_t *overflow, uint64_t a, uint64_t b, uint64_t c,
                                       uint64_t d, uint64_t e) {
    const uint64_t r = *row;
    if (r >= cap) {
        *overflow = 1;
        return;
    }
    uint64_t *p = log + 5 * r;
    p[0] = a;
    p[1] = b;
    p[2] = c;
    p[3] = d;
    p[4] = e;
    *row = r + 1;
}

// The copier's move for one round (one thread): the host copier's rules.
__global__ void k_dr_copier(const DrDev D, uint64_t quota, uint64_t round) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint64_t left = quota, moved = 0;
    uint32_t nc = 0, cur = D.cnt[2];
    const bool restore = D.mode == 1;
    while (left > 0) {
        while (cur < D.n && D.state[cur] == kDrDone) ++cur;
        if (cur >= D.n) break;
        const uint32_t i = cur;
        if (restore && D.flags[i]) {          // restored on demand: skip
            D.state[i] = kDrDone;
            continue;
        }
        const uint64_t sz = D.size[i], cp = D.copied[i];
        const uint64_t take = min(min(D.chunk, sz - cp), left);
        if (take == 0) break;
        if (nc >= D.cap_c) {                  // cannot happen with the begin-time capacity
            D.cnt[4] = 1;
            break;
        }
        const bool last = cp + take == sz;
        phos_copy_t d;
        d.len = take;
        d.buf = i;
        const uint64_t sh = restore ? 0 : D.shadow[i];
        if (restore) {
            d.src_off = D.img_off[i] + cp;
            d.dst_off = cp;
            d.flags = PHOS_COPY_IMAGE_TO_LIVE | (last && D.mark_present ? PHOS_COPY_MARK_PRESENT : 0);
        } else if (sh) {
            d.src_off = sh - 1 + cp;
            d.dst_off = D.img_off[i] + cp;
            d.flags = PHOS_COPY_STAGING_TO_IMAGE;
        } else {
            d.src_off = cp;
            d.dst_off = D.img_off[i] + cp;
            d.flags = PHOS_COPY_LIVE_TO_IMAGE;
        }
        D.lc[nc++] = d;
        dr_log(D.log_c, &D.ctr[0], D.cap_lc, &D.cnt[4], round, i, cp, take, sh ? 1 : 0);
        D.copied[i] = cp + take;
        moved += take;
        const uint64_t charge = a256(take);
        left = charge >= left ? 0 : left - charge;
        D.state[i] = last ? kDrDone : kDrInflight;
        if (last) {
            if (restore) {
                D.flags[i] = 1;
            } else if (sh) {
                // the drain precedes any later reuse in stream order
                dr_release(D, sh - 1, a256(sz));
                D.shadow[i] = 0;
            }
        }
    }
    D.cnt[0] = nc;
    D.cnt[2] = cur;
    D.ctr[2] += moved;
}

// Restore: the need set of one kernel (perm != 0, not restored), ascending.
__global__ void __launch_bounds__(1024) k_dr_need(const DrDev D, const uint8_t *perm,
                                                 uint64_t round) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_base;
    __shared__ unsigned long long s_bytes;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_base = 0;
        s_bytes = 0;
    }
    __syncthreads();
    const uint64_t row0 = D.ctr[1];
    for (uint32_t b0 = 0; b0 < D.n; b0 += blockDim.x) {
        const uint32_t i = b0 + tid;
        const bool c = i < D.n && perm[i] && !D.flags[i];
        const uint32_t bal = __ballot_sync(0xffffffffu, c);
        if (lane == 0) s_warp[warp] = __popc(bal);
        __syncthreads();
        uint32_t woff = 0, total = 0;
        for (uint32_t q = 0; q < (blockDim.x >> 5); ++q) {
            if (q < warp) woff += s_warp[q];
            total += s_warp[q];
        }
        const uint32_t pos = s_base + woff + __popc(bal & ((1u << lane) - 1));
        if (c) {
            const uint64_t cp = D.copied[i], sz = D.size[i];
            phos_copy_t d;
            d.src_off = D.img_off[i] + cp;
            d.dst_off = cp;
            d.len = sz - cp;
            d.buf = i;
            d.flags = PHOS_COPY_IMAGE_TO_LIVE | (D.mark_present ? PHOS_COPY_MARK_PRESENT : 0);
            D.la[pos] = d;
            const uint64_t r = row0 + pos;
            if (r < (uint64_t)D.n + 1) {
                uint64_t *p = D.log_a + 5 * r;
                p[0] = round;
                p[1] = i;
                p[2] = cp;
                p[3] = sz - cp;
                p[4] = 0;
            } else {
                D.cnt[4] = 1;
            }
            atomicAdd(&s_bytes, (unsigned long long)(sz - cp));
            D.copied[i] = sz;
            D.state[i] = kDrDone;
            D.flags[i] = 1;
        }
        __syncthreads();
        if (tid == 0) s_base += total;
        __syncthreads();
    }
    if (tid == 0) {
        D.cnt[1] = s_base;
        D.ctr[1] = row0 + s_base;
        D.ctr[5] += s_bytes;
    }
}

// CoW: the CoW set of one kernel (perm has W, not done, not shadowed).
__global__ void __launch_bounds__(1024) k_dr_cow(const DrDev D, const uint8_t *perm,
                                                uint64_t round) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_base;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_base = 0;
    __syncthreads();
    // candidates in ascending order
    for (uint32_t b0 = 0; b0 < D.n; b0 += blockDim.x) {
        const uint32_t i = b0 + tid;
        const bool c = i < D.n && (perm[i] & PHOS_PERM_W) && D.state[i] != kDrDone &&
                       D.shadow[i] == 0;
        const uint32_t bal = __ballot_sync(0xffffffffu, c);
        if (lane == 0) s_warp[warp] = __popc(bal);
        __syncthreads();
        uint32_t woff = 0, total = 0;
        for (uint32_t q = 0; q < (blockDim.x >> 5); ++q) {
            if (q < warp) woff += s_warp[q];
            total += s_warp[q];
        }
        if (c) D.cand[s_base + woff + __popc(bal & ((1u << lane) - 1))] = i;
        __syncthreads();
        if (tid == 0) s_base += total;
        __syncthreads();
    }
    // staging first fit in that order (one thread)
    if (tid == 0) {
        const uint32_t m = s_base;
        for (uint32_t k = 0; k < m; ++k) {
            const uint32_t i = D.cand[k];
            const uint64_t sz = D.size[i];
            phos_copy_t d;
            d.buf = i;
            uint64_t off;
            if (dr_alloc(D, a256(sz), &off)) {
                D.shadow[i] = off + 1;
                d.src_off = 0;
                d.dst_off = off;
                d.len = sz;
                d.flags = PHOS_COPY_LIVE_TO_STAGING;
                dr_log(D.log_a, &D.ctr[1], (uint64_t)D.n + 1, &D.cnt[4], round, i, 1, off, sz);
                D.ctr[3] += sz;
            } else {
                const uint64_t cp = D.copied[i];
                d.src_off = cp;
                d.dst_off = D.img_off[i] + cp;
                d.len = sz - cp;
                d.flags = PHOS_COPY_LIVE_TO_IMAGE;
                dr_log(D.log_a, &D.ctr[1], (uint64_t)D.n + 1, &D.cnt[4], round, i, 2, cp,
                       sz - cp);
                D.ctr[4] += sz - cp;
                D.copied[i] = sz;
                D.state[i] = kDrDone;
            }
            D.la[k] = d;
        }
        D.cnt[1] = m;
    }
    __syncthreads();
    // the rule's flags: done or shadowed when the kernel runs
    for (uint32_t i = tid; i < D.n; i += blockDim.x)
        D.flags[i] = D.state[i] == kDrDone || D.shadow[i] != 0;
}

}  // namespace phos

using namespace phos;

phos_status DevRounds::init(const phos_table *tt, uint32_t mode_, uint64_t chunk,
                            uint64_t staging_bytes, bool mark_present, cudaStream_t s) {
    t = tt;
    mode = mode_;
    const uint32_t n = t->n, nn = std::max(n, 1u);
    cap_c = (uint32_t)std::min<uint64_t>(t->image_bytes / chunk + n + 2, 1ull << 30);
    cap_lc = t->image_bytes / chunk + 2ull * n + (1ull << 16);
    // one device allocation, every array 256-byte aligned
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t o_state = take(nn), o_copied = take(8ull * nn), o_shadow = take(8ull * nn),
                 o_flags = take(nn), o_ext = take(16ull * (nn + 2)), o_cand = take(4ull * nn),
                 o_imgoff = take(8ull * nn), o_lc = take(sizeof(phos_copy_t) * cap_c),
                 o_la = take(sizeof(phos_copy_t) * nn), o_cnt = take(64),
                 o_logc = take(40ull * cap_lc), o_loga = take(40ull * (nn + 1)),
                 o_ctr = take(64);
    PHOS_CUDA(cudaMalloc(&mem, off));
    uint8_t *b = static_cast<uint8_t *>(mem);
    DrDev &D = *reinterpret_cast<DrDev *>(dev);
    static_assert(sizeof(DrDev) <= sizeof(dev), "DevRounds::dev too small");
    D.n = n;
    D.mode = mode;
    D.chunk = chunk;
    D.staging_bytes = staging_bytes;
    D.size = t->view.size;
    D.state = b + o_state;
    D.copied = reinterpret_cast<uint64_t *>(b + o_copied);
    D.shadow = reinterpret_cast<uint64_t *>(b + o_shadow);
    D.flags = b + o_flags;
    D.ext = reinterpret_cast<uint64_t *>(b + o_ext);
    D.cand = reinterpret_cast<uint32_t *>(b + o_cand);
    D.img_off = reinterpret_cast<const uint64_t *>(b + o_imgoff);
    D.lc = reinterpret_cast<phos_copy_t *>(b + o_lc);
    D.la = reinterpret_cast<phos_copy_t *>(b + o_la);
    D.cnt = reinterpret_cast<uint32_t *>(b + o_cnt);
    D.log_c = reinterpret_cast<uint64_t *>(b + o_logc);
    D.log_a = reinterpret_cast<uint64_t *>(b + o_loga);
    D.ctr = reinterpret_cast<unsigned long long *>(b + o_ctr);
    D.cap_c = cap_c;
    D.cap_lc = cap_lc;
    D.mark_present = mark_present ? 1u : 0u;
    PHOS_CUDA(cudaMemsetAsync(mem, 0, off, s));
    if (n) PHOS_CUDA(cudaMemcpyAsync(b + o_imgoff, t->img_off.data(), 8ull * n,
                                     cudaMemcpyHostToDevice, s));
    // staging: one free extent
    uint64_t e0[2] = {0, staging_bytes};
    uint32_t c0[8] = {0, 0, 0, staging_bytes ? 1u : 0u, 0, 0, 0, 0};
    PHOS_CUDA(cudaMemcpyAsync(D.ext, e0, sizeof e0, cudaMemcpyHostToDevice, s));
    PHOS_CUDA(cudaMemcpyAsync(D.cnt, c0, sizeof c0, cudaMemcpyHostToDevice, s));
    // the host arrays above are on this stack frame: wait for the uploads
    PHOS_CUDA(cudaStreamSynchronize(s));
    return PHOS_OK;
}

DevRounds::~DevRounds() {
    if (mem) cudaFree(mem);
}

namespace phos {
__global__ void k_dr_all(const DrDev D) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < D.n;
         i += gridDim.x * blockDim.x) {
        D.state[i] = kDrDone;
        D.copied[i] = D.size[i];
        D.shadow[i] = 0;
        D.flags[i] = 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) D.cnt[2] = D.n;
}
}  // namespace phos

phos_status DevRounds::mark_all(cudaStream_t s) {
    const DrDev &D = *reinterpret_cast<const DrDev *>(dev);
    k_dr_all<<<std::max<uint32_t>(1, std::min<uint32_t>((t->n + 255) / 256, 148)), 256, 0, s>>>(D);
    count_launch();
    PHOS_CUDA(cudaGetLastError());
    return PHOS_OK;
}

const uint8_t *DevRounds::flags() const {
    return reinterpret_cast<const DrDev *>(dev)->flags;
}

phos_status DevRounds::copier(uint64_t quota, uint64_t round, void *staging,
                              uint64_t staging_bytes, const void *image, uint64_t image_bytes,
                              uint32_t *d_present, uint32_t *d_status, cudaStream_t s) {
    const DrDev &D = *reinterpret_cast<const DrDev *>(dev);
    k_dr_copier<<<1, 32, 0, s>>>(D, quota, round);
    count_launch();
    PHOS_CUDA(cudaGetLastError());
    return copy_device_count(t, D.lc, D.cap_c, D.cnt + 0, staging, staging_bytes, image,
                             image_bytes, d_present, d_status, s);
}

phos_status DevRounds::action(const uint8_t *d_perm, uint64_t round, void *staging,
                              uint64_t staging_bytes, const void *image, uint64_t image_bytes,
                              uint32_t *d_present, uint32_t *d_status, cudaStream_t s) {
    const DrDev &D = *reinterpret_cast<const DrDev *>(dev);
    if (!t->n) return PHOS_OK;
    if (mode == 1)
        k_dr_need<<<1, 1024, 0, s>>>(D, d_perm, round);
    else
        k_dr_cow<<<1, 1024, 0, s>>>(D, d_perm, round);
    count_launch();
    PHOS_CUDA(cudaGetLastError());
    return copy_device_count(t, D.la, std::max(t->n, 1u), D.cnt + 1, staging, staging_bytes,
                             image, image_bytes, d_present, d_status, s);
}

phos_status DevRounds::collect(std::vector<uint64_t> &copier_log, std::vector<uint64_t> &act_log,
                               uint64_t out[6], std::vector<uint8_t> *state) {
    const DrDev &D = *reinterpret_cast<const DrDev *>(dev);
    unsigned long long ctr[8];
    uint32_t cnt[8];
    PHOS_CUDA(cudaMemcpy(ctr, D.ctr, sizeof ctr, cudaMemcpyDeviceToHost));
    PHOS_CUDA(cudaMemcpy(cnt, D.cnt, sizeof cnt, cudaMemcpyDeviceToHost));
    if (cnt[4]) return fail(PHOS_ENOMEM, "device rounds: log capacity exceeded");
    copier_log.resize(5 * ctr[0]);
    act_log.resize(5 * ctr[1]);
    if (ctr[0])
        PHOS_CUDA(cudaMemcpy(copier_log.data(), D.log_c, 40ull * ctr[0], cudaMemcpyDeviceToHost));
    if (ctr[1])
        PHOS_CUDA(cudaMemcpy(act_log.data(), D.log_a, 40ull * ctr[1], cudaMemcpyDeviceToHost));
    for (int k = 0; k < 6; ++k) out[k] = ctr[k];
    if (state && t->n) {
        state->resize(t->n);
        PHOS_CUDA(cudaMemcpy(state->data(), D.state, t->n, cudaMemcpyDeviceToHost));
    }
    return PHOS_OK;
}
