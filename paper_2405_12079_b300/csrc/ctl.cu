// Host control plane: lockstep drivers of soft copy-on-write (PhoenixOS
// Sec. 4.2), soft recopy (Sec. 4.3) and soft on-demand concurrent restore
// (Sec. 6).  The state machines run on the host (buffer states, the CoW
// shadow map, the dirty set, the present set); every byte moves through
// the copy engine and every trace through the validator, on the caller's
// stream.  Copy lists and each round's perm and rule-flag slot are staged
// in pinned host arenas and reach the device as kernel parameters
// (push_small: no copy-engine upload to queue behind the copier's DMA
// copies); the arenas are recycled at stream synchronisations.
//
// No-sync checkpoint sessions (PHOS_CKPT_NO_SYNC) take that round trip out:
// after_kernel enqueues the validation, whose last CTA (or, after the ring
// variant, a one-CTA rule kernel) applies the protocol's response on the
// device (recopy: store victims that were in flight or done become dirty;
// CoW: the first round with a store victim neither done nor shadowed is
// recorded and published to a mapped host word), and returns at once.  Every host decision of a round
// (copier pieces, CoW set, staging, dirty marks of speculated writes)
// depends only on the speculation and on earlier host decisions, never on
// a validation result, so the host can run ahead of the device; it learns
// of a CoW mis-speculation from the mapped word at its next call, and at
// the latest at finish, which then copies every buffer stop-the-world.
// With PHOS_CKPT_DEFER a no-sync session goes one step further: after_kernel
// only queues the round (trace, perm slot, rule-flag slot, round number),
// and up to kMaxRounds queued rounds are validated in one launch
// (validate_rounds) -- when the queue is full, and before anything that
// reads the rule's results or recycles the upload arena.
#include <limits.h>
#include <math.h>
#include <string.h>

#include <cmath>

#include <algorithm>
#include <deque>
#include <vector>

#include "internal.h"

namespace phos {

enum : uint8_t { kPending = 0, kInflight = 1, kDone = 2 };

// Host-leg pieces of at least this many bytes go to the DMA engines
// (cudaMemcpyAsync) instead of the SM copy kernel; 0 = never.  SM-issued
// stores reach the host in small PCIe write packets (measured 12 % link
// overhead, 52.8 GB/s of payload) while the copy engines deliver 57.3 GB/s
// on the same link.  With 5 MB copier batches a 1 MiB threshold left each
// batch's sub-MiB remainder to a copy launch pair on the copier stream
// (47.8 GB/s for the copier alone); from 256 KiB up the engines take it
// (55.5 GB/s), and pieces below it stay batched in one launch.
static uint64_t g_dma_min = 256ull << 10;

// Copier window of concurrent sessions (phos_copier_window): 0 = the host
// issues copier batches as fast as the rounds go; else an advance first
// waits until at most this many bytes of earlier batches are in flight.
static uint64_t g_copier_window = 0;

// First fit over free extents sorted by offset, coalesced on release.
struct FirstFit {
    std::vector<std::pair<uint64_t, uint64_t>> free;  // (off, len)
    explicit FirstFit(uint64_t total) {
        if (total) free.push_back({0, total});
    }
    bool alloc(uint64_t need, uint64_t *off) {
        for (size_t j = 0; j < free.size(); ++j) {
            if (free[j].second >= need) {
                *off = free[j].first;
                if (free[j].second == need)
                    free.erase(free.begin() + j);
                else
                    free[j] = {free[j].first + need, free[j].second - need};
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t len) {
        auto it = std::lower_bound(free.begin(), free.end(), std::make_pair(off, (uint64_t)0));
        it = free.insert(it, {off, len});
        size_t j = it - free.begin();
        if (j + 1 < free.size() && free[j].first + free[j].second == free[j + 1].first) {
            free[j].second += free[j + 1].second;
            free.erase(free.begin() + j + 1);
        }
        if (j > 0 && free[j - 1].first + free[j - 1].second == free[j].first) {
            free[j - 1].second += free[j].second;
            free.erase(free.begin() + j);
        }
    }
};

// One kernel's validation outcome applied on the device (no-sync sessions).
// victim_st: the validation's store-victim bitmap (restore: its victim
// bitmap of any access); flags[i]: recopy, the buffer was in flight or done
// when the kernel ran (touched); CoW, it was done or shadowed (safe);
// restore, it was restored (present and landed).  cow = 1 for the
// mis-speculation rule of CoW and restore.  acc: u64[8] device words, [0..2] the
// validation's counts, [3] running violation total, [4] first mis-speculated
// round (-1 = none).  One CTA.
__global__ void k_rule(const uint32_t *victim_st, const uint8_t *flags, uint32_t n, int cow,
                       int64_t round, uint8_t *dirty, uint64_t *acc, int64_t *h_flag) {
    __shared__ int hit;
    if (threadIdx.x == 0) hit = 0;
    __syncthreads();
    const uint32_t nvw = (n + 31) / 32;
    for (uint32_t w = threadIdx.x; w < nvw; w += blockDim.x) {
        uint32_t v = victim_st[w];
        while (v) {
            const uint32_t i = w * 32 + (uint32_t)(__ffs(v) - 1);
            v &= v - 1;
            if (i >= n) break;
            if (cow) {
                if (!flags[i]) hit = 1;
            } else if (flags[i]) {
                dirty[i] = 1;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        acc[3] += acc[0];
        if (cow && hit && (int64_t)acc[4] < 0) {
            // rounds run in stream order: the first one to get here wins
            acc[4] = (uint64_t)round;
            *(volatile int64_t *)h_flag = round;
            __threadfence_system();
        }
    }
}

// Device and pinned resources shared by the sessions.
struct Session {
    const phos_table *t = nullptr;
    cudaStream_t s = nullptr;
    uint32_t n = 0, w = 4;
    uint64_t chunk = 4ull << 20;
    // pinned host arena for copy lists (recycled at synchronisations); the
    // host arenas are mapped and reach the device by push_small
    phos_copy_t *h_list = nullptr;
    const phos_copy_t *h_list_dev = nullptr;
    size_t h_cap = 0, h_used = 0;
    phos_copy_t *d_list = nullptr;
    size_t d_cap = 0;
    // validator I/O
    uint8_t *h_perm = nullptr, *d_perm = nullptr;
    const uint8_t *h_perm_dev = nullptr;
    uint32_t *d_bitmap = nullptr;
    uint64_t bitmap_words = 0;
    uint64_t *h_count = nullptr;      // pinned mapped: count[3]
    uint32_t *h_victim = nullptr;     // pinned mapped: victim | victim_st
    uint32_t *h_status = nullptr;     // pinned mapped
    uint64_t *d_count = nullptr;
    uint32_t *d_victim = nullptr, *d_status = nullptr;
    // copier
    std::vector<uint8_t> state;
    std::vector<uint64_t> copied;
    uint32_t cursor = 0;
    uint64_t round = 0;
    std::vector<uint64_t> copier_log;
    uint64_t validated = 0, violations = 0;
    // no-sync sessions: per-round perm | flags slots in a pinned upload
    // arena (recycled at synchronisations), validation outputs and rule
    // state in device memory, the mis-speculation word mapped
    bool nosync = false;
    // device-decided rounds: the round's perm and rule flags on the device
    const uint8_t *perm_dev = nullptr, *flags_dev = nullptr;
    uint8_t *h_up = nullptr, *d_up = nullptr;
    const uint8_t *h_up_dev = nullptr;  // h_up's device-mapped address
    size_t up_cap = 0, up_used = 0, slot = 0;
    uint64_t *d_acc = nullptr;      // u64[8], see k_rule
    uint32_t *d_vic = nullptr;      // victim | victim_st
    uint8_t *d_dirty = nullptr;     // u8[n]
    int64_t *h_flag = nullptr, *d_flag = nullptr;
    // deferred validation (PHOS_CKPT_DEFER): rounds queued for one launch;
    // traces longer than kDeferMaxRec records are validated at once by the
    // streaming kernel, which is the faster one at that length
    static constexpr uint64_t kDeferMaxRec = 1ull << 24;
    uint32_t defer_k = 0;            // rounds per launch, 0 = validate at once
    uint32_t defer_rule = 0;         // ProtoRule kind of the queued rounds
    std::vector<RoundSeg> pend;
    void *d_rscratch = nullptr;
    // concurrent sessions: the copier's own stream, a clone of the table
    // (its own copy-engine scratch), one event per copier batch, kept until
    // that batch has completed (batches complete in order on the copier
    // stream; an event is reused only once its batch is known complete, so
    // a wait never lands on a later batch than the one it names)
    cudaStream_t cs = nullptr;
    phos_table_t *tc = nullptr;
    cudaEvent_t app_ev = nullptr;
    struct Batch {
        uint64_t b, bytes;
        cudaEvent_t ev;
    };
    std::deque<Batch> bq;               // in flight, ascending
    std::vector<cudaEvent_t> ev_free;
    uint64_t batch_done = 0;            // every batch <= this has completed
    uint64_t batch = 0;                 // copier batches issued on cs
    uint64_t inflight_bytes = 0;        // bytes of the batches in bq
    std::vector<uint64_t> last_batch;   // per buffer: batch of its last piece

    phos_status init(const phos_table *tt, cudaStream_t ss, uint32_t ww, uint64_t ch) {
        t = tt;
        s = ss;
        n = tt->n;
        w = ww;
        chunk = ch;
        state.assign(n, kPending);
        copied.assign(n, 0);
        const uint32_t nvw = (n + 31) / 32;
        PHOS_CUDA(cudaHostAlloc(&h_perm, std::max(n, 1u), cudaHostAllocMapped));
        PHOS_CUDA(cudaHostGetDevicePointer((void **)&h_perm_dev, h_perm, 0));
        PHOS_CUDA(cudaMalloc(&d_perm, std::max(n, 1u)));
        PHOS_CUDA(cudaHostAlloc(&h_count, 64, cudaHostAllocMapped));
        PHOS_CUDA(cudaHostAlloc(&h_victim, 8ull * std::max(nvw, 1u), cudaHostAllocMapped));
        PHOS_CUDA(cudaHostAlloc(&h_status, 64, cudaHostAllocMapped));
        PHOS_CUDA(cudaHostGetDevicePointer((void **)&d_count, h_count, 0));
        PHOS_CUDA(cudaHostGetDevicePointer((void **)&d_victim, h_victim, 0));
        PHOS_CUDA(cudaHostGetDevicePointer((void **)&d_status, h_status, 0));
        *h_status = 0;
        return reserve_list(1024);
    }

    phos_status init_nosync() {
        nosync = true;
        const uint32_t nvw = std::max((n + 31) / 32, 1u);
        PHOS_CUDA(cudaMalloc(&d_acc, 64));
        PHOS_CUDA(cudaMalloc(&d_vic, 8ull * nvw));
        PHOS_CUDA(cudaMalloc(&d_dirty, std::max(n, 1u)));
        PHOS_CUDA(cudaHostAlloc(&h_flag, 64, cudaHostAllocMapped));
        PHOS_CUDA(cudaHostGetDevicePointer((void **)&d_flag, h_flag, 0));
        *(volatile int64_t *)h_flag = -1;
        uint64_t a0[8] = {0, 0, 0, 0, ~0ull, 0, 0, 0};
        PHOS_CUDA(cudaMemcpy(d_acc, a0, sizeof a0, cudaMemcpyHostToDevice));
        PHOS_CUDA(cudaMemset(d_dirty, 0, std::max(n, 1u)));
        return reserve_list(65536);
    }

    // Deferred validation (after init_nosync); a table too large for even
    // two rounds per launch keeps validating at once.
    phos_status init_defer() {
        defer_k = rounds_cap(n, t->device);
        if (!defer_k) return PHOS_OK;
        const size_t b = rounds_scratch_bytes(n, kMaxRounds);
        PHOS_CUDA(cudaMalloc(&d_rscratch, b));
        PHOS_CUDA(cudaMemset(d_rscratch, 0, b));
        pend.reserve(kMaxRounds);
        return PHOS_OK;
    }

    // Validate the queued rounds (one launch, on the caller's stream).
    phos_status flush_pending() {
        if (pend.empty()) return PHOS_OK;
        phos_status r = validate_rounds(t, pend.data(), (uint32_t)pend.size(), w, defer_rule,
                                        d_dirty, d_acc, d_flag, d_status, d_rscratch, s);
        pend.clear();
        return r;
    }

    phos_status init_concurrent() {
        phos_status r = init_nosync();
        if (r) return r;
        PHOS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        std::vector<phos_buf_t> b(n);
        for (uint32_t i = 0; i < n; ++i) b[i] = phos_buf_t{t->base[i], t->size[i]};
        r = phos_table_create(b.data(), n, &tc);
        if (r) return r;
        PHOS_CUDA(cudaEventCreateWithFlags(&app_ev, cudaEventDisableTiming));
        last_batch.assign(n, 0);
        return PHOS_OK;
    }

    // Both streams (the upload and list arenas are shared by them); queued
    // rounds are validated first (their slots live in the upload arena).
    cudaError_t sync_streams() {
        if (!pend.empty() && flush_pending() != PHOS_OK) return cudaErrorLaunchFailure;
        cudaError_t e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && cs) e = cudaStreamSynchronize(cs);
        return e;
    }

    void retire_front() {
        batch_done = bq.front().b;
        inflight_bytes -= bq.front().bytes;
        ev_free.push_back(bq.front().ev);
        bq.pop_front();
    }

    // Retire the batches that have completed; then, with a copier window,
    // wait (on the host) until at most `window` bytes are in flight.
    phos_status retire_batches() {
        while (!bq.empty()) {
            const cudaError_t q = cudaEventQuery(bq.front().ev);
            if (q == cudaErrorNotReady) {
                cudaGetLastError();
                break;
            }
            if (q != cudaSuccess) return cuda_fail(q, "copier batch event");
            retire_front();
        }
        while (g_copier_window && inflight_bytes > g_copier_window && !bq.empty()) {
            PHOS_CUDA(cudaEventSynchronize(bq.front().ev));
            retire_front();
        }
        return PHOS_OK;
    }

    // Record the event of copier batch b (b = the previous batch + 1, bytes
    // its payload) on the copier stream.
    phos_status record_batch(uint64_t b, uint64_t bytes) {
        cudaEvent_t e;
        if (ev_free.empty()) {
            PHOS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        } else {
            e = ev_free.back();
            ev_free.pop_back();
        }
        PHOS_CUDA(cudaEventRecord(e, cs));
        bq.push_back({b, bytes, e});
        inflight_bytes += bytes;
        batch = b;
        return PHOS_OK;
    }

    // Make the caller's stream wait for copier batch b (and so for every
    // earlier one).
    phos_status app_wait(uint64_t b) {
        if (!b || b <= batch_done || bq.empty() || b < bq.front().b) return PHOS_OK;
        const uint64_t k = std::min<uint64_t>(b - bq.front().b, bq.size() - 1);
        PHOS_CUDA(cudaStreamWaitEvent(s, bq[k].ev, 0));
        return PHOS_OK;
    }

    // A 256-aligned slot of `bytes` in the upload arena.
    phos_status alloc_up(size_t bytes, size_t *off) {
        bytes = align_up(std::max<size_t>(bytes, 1), 256);
        if (up_used + bytes > up_cap) {
            PHOS_CUDA(sync_streams());
            h_used = 0;
            up_used = 0;
            if (bytes > up_cap) {
                if (h_up) cudaFreeHost(h_up);
                if (d_up) cudaFree(d_up);
                h_up = nullptr;
                d_up = nullptr;
                const size_t cap = std::max<size_t>({bytes * 64, 2 * up_cap, 1 << 20});
                PHOS_CUDA(cudaHostAlloc(&h_up, cap, cudaHostAllocMapped));
                PHOS_CUDA(cudaHostGetDevicePointer((void **)&h_up_dev, h_up, 0));
                PHOS_CUDA(cudaMalloc(&d_up, cap));
                up_cap = cap;
            }
        }
        *off = up_used;
        up_used += bytes;
        return PHOS_OK;
    }

    ~Session() {
        if (s) cudaStreamSynchronize(s);
        if (cs) {
            cudaStreamSynchronize(cs);
            cudaStreamDestroy(cs);
        }
        if (tc) phos_table_destroy(tc);
        if (app_ev) cudaEventDestroy(app_ev);
        for (auto &be : bq) cudaEventDestroy(be.ev);
        for (cudaEvent_t e : ev_free) cudaEventDestroy(e);
        if (h_up) cudaFreeHost(h_up);
        if (d_up) cudaFree(d_up);
        if (d_acc) cudaFree(d_acc);
        if (d_vic) cudaFree(d_vic);
        if (d_dirty) cudaFree(d_dirty);
        if (d_rscratch) cudaFree(d_rscratch);
        if (h_flag) cudaFreeHost(h_flag);
        if (h_list) cudaFreeHost(h_list);
        if (d_list) cudaFree(d_list);
        if (h_perm) cudaFreeHost(h_perm);
        if (d_perm) cudaFree(d_perm);
        if (d_bitmap) cudaFree(d_bitmap);
        if (h_count) cudaFreeHost(h_count);
        if (h_victim) cudaFreeHost(h_victim);
        if (h_status) cudaFreeHost(h_status);
    }

    phos_status reserve_list(size_t need) {
        if (need <= h_cap) return PHOS_OK;
        size_t cap = std::max(need, 2 * h_cap);
        if (h_list) {
            PHOS_CUDA(sync_streams());
            cudaFreeHost(h_list);
            cudaFree(d_list);
            h_used = 0;
        }
        PHOS_CUDA(cudaHostAlloc(&h_list, cap * sizeof(phos_copy_t), cudaHostAllocMapped));
        PHOS_CUDA(cudaHostGetDevicePointer((void **)&h_list_dev, h_list, 0));
        PHOS_CUDA(cudaMalloc(&d_list, cap * sizeof(phos_copy_t)));
        h_cap = d_cap = cap;
        return PHOS_OK;
    }

    // Launch one batch through the copy engine.  With DMA enabled, host-leg
    // pieces of at least g_dma_min bytes become cudaMemcpyAsync calls issued
    // first; their present marks ride in the kernel batch that follows on
    // the same stream (a zero-length descriptor), so no bit precedes its
    // bytes.
    // copier = true in a concurrent session: on the copier's stream, through
    // the table clone.
    phos_status submit(const std::vector<phos_copy_t> &v0, void *staging, uint64_t staging_bytes,
                       const void *image, uint64_t image_bytes, uint32_t *present,
                       bool copier = false) {
        if (v0.empty()) return PHOS_OK;
        const bool on_cs = copier && cs;
        const cudaStream_t st = on_cs ? cs : s;
        const phos_table_t *tt = on_cs ? tc : t;
        std::vector<phos_copy_t> keep;
        const std::vector<phos_copy_t> *vp = &v0;
        if (g_dma_min) {
            keep.reserve(v0.size());
            for (const phos_copy_t &d : v0) {
                const uint32_t dir = d.flags & PHOS_COPY_DIR_MASK;
                const bool host_leg = dir == PHOS_COPY_LIVE_TO_IMAGE ||
                                      dir == PHOS_COPY_STAGING_TO_IMAGE ||
                                      dir == PHOS_COPY_IMAGE_TO_LIVE;
                if (!host_leg || d.len < g_dma_min) {
                    keep.push_back(d);
                    continue;
                }
                const uint8_t *src;
                uint8_t *dst;
                if (dir == PHOS_COPY_LIVE_TO_IMAGE) {
                    src = reinterpret_cast<const uint8_t *>(t->base[d.buf] + d.src_off);
                    dst = static_cast<uint8_t *>(const_cast<void *>(image)) + d.dst_off;
                } else if (dir == PHOS_COPY_STAGING_TO_IMAGE) {
                    src = static_cast<const uint8_t *>(staging) + d.src_off;
                    dst = static_cast<uint8_t *>(const_cast<void *>(image)) + d.dst_off;
                } else {
                    src = static_cast<const uint8_t *>(image) + d.src_off;
                    dst = reinterpret_cast<uint8_t *>(t->base[d.buf] + d.dst_off);
                }
                PHOS_CUDA(cudaMemcpyAsync(dst, src, d.len, cudaMemcpyDefault, st));
                if (d.flags & PHOS_COPY_MARK_PRESENT) {
                    phos_copy_t m = d;
                    m.len = 0;
                    m.src_off = dir == PHOS_COPY_IMAGE_TO_LIVE ? d.src_off : 0;
                    m.dst_off = dir == PHOS_COPY_IMAGE_TO_LIVE ? d.dst_off : 0;
                    keep.push_back(m);
                }
            }
            vp = &keep;
            if (keep.empty()) return PHOS_OK;
        }
        const std::vector<phos_copy_t> &v = *vp;
        if (h_used + v.size() > h_cap) {
            PHOS_CUDA(sync_streams());
            h_used = 0;
            phos_status r = reserve_list(v.size());
            if (r) return r;
        }
        phos_copy_t *hp = h_list + h_used;
        phos_copy_t *dp = d_list + h_used;
        memcpy(hp, v.data(), v.size() * sizeof(phos_copy_t));
        phos_status rp = push_small(dp, hp, h_list_dev + h_used, v.size() * sizeof(phos_copy_t),
                                    st);
        if (rp) return rp;
        h_used += v.size();
        return phos_copy(tt, dp, (uint32_t)v.size(), staging, staging_bytes,
                         const_cast<void *>(image), image_bytes, present, d_status, st);
    }

    phos_status sync() {
        PHOS_CUDA(sync_streams());
        h_used = 0;
        up_used = 0;
        if (*h_status) return fail((phos_status)*h_status, "device reported %s",
                                   phos_status_name((phos_status)*h_status));
        return PHOS_OK;
    }

    // perm for the next kernel -> device (no-sync: into this round's slot,
    // uploaded with the round's flags by upload_slot)
    phos_status stage_perm(const uint8_t *perm) {
        if (!perm && n) return fail(PHOS_EINVAL, "perm is NULL");
        if (nosync) {
            phos_status r = alloc_up(2ull * n, &slot);
            if (r) return r;
            if (n) memcpy(h_up + slot, perm, n);
            return PHOS_OK;
        }
        if (n) {
            memcpy(h_perm, perm, n);
            phos_status r = push_small(d_perm, h_perm, h_perm_dev, n, s);
            if (r) return r;
        }
        return PHOS_OK;
    }

    phos_status upload_slot(const std::vector<uint8_t> &flags) {
        if (!n) return PHOS_OK;
        memcpy(h_up + slot + n, flags.data(), n);
        phos_status r = push_small(d_up + slot, h_up + slot, h_up_dev + slot, 2ull * n, s);
        if (r) return r;
        return PHOS_OK;
    }

    phos_status bitmap_for(uint64_t n_rec) {
        const uint64_t words = std::max<uint64_t>((n_rec + 31) / 32, 1);
        if (words > bitmap_words) {
            PHOS_CUDA(sync_streams());
            h_used = 0;
            up_used = 0;
            if (d_bitmap) cudaFree(d_bitmap);
            PHOS_CUDA(cudaMalloc(&d_bitmap, words * 4));
            bitmap_words = words;
        }
        return PHOS_OK;
    }

    // Validate and apply the rule on the device; returns without waiting.
    // rule: 0 recopy (dirty marks), 1 CoW (store victims not safe), 2
    // restore (victims of any access not restored).
    phos_status validate_nosync(const uint64_t *d_trace, uint64_t n_rec, int rule) {
        // a long trace goes to the streaming kernel at once (after the
        // queued rounds, so the rule still sees rounds in order)
        if (defer_k && !perm_dev && n_rec > kDeferMaxRec) {
            phos_status rf = flush_pending();
            if (rf) return rf;
        } else if (defer_k && !perm_dev) {
            if (n_rec && !d_trace) return fail(PHOS_EINVAL, "validate: NULL trace");
            if (n_rec && ((uintptr_t)d_trace & 15))
                return fail(PHOS_EINVAL, "validate: trace must be 16-byte aligned");
            defer_rule = rule == 0 ? 1u : (rule == 1 ? 2u : 3u);
            // an empty trace has no victim: the rule would change nothing
            if (n_rec)
                pend.push_back(RoundSeg{d_trace, n_rec, d_up + slot, d_up + slot + n,
                                        (int64_t)round - 1});
            validated += n_rec;
            return pend.size() >= defer_k ? flush_pending() : PHOS_OK;
        }
        // growth synchronises: this round's slot is uploaded by then and
        // later uploads into its device copy are stream-ordered after the
        // validation below
        phos_status r0 = bitmap_for(n_rec);
        if (r0) return r0;
        const uint32_t nvw = std::max((n + 31) / 32, 1u);
        // the validation kernel's last CTA applies the rule when it can;
        // otherwise (ring variant, empty trace) k_rule does
        const uint8_t *pp = perm_dev ? perm_dev : d_up + slot;
        const uint8_t *ff = flags_dev ? flags_dev : d_up + slot + n;
        ProtoRule pr;
        pr.flags = ff;
        pr.dirty = d_dirty;
        pr.acc = d_acc;
        pr.h_flag = d_flag;
        pr.round = (int64_t)round - 1;
        pr.kind = rule == 0 ? 1u : (rule == 1 ? 2u : 3u);
        bool fused = false;
        phos_status r = validate_impl(t, pp, d_trace, n_rec, w, d_bitmap, d_acc, d_vic,
                                      d_vic + nvw, nullptr, 0, d_status, s, &pr, &fused);
        if (r) return r;
        if (!fused) {
            k_rule<<<1, 256, 0, s>>>(rule == 2 ? d_vic : d_vic + nvw, ff, n,
                                     rule ? 1 : 0, (int64_t)round - 1, d_dirty, d_acc, d_flag);
            PHOS_CUDA(cudaGetLastError());
            count_launch();
        }
        validated += n_rec;
        return PHOS_OK;
    }

    // No-sync: wait, then fold the device's violation total and dirty marks
    // into the host state (the device dirty marks are cleared).
    phos_status collect(std::vector<uint8_t> *dirty) {
        phos_status r = sync();
        if (r) return r;
        uint64_t acc[8];
        PHOS_CUDA(cudaMemcpy(acc, d_acc, sizeof acc, cudaMemcpyDeviceToHost));
        violations = acc[3];
        if (dirty && n) {
            std::vector<uint8_t> dd(n);
            PHOS_CUDA(cudaMemcpy(dd.data(), d_dirty, n, cudaMemcpyDeviceToHost));
            for (uint32_t i = 0; i < n; ++i) (*dirty)[i] |= dd[i];
            PHOS_CUDA(cudaMemset(d_dirty, 0, n));
        }
        return PHOS_OK;
    }

    int64_t flag() const { return *(volatile const int64_t *)h_flag; }

    // Validate and wait: fills h_count and h_victim (victim | victim_st).
    phos_status validate_sync(const uint64_t *d_trace, uint64_t n_rec) {
        phos_status r0 = bitmap_for(n_rec);
        if (r0) return r0;
        const uint32_t nvw = (n + 31) / 32;
        phos_status r = phos_validate(t, d_perm, d_trace, n_rec, w, d_bitmap, d_count, d_victim,
                                      d_victim + std::max(nvw, 1u), nullptr, 0, d_status, s);
        if (r) return r;
        r = sync();
        if (r) return r;
        validated += n_rec;
        violations += h_count[0];
        return PHOS_OK;
    }

    bool victim_bit(bool store_only, uint32_t i) const {
        const uint32_t nvw = std::max((n + 31) / 32, 1u);
        const uint32_t *v = h_victim + (store_only ? nvw : 0);
        return (v[i >> 5] >> (i & 31)) & 1u;
    }

    bool done() {
        while (cursor < n && state[cursor] == kDone) ++cursor;
        return cursor >= n;
    }

    // One copier advance; piece(i, off, len) appends a descriptor and
    // returns whether it came from a shadow; skip(i) marks i done untouched.
    template <typename Piece, typename Skip>
    uint64_t advance(uint64_t quota, Piece piece, Skip skip) {
        uint64_t left = quota, moved = 0;
        while (left > 0 && !done()) {
            const uint32_t i = cursor;
            if (skip(i)) {
                state[i] = kDone;
                continue;
            }
            const uint64_t rem = t->size[i] - copied[i];
            const uint64_t take = std::min(std::min(chunk, rem), left);
            if (take == 0) break;
            const bool sh = piece(i, copied[i], take);
            copier_log.insert(copier_log.end(), {round, i, copied[i], take, sh ? 1ull : 0ull});
            copied[i] += take;
            moved += take;
            const uint64_t charge = align_up(take, 256);
            left = charge >= left ? 0 : left - charge;
            state[i] = copied[i] == t->size[i] ? kDone : kInflight;
        }
        return moved;
    }
};

phos_status copy_log(const std::vector<uint64_t> &log, uint64_t *out, uint64_t cap,
                     uint64_t *n_out) {
    const uint64_t ev = log.size() / 5;
    if (n_out) *n_out = ev;
    if (out) memcpy(out, log.data(), 8 * 5 * std::min(ev, cap));
    return PHOS_OK;
}

}  // namespace phos

using namespace phos;

extern "C" phos_status phos_ckpt_frequency(double n, double f_fail, double o, double r,
                                           double t, double *f_opt, double *wasted) {
    if (!(n > 0) || !(f_fail > 0) || !(o > 0) || !(r >= 0) || !(t >= 0))
        return fail(PHOS_EINVAL, "ckpt_frequency: need N, F, O > 0 and R, T >= 0");
    const double fs = std::sqrt(n * f_fail / (2.0 * o));
    if (f_opt) *f_opt = fs;
    if (wasted) *wasted = n * f_fail * t * (r + n / (2.0 * fs)) + n * o * fs * t;
    return PHOS_OK;
}

extern "C" phos_status phos_copier_window(uint64_t bytes) {
    g_copier_window = bytes;
    return PHOS_OK;
}

extern "C" phos_status phos_host_copy_config(uint64_t dma_min_bytes) {
    g_dma_min = dma_min_bytes;
    return PHOS_OK;
}

struct phos_ckpt {
    Session ss;
    uint32_t mode = PHOS_CKPT_COW;
    void *staging = nullptr;
    uint64_t staging_bytes = 0;
    void *image = nullptr;
    uint64_t image_bytes = 0;
    FirstFit alloc{0};
    std::vector<int64_t> shadow;   // staging offset or -1
    std::vector<uint8_t> safe;     // CoW: done or shadowed when the kernel ran
    std::vector<uint8_t> touched;  // recopy: in flight or done when the kernel ran
    std::vector<uint8_t> dirty;
    std::vector<uint64_t> cow_log;
    std::vector<uint64_t> pass_log;
    uint64_t cow_bytes = 0, direct_bytes = 0, copier_bytes = 0, recopy_bytes = 0;
    int64_t misspec = -1;
    bool complete = false, finished = false, in_kernel = false;
    // concurrent: copier batch of the last staging release, and the latest
    // release batch the caller's stream has waited for
    uint64_t release_batch = 0, waited_release = 0;
    DevRounds *dr = nullptr;      // PHOS_CKPT_DEVICE: decisions on the device
    ~phos_ckpt() {
        ss.pend.clear();      // an ended session validates nothing more
        ss.sync_streams();
        delete dr;
    }
};

extern "C" phos_status phos_ckpt_begin(const phos_table_t *t, const phos_ckpt_desc_t *d,
                                       phos_stream_t stream, phos_ckpt_t **out) {
    if (!t || !d || !out) return fail(PHOS_EINVAL, "ckpt_begin: NULL argument");
    *out = nullptr;
    const uint32_t mode = d->mode & ~(uint32_t)(PHOS_CKPT_NO_SYNC | PHOS_CKPT_CONCURRENT |
                                                PHOS_CKPT_DEVICE | PHOS_CKPT_DEFER);
    if (mode != PHOS_CKPT_COW && mode != PHOS_CKPT_RECOPY)
        return fail(PHOS_EINVAL, "ckpt_begin: mode %u", d->mode);
    if ((d->mode & PHOS_CKPT_DEVICE) &&
        (mode != PHOS_CKPT_COW || (d->mode & PHOS_CKPT_CONCURRENT)))
        return fail(PHOS_EINVAL, "ckpt_begin: PHOS_CKPT_DEVICE is for CoW sessions, without "
                                 "PHOS_CKPT_CONCURRENT");
    if ((d->mode & PHOS_CKPT_DEFER) && (d->mode & PHOS_CKPT_DEVICE))
        return fail(PHOS_EINVAL, "ckpt_begin: PHOS_CKPT_DEFER goes without PHOS_CKPT_DEVICE");
    if (d->access_bytes == 0 || d->chunk == 0 || d->chunk % 256)
        return fail(PHOS_EINVAL, "ckpt_begin: access_bytes >= 1, chunk a multiple of 256");
    if (!d->image || d->image_bytes < t->image_bytes)
        return fail(PHOS_EINVAL, "ckpt_begin: image smaller than %llu bytes",
                    (unsigned long long)t->image_bytes);
    phos_ckpt *c = new phos_ckpt();
    phos_status r = c->ss.init(t, static_cast<cudaStream_t>(stream), d->access_bytes, d->chunk);
    if (r) {
        delete c;
        return r;
    }
    if ((d->mode & PHOS_CKPT_CONCURRENT) && (r = c->ss.init_concurrent())) {
        delete c;
        return r;
    }
    if ((d->mode & (PHOS_CKPT_NO_SYNC | PHOS_CKPT_DEVICE | PHOS_CKPT_DEFER)) && !c->ss.nosync &&
        (r = c->ss.init_nosync())) {
        delete c;
        return r;
    }
    if ((d->mode & PHOS_CKPT_DEFER) && (r = c->ss.init_defer())) {
        delete c;
        return r;
    }
    if (d->mode & PHOS_CKPT_DEVICE) {
        c->dr = new DevRounds();
        if ((r = c->dr->init(t, 2, d->chunk, d->d_staging ? d->staging_bytes : 0, false,
                             c->ss.s))) {
            delete c;
            return r;
        }
    }
    c->mode = mode;
    c->staging = mode == PHOS_CKPT_COW ? d->d_staging : nullptr;
    c->staging_bytes = c->staging ? d->staging_bytes : 0;
    c->image = d->image;
    c->image_bytes = d->image_bytes;
    c->alloc = FirstFit(c->staging_bytes);
    c->shadow.assign(t->n, -1);
    c->safe.assign(t->n, 0);
    c->touched.assign(t->n, 0);
    c->dirty.assign(t->n, 0);
    c->complete = t->n == 0;
    *out = c;
    return PHOS_OK;
}

static phos_status ckpt_advance(phos_ckpt *c, uint64_t quota) {
    Session &S = c->ss;
    const phos_table *t = S.t;
    std::vector<phos_copy_t> v;
    // concurrent: this batch runs on the copier's stream after everything
    // the caller has enqueued so far (the previous kernels and their CoW
    // copies); the kernels that follow wait for it only where they write
    const uint64_t b = S.batch + 1;
    if (S.cs) {
        phos_status r0 = S.retire_batches();
        if (r0) return r0;
        PHOS_CUDA(cudaEventRecord(S.app_ev, S.s));
        PHOS_CUDA(cudaStreamWaitEvent(S.cs, S.app_ev, 0));
    }
    uint64_t moved = S.advance(
        quota,
        [&](uint32_t i, uint64_t off, uint64_t len) {
            const int64_t sh = c->shadow[i];
            phos_copy_t d;
            d.len = len;
            d.buf = i;
            d.dst_off = t->img_off[i] + off;
            if (sh >= 0) {
                d.src_off = (uint64_t)sh + off;
                d.flags = PHOS_COPY_STAGING_TO_IMAGE;
            } else {
                d.src_off = off;
                d.flags = PHOS_COPY_LIVE_TO_IMAGE;
            }
            v.push_back(d);
            if (S.cs) S.last_batch[i] = b;
            if (off + len == t->size[i] && sh >= 0) {
                // the drain is stream-ordered before any later reuse (on
                // the copier's stream: a CoW copy into the extent waits
                // for this batch first)
                c->alloc.release((uint64_t)sh, align_up(t->size[i], 256));
                c->shadow[i] = -1;
                c->release_batch = b;
            }
            return sh >= 0;
        },
        [](uint32_t) { return false; });
    c->copier_bytes += moved;
    phos_status r = S.submit(v, c->staging, c->staging_bytes, c->image, c->image_bytes, nullptr,
                             true);
    if (r) return r;
    uint64_t vb = 0;
    for (const phos_copy_t &d : v) vb += d.len;
    if (S.cs && !v.empty() && (r = S.record_batch(b, vb))) return r;
    return PHOS_OK;
}

extern "C" phos_status phos_ckpt_advance(phos_ckpt_t *c, uint64_t quota, int *done) {
    if (!c) return fail(PHOS_EINVAL, "ckpt_advance: NULL session");
    if (c->in_kernel) return fail(PHOS_EINVAL, "ckpt_advance: inside a kernel round");
    phos_status r = PHOS_OK;
    if (c->dr) {
        // the device decides; the host only learns of a mis-speculation
        Session &S = c->ss;
        if (!c->complete && S.flag() >= 0) {
            c->misspec = S.flag();
            c->complete = true;
        }
        if (!c->complete)
            r = c->dr->copier(quota, S.round, c->staging, c->staging_bytes, c->image,
                              c->image_bytes, nullptr, S.d_status, S.s);
        if (done) *done = c->complete ? 1 : 0;
        return r;
    }
    if (c->ss.nosync && c->mode == PHOS_CKPT_COW && !c->complete && c->ss.flag() >= 0) {
        c->misspec = c->ss.flag();        // the device saw it; finish falls back
        c->complete = true;
    }
    if (!c->complete) {
        r = ckpt_advance(c, quota);
        if (c->ss.done()) c->complete = true;
    }
    if (done) *done = c->complete ? 1 : 0;
    return r;
}

extern "C" phos_status phos_ckpt_before_kernel(phos_ckpt_t *c, const uint8_t *perm) {
    if (!c) return fail(PHOS_EINVAL, "ckpt_before_kernel: NULL session");
    if (c->in_kernel) return fail(PHOS_EINVAL, "ckpt_before_kernel: after_kernel missing");
    if (c->complete) return fail(PHOS_EINVAL, "ckpt_before_kernel: checkpoint already complete");
    Session &S = c->ss;
    const phos_table *t = S.t;
    phos_status r = S.stage_perm(perm);
    if (r) return r;
    const uint32_t n = S.n;
    if (c->mode == PHOS_CKPT_COW) {
        if (S.cs) {
            // the kernel may not overwrite a buffer the copier still reads
            // live, nor a CoW copy land in staging a drain still reads
            uint64_t need = 0;
            for (uint32_t i = 0; i < n; ++i)
                if (perm[i] & PHOS_PERM_W) need = std::max(need, S.last_batch[i]);
            if (c->release_batch > c->waited_release) {
                need = std::max(need, c->release_batch);
                c->waited_release = c->release_batch;
            }
            r = S.app_wait(need);
            if (r) return r;
        }
        std::vector<phos_copy_t> v;
        for (uint32_t i = 0; i < n; ++i) {
            if (!(perm[i] & PHOS_PERM_W)) continue;
            if (S.state[i] == kDone || c->shadow[i] >= 0) continue;
            const uint64_t sz = t->size[i];
            uint64_t off;
            phos_copy_t d;
            d.buf = i;
            if (c->alloc.alloc(align_up(sz, 256), &off)) {
                c->shadow[i] = (int64_t)off;
                d.src_off = 0;
                d.dst_off = off;
                d.len = sz;
                d.flags = PHOS_COPY_LIVE_TO_STAGING;
                c->cow_log.insert(c->cow_log.end(), {S.round, i, 1ull, off, sz});
                c->cow_bytes += sz;
            } else {
                const uint64_t cp = S.copied[i];
                d.src_off = cp;
                d.dst_off = t->img_off[i] + cp;
                d.len = sz - cp;
                d.flags = PHOS_COPY_LIVE_TO_IMAGE;
                c->cow_log.insert(c->cow_log.end(), {S.round, i, 2ull, cp, sz - cp});
                c->direct_bytes += sz - cp;
                S.copied[i] = sz;
                S.state[i] = kDone;
            }
            v.push_back(d);
        }
        for (uint32_t i = 0; i < n; ++i) c->safe[i] = S.state[i] == kDone || c->shadow[i] >= 0;
        r = S.submit(v, c->staging, c->staging_bytes, c->image, c->image_bytes, nullptr);
        if (r) return r;
        if (S.nosync && (r = S.upload_slot(c->safe))) return r;
    } else {
        for (uint32_t i = 0; i < n; ++i) {
            c->touched[i] = S.state[i] != kPending;
            if ((perm[i] & PHOS_PERM_W) && c->touched[i]) c->dirty[i] = 1;
        }
        if (S.nosync && (r = S.upload_slot(c->touched))) return r;
    }
    c->in_kernel = true;
    return PHOS_OK;
}

extern "C" phos_status phos_ckpt_before_kernel_dev(phos_ckpt_t *c, const uint8_t *d_perm) {
    if (!c) return fail(PHOS_EINVAL, "ckpt_before_kernel_dev: NULL session");
    if (!c->dr) return fail(PHOS_EINVAL, "ckpt_before_kernel_dev: not a PHOS_CKPT_DEVICE session");
    if (c->in_kernel) return fail(PHOS_EINVAL, "ckpt_before_kernel_dev: after_kernel missing");
    if (c->complete) return fail(PHOS_EINVAL, "ckpt_before_kernel_dev: checkpoint already complete");
    if (!d_perm && c->ss.n) return fail(PHOS_EINVAL, "ckpt_before_kernel_dev: d_perm is NULL");
    Session &S = c->ss;
    phos_status r = c->dr->action(d_perm, S.round, c->staging, c->staging_bytes, c->image,
                                  c->image_bytes, nullptr, S.d_status, S.s);
    if (r) return r;
    S.perm_dev = d_perm;
    S.flags_dev = c->dr->flags();
    c->in_kernel = true;
    return PHOS_OK;
}

static phos_status stw_checkpoint(phos_ckpt *c) {
    Session &S = c->ss;
    std::vector<phos_copy_t> v;
    for (uint32_t i = 0; i < S.n; ++i) {
        phos_copy_t d;
        d.src_off = 0;
        d.dst_off = S.t->img_off[i];
        d.len = S.t->size[i];
        d.buf = i;
        d.flags = PHOS_COPY_LIVE_TO_IMAGE;
        v.push_back(d);
        S.state[i] = kDone;
        S.copied[i] = S.t->size[i];
    }
    phos_status r = S.submit(v, nullptr, 0, c->image, c->image_bytes, nullptr);
    if (r) return r;
    return S.sync();
}

extern "C" phos_status phos_ckpt_after_kernel(phos_ckpt_t *c, const uint64_t *d_trace,
                                              uint64_t n_rec, int *misspec) {
    if (!c) return fail(PHOS_EINVAL, "ckpt_after_kernel: NULL session");
    if (!c->in_kernel) return fail(PHOS_EINVAL, "ckpt_after_kernel: before_kernel missing");
    Session &S = c->ss;
    c->in_kernel = false;
    const uint64_t k = S.round++;
    if (misspec) *misspec = 0;
    if (S.nosync) {
        phos_status r = S.validate_nosync(d_trace, n_rec, c->mode == PHOS_CKPT_COW ? 1 : 0);
        if (r) return r;
        if (c->mode == PHOS_CKPT_COW && S.flag() >= 0) {
            c->misspec = S.flag();
            c->complete = true;
            if (misspec) *misspec = 1;
        }
        return PHOS_OK;
    }
    phos_status r = S.validate_sync(d_trace, n_rec);
    if (r) return r;
    if (S.h_count[1] == 0) return PHOS_OK;  // no store violated the speculation
    if (c->mode == PHOS_CKPT_COW) {
        for (uint32_t i = 0; i < S.n; ++i) {
            if (S.victim_bit(true, i) && !c->safe[i]) {
                c->misspec = (int64_t)k;
                r = stw_checkpoint(c);
                if (r) return r;
                c->complete = true;
                for (uint32_t j = 0; j < S.n; ++j)
                    if (c->shadow[j] >= 0) c->shadow[j] = -1;
                if (misspec) *misspec = 1;
                return PHOS_OK;
            }
        }
    } else {
        for (uint32_t i = 0; i < S.n; ++i)
            if (S.victim_bit(true, i) && c->touched[i]) c->dirty[i] = 1;
    }
    return PHOS_OK;
}

extern "C" phos_status phos_ckpt_finish(phos_ckpt_t *c) {
    if (!c) return fail(PHOS_EINVAL, "ckpt_finish: NULL session");
    if (c->in_kernel) return fail(PHOS_EINVAL, "ckpt_finish: inside a kernel round");
    Session &S = c->ss;
    phos_status r;
    if (c->dr && !c->finished) {
        if ((r = S.collect(nullptr))) return r;
        if (S.flag() >= 0) {
            c->misspec = S.flag();
            if ((r = stw_checkpoint(c))) return r;
        } else {
            // drain what the copier has not moved yet
            r = c->dr->copier(~0ull >> 2, S.round, c->staging, c->staging_bytes, c->image,
                              c->image_bytes, nullptr, S.d_status, S.s);
            if (r) return r;
        }
        if ((r = S.sync())) return r;
        uint64_t ctr[6];
        std::vector<uint8_t> st;
        if ((r = c->dr->collect(S.copier_log, c->cow_log, ctr, &st))) return r;
        c->copier_bytes = ctr[2];
        c->cow_bytes = ctr[3];
        c->direct_bytes = ctr[4];
        c->complete = true;
        c->finished = true;
        return PHOS_OK;
    }
    if (S.nosync && !c->finished) {
        // everything enqueued has run: the rule's outcome is final
        r = S.collect(c->mode == PHOS_CKPT_RECOPY ? &c->dirty : nullptr);
        if (r) return r;
        if (c->mode == PHOS_CKPT_COW && S.flag() >= 0) {
            // mis-speculation: discard, copy everything stop-the-world now
            c->misspec = S.flag();
            r = stw_checkpoint(c);
            if (r) return r;
            c->complete = true;
            std::fill(c->shadow.begin(), c->shadow.end(), -1);
        }
    }
    if (!c->complete && c->misspec < 0) {
        r = ckpt_advance(c, ~0ull >> 2);
        if (r) return r;
        c->complete = S.done();
    }
    // concurrent: the recopy below lands after every copier piece
    if (S.cs && (r = S.app_wait(S.batch))) return r;
    if (c->mode == PHOS_CKPT_RECOPY && !c->finished) {
        // t2: quiesce (the caller has stopped issuing kernels), recopy the
        // dirty buffers whole from live memory
        std::vector<phos_copy_t> v;
        for (uint32_t i = 0; i < S.n; ++i) {
            if (!c->dirty[i]) continue;
            phos_copy_t d;
            d.src_off = 0;
            d.dst_off = S.t->img_off[i];
            d.len = S.t->size[i];
            d.buf = i;
            d.flags = PHOS_COPY_LIVE_TO_IMAGE;
            v.push_back(d);
            c->recopy_bytes += S.t->size[i];
        }
        r = S.submit(v, nullptr, 0, c->image, c->image_bytes, nullptr);
        if (r) return r;
    }
    c->finished = true;
    return S.sync();
}

extern "C" phos_status phos_ckpt_begin_pass(phos_ckpt_t *c, uint64_t *pass_bytes) {
    if (!c) return fail(PHOS_EINVAL, "ckpt_begin_pass: NULL session");
    if (c->mode != PHOS_CKPT_RECOPY) return fail(PHOS_EINVAL, "ckpt_begin_pass: recopy only");
    if (c->in_kernel || c->finished)
        return fail(PHOS_EINVAL, "ckpt_begin_pass: inside a kernel round or finished");
    Session &S = c->ss;
    if (!S.done()) return fail(PHOS_EINVAL, "ckpt_begin_pass: the current pass is not done");
    if (S.nosync) {
        phos_status r = S.collect(&c->dirty);
        if (r) return r;
    }
    uint64_t bytes = 0, nb = 0;
    for (uint32_t i = 0; i < S.n; ++i) {
        if (!c->dirty[i]) continue;
        S.state[i] = kPending;
        S.copied[i] = 0;
        c->dirty[i] = 0;
        bytes += S.t->size[i];
        ++nb;
    }
    S.cursor = 0;
    c->complete = S.done();
    c->pass_log.insert(c->pass_log.end(), {S.round, nb, bytes, 0, 0});
    if (pass_bytes) *pass_bytes = bytes;
    return PHOS_OK;
}

// No-sync sessions: bring the device-side dirty marks and violation total
// into the host state before reporting them.
static phos_status ckpt_collect(const phos_ckpt_t *cc) {
    phos_ckpt *c = const_cast<phos_ckpt *>(cc);
    if (!c->ss.nosync || c->finished) return PHOS_OK;
    return c->ss.collect(c->mode == PHOS_CKPT_RECOPY ? &c->dirty : nullptr);
}

extern "C" phos_status phos_ckpt_stats(const phos_ckpt_t *c, phos_ckpt_stats_t *o) {
    if (!c || !o) return fail(PHOS_EINVAL, "ckpt_stats: NULL argument");
    if (c->in_kernel) return fail(PHOS_EINVAL, "ckpt_stats: inside a kernel round");
    phos_status r = ckpt_collect(c);
    if (r) return r;
    memset(o, 0, sizeof *o);
    o->kernels = c->ss.round;
    o->copier_bytes = c->copier_bytes;
    o->cow_bytes = c->cow_bytes;
    o->direct_bytes = c->direct_bytes;
    o->recopy_bytes = c->recopy_bytes;
    o->validated = c->ss.validated;
    o->violations = c->ss.violations;
    o->misspec_round = c->misspec;
    o->done = c->complete ? 1 : 0;
    uint32_t nd = 0;
    for (uint8_t x : c->dirty) nd += x;
    o->dirty = nd;
    o->passes = c->pass_log.size() / 5;
    return PHOS_OK;
}

extern "C" phos_status phos_ckpt_log(const phos_ckpt_t *c, uint32_t kind, uint64_t *out,
                                     uint64_t cap, uint64_t *n_out) {
    if (!c) return fail(PHOS_EINVAL, "ckpt_log: NULL session");
    if (kind == 0) return copy_log(c->cow_log, out, cap, n_out);
    if (kind == 1) return copy_log(c->ss.copier_log, out, cap, n_out);
    if (kind == 2) {
        if (c->in_kernel) return fail(PHOS_EINVAL, "ckpt_log: inside a kernel round");
        phos_status r = ckpt_collect(c);
        if (r) return r;
        std::vector<uint64_t> v;
        for (uint32_t i = 0; i < c->ss.n; ++i)
            if (c->dirty[i]) v.insert(v.end(), {i, 0, 0, 0, 0});
        return copy_log(v, out, cap, n_out);
    }
    if (kind == 3) return copy_log(c->pass_log, out, cap, n_out);
    return fail(PHOS_EINVAL, "ckpt_log: kind %u", kind);
}

extern "C" phos_status phos_ckpt_end(phos_ckpt_t *c) {
    delete c;
    return PHOS_OK;
}

// ------------------------------------------------------------- restore

struct phos_restore {
    Session ss;
    const void *image = nullptr;
    uint64_t image_bytes = 0;
    uint32_t *d_present = nullptr;
    std::vector<uint8_t> present, before;
    std::vector<uint64_t> od_log;
    uint64_t copier_bytes = 0, ondemand_bytes = 0;
    int64_t misspec = -1;
    bool in_kernel = false;
    // PHOS_RESTORE_ONDEMAND_FIRST: a round's copier move comes after its
    // on-demand copies (advance inside the round, once)
    bool odf = false, advanced = false;
    uint64_t waited = 0;     // concurrent: latest copier batch the caller's stream waited for
    // integrity check: manifest digests, per-buffer accumulators and tile
    // counters, the lowest corrupt buffer (mapped host word)
    const uint64_t *d_manifest = nullptr;
    unsigned long long *d_vacc = nullptr;
    uint32_t *d_vcnt = nullptr;
    int *h_bad = nullptr, *d_bad = nullptr;

    // Verify the buffers whose last byte was just copied, on the stream of
    // that copy (before any kernel can use them).
    phos_status verify(const std::vector<uint32_t> &bufs, cudaStream_t st) {
        if (!d_manifest || bufs.empty()) return PHOS_OK;
        return verify_buffers(ss.t, bufs, d_manifest, d_vacc, d_vcnt, ss.d_status, d_bad, st);
    }

    DevRounds *dr = nullptr;      // PHOS_CKPT_DEVICE: decisions on the device

    ~phos_restore() {
        ss.pend.clear();      // an ended session validates nothing more
        ss.sync_streams();
        delete dr;
        if (d_vacc) cudaFree(d_vacc);
        if (d_vcnt) cudaFree(d_vcnt);
        if (h_bad) cudaFreeHost(h_bad);
    }

    bool all_present() const {
        for (uint8_t p : present)
            if (!p) return false;
        return true;
    }
};

extern "C" phos_status phos_restore_begin(const phos_table_t *t, const phos_restore_desc_t *d,
                                          phos_stream_t stream, phos_restore_t **out) {
    if (!t || !d || !out) return fail(PHOS_EINVAL, "restore_begin: NULL argument");
    *out = nullptr;
    if (d->access_bytes == 0 || d->chunk == 0 || d->chunk % 256)
        return fail(PHOS_EINVAL, "restore_begin: access_bytes >= 1, chunk a multiple of 256");
    if (d->d_manifest && d->image && d->image_bytes < t->image_bytes)
        return fail(PHOS_ECORRUPT, "restore_begin: image truncated (%llu of %llu bytes)",
                    (unsigned long long)d->image_bytes, (unsigned long long)t->image_bytes);
    if (!d->image || d->image_bytes < t->image_bytes)
        return fail(PHOS_EINVAL, "restore_begin: image smaller than %llu bytes",
                    (unsigned long long)t->image_bytes);
    if (d->flags & ~(uint32_t)(PHOS_CKPT_NO_SYNC | PHOS_CKPT_CONCURRENT | PHOS_CKPT_DEVICE |
                               PHOS_CKPT_DEFER | PHOS_RESTORE_ONDEMAND_FIRST))
        return fail(PHOS_EINVAL, "restore_begin: flags %#x", d->flags);
    if ((d->flags & PHOS_RESTORE_ONDEMAND_FIRST) && !(d->flags & PHOS_CKPT_CONCURRENT))
        return fail(PHOS_EINVAL, "restore_begin: PHOS_RESTORE_ONDEMAND_FIRST needs "
                                 "PHOS_CKPT_CONCURRENT");
    if ((d->flags & PHOS_CKPT_DEFER) && (d->flags & PHOS_CKPT_DEVICE))
        return fail(PHOS_EINVAL, "restore_begin: PHOS_CKPT_DEFER goes without PHOS_CKPT_DEVICE");
    if ((d->flags & PHOS_CKPT_DEVICE) && ((d->flags & PHOS_CKPT_CONCURRENT) || d->d_manifest))
        return fail(PHOS_EINVAL, "restore_begin: PHOS_CKPT_DEVICE goes without "
                                 "PHOS_CKPT_CONCURRENT and without a manifest");
    phos_restore *r = new phos_restore();
    phos_status e = r->ss.init(t, static_cast<cudaStream_t>(stream), d->access_bytes, d->chunk);
    if (!e && (d->flags & PHOS_CKPT_CONCURRENT)) e = r->ss.init_concurrent();
    if (!e && (d->flags & (PHOS_CKPT_NO_SYNC | PHOS_CKPT_DEVICE | PHOS_CKPT_DEFER)) &&
        !r->ss.nosync)
        e = r->ss.init_nosync();
    if (!e && (d->flags & PHOS_CKPT_DEFER)) e = r->ss.init_defer();
    if (!e && (d->flags & PHOS_CKPT_DEVICE)) {
        r->dr = new DevRounds();
        e = r->dr->init(t, 1, d->chunk, 0, d->d_present != nullptr, r->ss.s);
    }
    if (e) {
        delete r;
        return e;
    }
    r->image = d->image;
    r->image_bytes = d->image_bytes;
    r->d_present = d->d_present;
    r->odf = (d->flags & PHOS_RESTORE_ONDEMAND_FIRST) != 0;
    if (d->d_manifest) {
        cudaError_t ce;
        const size_t nn = std::max(t->n, 1u);
        if ((ce = cudaMalloc(&r->d_vacc, 8 * nn)) != cudaSuccess ||
            (ce = cudaMalloc(&r->d_vcnt, 4 * nn)) != cudaSuccess ||
            (ce = cudaMemset(r->d_vacc, 0, 8 * nn)) != cudaSuccess ||
            (ce = cudaMemset(r->d_vcnt, 0, 4 * nn)) != cudaSuccess ||
            (ce = cudaHostAlloc(&r->h_bad, 64, cudaHostAllocMapped)) != cudaSuccess ||
            (ce = cudaHostGetDevicePointer((void **)&r->d_bad, r->h_bad, 0)) != cudaSuccess) {
            delete r;
            return cuda_fail(ce, "restore_begin: integrity scratch");
        }
        *(volatile int *)r->h_bad = INT_MAX;
        r->d_manifest = d->d_manifest;
    }
    r->present.assign(t->n, 0);
    r->before.assign(t->n, 0);
    if (r->d_present && t->n) {
        cudaError_t ce = cudaMemsetAsync(r->d_present, 0, 4ull * ((t->n + 31) / 32),
                                         r->ss.s);
        if (ce != cudaSuccess) {
            delete r;
            return cuda_fail(ce, "restore_begin: cudaMemsetAsync(present)");
        }
    }
    *out = r;
    return PHOS_OK;
}

// With the copier on its own stream a round's pieces go out in sub-batches
// of about this many bytes, each closed at a buffer's last piece and
// followed by its own event, so a kernel waits only for the sub-batch that
// lands its buffers, not for the whole round's quota.
constexpr uint64_t kSubBatch = 16ull << 20;

static phos_status restore_advance(phos_restore *R, uint64_t quota) {
    Session &S = R->ss;
    const phos_table *t = S.t;
    std::vector<phos_copy_t> v;
    std::vector<uint32_t> landed, touched;
    uint64_t b = S.batch + 1, sub_bytes = 0;
    if (S.cs) {
        phos_status r0 = S.retire_batches();
        if (r0) return r0;
        PHOS_CUDA(cudaEventRecord(S.app_ev, S.s));
        PHOS_CUDA(cudaStreamWaitEvent(S.cs, S.app_ev, 0));
    }
    phos_status err = PHOS_OK;
    // issue the pieces gathered so far; with the copier stream, as
    // sub-batch b with its own event
    auto flush = [&]() -> phos_status {
        if (v.empty()) return PHOS_OK;
        phos_status r = S.submit(v, nullptr, 0, R->image, R->image_bytes, R->d_present, true);
        if (r) return r;
        if ((r = R->verify(landed, S.cs ? S.cs : S.s))) return r;
        if (S.cs) {
            for (uint32_t i : touched) S.last_batch[i] = b;
            if ((r = S.record_batch(b, sub_bytes))) return r;
            ++b;
        }
        v.clear();
        landed.clear();
        touched.clear();
        sub_bytes = 0;
        return PHOS_OK;
    };
    uint64_t moved = S.advance(
        quota,
        [&](uint32_t i, uint64_t off, uint64_t len) {
            phos_copy_t d;
            d.src_off = t->img_off[i] + off;
            d.dst_off = off;
            d.len = len;
            d.buf = i;
            d.flags = PHOS_COPY_IMAGE_TO_LIVE;
            const bool last = off + len == t->size[i];
            if (last) {
                R->present[i] = 1;
                landed.push_back(i);
                if (R->d_present) d.flags |= PHOS_COPY_MARK_PRESENT;
            }
            v.push_back(d);
            touched.push_back(i);
            sub_bytes += len;
            if (S.cs && last && sub_bytes >= kSubBatch && !err) err = flush();
            return false;
        },
        [&](uint32_t i) { return R->present[i] != 0; });
    R->copier_bytes += moved;
    if (err) return err;
    return flush();
}

// Mis-speculation (Sec. 6): roll back to the checkpoint's state, every
// buffer from the image, stop-the-world.  The caller replays the kernels.
static phos_status restore_rollback(phos_restore *R, int64_t k) {
    Session &S = R->ss;
    R->misspec = k;
    // concurrent: no copier piece may land after the rollback's bytes
    phos_status r = S.cs ? S.app_wait(S.batch) : PHOS_OK;
    if (r) return r;
    std::vector<phos_copy_t> v;
    std::vector<uint32_t> all(S.n);
    for (uint32_t j = 0; j < S.n; ++j) {
        all[j] = j;
        phos_copy_t d;
        d.src_off = S.t->img_off[j];
        d.dst_off = 0;
        d.len = S.t->size[j];
        d.buf = j;
        d.flags = PHOS_COPY_IMAGE_TO_LIVE | (R->d_present ? PHOS_COPY_MARK_PRESENT : 0);
        v.push_back(d);
        R->present[j] = 1;
        S.state[j] = kDone;
        S.copied[j] = S.t->size[j];
    }
    phos_status r2 = S.submit(v, nullptr, 0, R->image, R->image_bytes, R->d_present);
    if (r2) return r2;
    if (R->dr && (r2 = R->dr->mark_all(S.s))) return r2;
    return R->verify(all, S.s);
}

extern "C" phos_status phos_restore_advance(phos_restore_t *R, uint64_t quota, int *done) {
    if (!R) return fail(PHOS_EINVAL, "restore_advance: NULL session");
    if (R->odf) {
        // inside the round, after its on-demand copies, once
        if (!R->in_kernel || R->advanced)
            return fail(PHOS_EINVAL, "restore_advance: with PHOS_RESTORE_ONDEMAND_FIRST, once "
                                     "per round, after before_kernel");
        R->advanced = true;
        // a mis-speculation the device has seen: the round's kernel and
        // after_kernel still follow (they roll back); no more copier moves
        const bool seen = R->ss.nosync && R->misspec < 0 && R->ss.flag() >= 0;
        phos_status r = (seen || R->all_present()) ? PHOS_OK : restore_advance(R, quota);
        if (done) *done = (seen || R->all_present()) ? 1 : 0;
        return r;
    }
    if (R->in_kernel) return fail(PHOS_EINVAL, "restore_advance: inside a kernel round");
    phos_status r = PHOS_OK;
    if (R->ss.nosync && R->misspec < 0 && R->ss.flag() >= 0) {
        r = restore_rollback(R, R->ss.flag());  // the device saw it
        if (r) return r;
    }
    if (R->dr) {
        Session &S = R->ss;
        if (R->misspec < 0)
            r = R->dr->copier(quota, S.round, nullptr, 0, R->image, R->image_bytes, R->d_present,
                              S.d_status, S.s);
        if (done) *done = R->misspec >= 0 ? 1 : 0;
        return r;
    }
    if (!R->all_present()) r = restore_advance(R, quota);
    if (done) *done = R->all_present() ? 1 : 0;
    return r;
}

extern "C" phos_status phos_restore_before_kernel(phos_restore_t *R, const uint8_t *perm) {
    if (!R) return fail(PHOS_EINVAL, "restore_before_kernel: NULL session");
    if (R->in_kernel) return fail(PHOS_EINVAL, "restore_before_kernel: after_kernel missing");
    R->advanced = false;
    Session &S = R->ss;
    const phos_table *t = S.t;
    phos_status r = S.stage_perm(perm);
    if (r) return r;
    if (S.cs) {
        // the kernel starts after the copier's pieces of every buffer it is
        // speculated to access (and so after all earlier pieces)
        uint64_t need = 0;
        for (uint32_t i = 0; i < S.n; ++i)
            if (perm[i]) need = std::max(need, S.last_batch[i]);
        if (need > R->waited) {
            r = S.app_wait(need);
            if (r) return r;
            R->waited = need;
        }
    }
    std::vector<phos_copy_t> v;
    std::vector<uint32_t> landed;
    for (uint32_t i = 0; i < S.n; ++i) {
        if (!perm[i] || R->present[i]) continue;
        landed.push_back(i);
        const uint64_t cp = S.copied[i], sz = t->size[i];
        phos_copy_t d;
        d.src_off = t->img_off[i] + cp;
        d.dst_off = cp;
        d.len = sz - cp;
        d.buf = i;
        d.flags = PHOS_COPY_IMAGE_TO_LIVE | (R->d_present ? PHOS_COPY_MARK_PRESENT : 0);
        v.push_back(d);
        R->od_log.insert(R->od_log.end(), {S.round, i, cp, sz - cp, 0});
        R->ondemand_bytes += sz - cp;
        S.copied[i] = sz;
        S.state[i] = kDone;
        R->present[i] = 1;
    }
    // restored before the kernel: present, and (concurrent) landed
    for (uint32_t i = 0; i < S.n; ++i)
        R->before[i] = R->present[i] && (!S.cs || S.last_batch[i] <= R->waited);
    r = S.submit(v, nullptr, 0, R->image, R->image_bytes, R->d_present);
    if (r) return r;
    if ((r = R->verify(landed, S.s))) return r;
    if (S.nosync && (r = S.upload_slot(R->before))) return r;
    R->in_kernel = true;
    return PHOS_OK;
}

extern "C" phos_status phos_restore_before_kernel_dev(phos_restore_t *R, const uint8_t *d_perm) {
    if (!R) return fail(PHOS_EINVAL, "restore_before_kernel_dev: NULL session");
    if (!R->dr) return fail(PHOS_EINVAL, "restore_before_kernel_dev: not a PHOS_CKPT_DEVICE session");
    if (R->in_kernel) return fail(PHOS_EINVAL, "restore_before_kernel_dev: after_kernel missing");
    if (!d_perm && R->ss.n) return fail(PHOS_EINVAL, "restore_before_kernel_dev: d_perm is NULL");
    Session &S = R->ss;
    if (R->misspec < 0) {
        phos_status r = R->dr->action(d_perm, S.round, nullptr, 0, R->image, R->image_bytes,
                                      R->d_present, S.d_status, S.s);
        if (r) return r;
    }
    S.perm_dev = d_perm;
    S.flags_dev = R->dr->flags();
    R->in_kernel = true;
    return PHOS_OK;
}

extern "C" phos_status phos_restore_after_kernel(phos_restore_t *R, const uint64_t *d_trace,
                                                 uint64_t n_rec, int *misspec) {
    if (!R) return fail(PHOS_EINVAL, "restore_after_kernel: NULL session");
    if (!R->in_kernel) return fail(PHOS_EINVAL, "restore_after_kernel: before_kernel missing");
    Session &S = R->ss;
    R->in_kernel = false;
    const uint64_t k = S.round++;
    if (misspec) *misspec = 0;
    if (S.nosync) {
        phos_status r = S.validate_nosync(d_trace, n_rec, 2);
        if (r) return r;
        if (R->misspec < 0 && S.flag() >= 0) {
            r = restore_rollback(R, S.flag());
            if (r) return r;
            if (misspec) *misspec = 1;
        }
        return PHOS_OK;
    }
    phos_status r = S.validate_sync(d_trace, n_rec);
    if (r) return r;
    if (S.h_count[0] == S.h_count[2]) return PHOS_OK;  // only unmapped accesses
    for (uint32_t i = 0; i < S.n; ++i) {
        if (S.victim_bit(false, i) && !R->before[i]) {
            r = restore_rollback(R, (int64_t)k);
            if (r) return r;
            r = S.sync();
            if (r) return r;
            if (misspec) *misspec = 1;
            return PHOS_OK;
        }
    }
    return PHOS_OK;
}

extern "C" phos_status phos_restore_finish(phos_restore_t *R) {
    if (!R) return fail(PHOS_EINVAL, "restore_finish: NULL session");
    if (R->in_kernel) return fail(PHOS_EINVAL, "restore_finish: inside a kernel round");
    if (R->dr) {
        Session &S = R->ss;
        phos_status r = S.collect(nullptr);
        if (r) return r;
        if (R->misspec < 0 && S.flag() >= 0 && (r = restore_rollback(R, S.flag()))) return r;
        if (R->misspec < 0 &&
            (r = R->dr->copier(~0ull >> 2, S.round, nullptr, 0, R->image, R->image_bytes,
                               R->d_present, S.d_status, S.s)))
            return r;
        if ((r = S.sync())) return r;
        uint64_t ctr[6];
        if ((r = R->dr->collect(S.copier_log, R->od_log, ctr, nullptr))) return r;
        R->copier_bytes = ctr[2];
        R->ondemand_bytes = ctr[5];
        std::fill(R->present.begin(), R->present.end(), 1);
        return PHOS_OK;
    }
    if (R->ss.nosync) {
        phos_status r = R->ss.collect(nullptr);
        if (r) return r;
        if (R->misspec < 0 && R->ss.flag() >= 0 && (r = restore_rollback(R, R->ss.flag())))
            return r;
    }
    if (!R->all_present()) {
        phos_status r = restore_advance(R, ~0ull >> 2);
        if (r) return r;
    }
    return R->ss.sync();
}

extern "C" phos_status phos_restore_stats(const phos_restore_t *R, phos_restore_stats_t *o) {
    if (!R || !o) return fail(PHOS_EINVAL, "restore_stats: NULL argument");
    memset(o, 0, sizeof *o);
    o->kernels = R->ss.round;
    o->copier_bytes = R->copier_bytes;
    o->ondemand_bytes = R->ondemand_bytes;
    o->validated = R->ss.validated;
    o->violations = R->ss.violations;
    o->misspec_round = R->misspec;
    o->done = R->all_present() ? 1 : 0;
    o->corrupt_buf = -1;
    if (R->h_bad) {
        const int b = *(volatile int *)R->h_bad;
        if (b != INT_MAX) o->corrupt_buf = b;
    }
    return PHOS_OK;
}

extern "C" phos_status phos_restore_log(const phos_restore_t *R, uint32_t kind, uint64_t *out,
                                        uint64_t cap, uint64_t *n_out) {
    if (!R) return fail(PHOS_EINVAL, "restore_log: NULL session");
    if (kind == 0) return copy_log(R->od_log, out, cap, n_out);
    if (kind == 1) return copy_log(R->ss.copier_log, out, cap, n_out);
    return fail(PHOS_EINVAL, "restore_log: kind %u", kind);
}

extern "C" phos_status phos_restore_end(phos_restore_t *R) {
    delete R;
    return PHOS_OK;
}
