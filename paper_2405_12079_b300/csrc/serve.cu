// Serving loop: continuous batching of checkpoint and restore requests
// (the restore-mostly serverless case of PhoenixOS Sec. 7 "Fast GPU
// serverless function startups", and periodic checkpoints of Sec. 7
// "Fault tolerance", served as a stream of requests).
//
// A scheduler thread owns three streams: device->device snapshots,
// device->host drains and host->device loads.  Requests are admitted, in
// arrival order where possible, as slots and staging budget free up (a
// checkpoint needs staging for its whole image; a restore needs none, so
// it may pass a checkpoint that waits for staging).  A checkpoint is
// snapshotted into staging with one copy-engine launch (HBM speed), then
// drained to its pinned host image in pieces; a restore is loaded piece by
// piece.  Each scheduling turn fills one batch per direction (up to 64 MB,
// at most two batches queued per direction) with pieces of the admitted
// requests, oldest first, so a request that arrives while others are on the
// GPU joins the next batch that has room, and the two directions run
// concurrently.  Completion is tracked with events; no turn blocks on the
// device.
//
// Application transfers (phos_server_app_copy) run on the application's
// own stream.  With APP_PRIORITY the scheduler issues no new C/R batch, in
// either direction, while an application transfer is pending or running:
// a copy engine may serve streams of both directions, so holding back only
// the transfer's own direction left it queued behind the other one's DMA
// copies (hundreds of ms under load on B300).  At most `window` C/R bytes
// per direction are then ahead of it.  The pause is a host decision per
// turn and never waits on the device.
#include <string.h>
#include <time.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>
#include <vector>

#include "internal.h"

namespace phos {

static uint64_t now_ns() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}

struct Req {
    uint64_t ticket;
    phos_request_t r;
    phos_result_t res;
    // progress
    uint64_t stg_off = 0;          // checkpoint: staging extent
    uint64_t img_bytes = 0;
    uint64_t issued = 0;           // host-leg bytes issued
    uint32_t buf = 0;              // restore: next buffer / offset
    uint64_t buf_off = 0;
    bool snap_done = false;
    cudaEvent_t snap_ev = nullptr;
    bool cancel = false;           // phos_server_cancel on an admitted request
    uint32_t inflight = 0;         // issued batches holding its pieces, not retired
};

// One batch issued on a host-leg stream.
struct Issue {
    cudaEvent_t ev;
    std::vector<uint64_t> finishing;  // tickets whose last piece is in this batch
    std::vector<uint64_t> members;    // tickets with pieces in this batch
};

// An application transfer the scheduler yields to.
struct AppCopy {
    cudaEvent_t ev;
    bool d2h;
};

}  // namespace phos

using namespace phos;

struct phos_server {
    static constexpr uint64_t kMaxRun = 64ull << 20;   // largest merged DMA copy
    phos_server_desc_t d{};
    int device = 0;
    cudaStream_t s_snap = nullptr, s_d2h = nullptr, s_h2d = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::deque<uint64_t> queue;                 // submitted, not admitted
    std::map<uint64_t, Req> reqs;               // all requests by ticket
    std::vector<uint64_t> active;               // admitted, not done
    std::vector<std::pair<uint64_t, uint64_t>> free_stg;  // staging extents
    std::deque<Issue> inflight_d2h, inflight_h2d;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<AppCopy> app_inflight;          // recorded, maybe not complete
    uint32_t app_pending[2] = {0, 0};           // being issued (h2d, d2h)
    phos_server_stats_t st{};
    // device descriptor rings per direction (pinned staging of lists)
    phos_copy_t *h_ring[3] = {nullptr, nullptr, nullptr};         // pinned, mapped
    const phos_copy_t *h_ring_dev[3] = {nullptr, nullptr, nullptr}; // their device addresses
    phos_copy_t *d_ring[3] = {nullptr, nullptr, nullptr};
    uint32_t *d_status = nullptr;
    size_t ring_cap = 65536;
    size_t ring_pos[3] = {0, 0, 0};

    cudaEvent_t get_ev() {
        if (!ev_pool.empty()) {
            cudaEvent_t e = ev_pool.back();
            ev_pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        return e;
    }

    bool stg_alloc(uint64_t need, uint64_t *off) {
        for (size_t j = 0; j < free_stg.size(); ++j)
            if (free_stg[j].second >= need) {
                *off = free_stg[j].first;
                if (free_stg[j].second == need)
                    free_stg.erase(free_stg.begin() + j);
                else
                    free_stg[j] = {free_stg[j].first + need, free_stg[j].second - need};
                return true;
            }
        return false;
    }
    void stg_release(uint64_t off, uint64_t len) {
        auto it = std::lower_bound(free_stg.begin(), free_stg.end(),
                                   std::make_pair(off, (uint64_t)0));
        it = free_stg.insert(it, {off, len});
        size_t j = it - free_stg.begin();
        if (j + 1 < free_stg.size() && free_stg[j].first + free_stg[j].second == free_stg[j + 1].first) {
            free_stg[j].second += free_stg[j + 1].second;
            free_stg.erase(free_stg.begin() + j + 1);
        }
        if (j > 0 && free_stg[j - 1].first + free_stg[j - 1].second == free_stg[j].first) {
            free_stg[j - 1].second += free_stg[j].second;
            free_stg.erase(free_stg.begin() + j);
        }
    }

    // Copy descriptors through the copy engine on stream s.  Lists go
    // through ring r of pinned + device memory; before the ring wraps, the
    // stream is synchronised so no list is overwritten before its upload.
    phos_status launch(int r, cudaStream_t s, const phos_table_t *t,
                       const std::vector<phos_copy_t> &v, void *img, uint64_t img_bytes) {
        if (v.empty()) return PHOS_OK;
        if (v.size() > ring_cap) return fail(PHOS_EINVAL, "server: batch of %zu pieces", v.size());
        if (ring_pos[r] + v.size() > ring_cap) {
            PHOS_CUDA(cudaStreamSynchronize(s));
            ring_pos[r] = 0;
        }
        phos_copy_t *hp = h_ring[r] + ring_pos[r];
        phos_copy_t *dp = d_ring[r] + ring_pos[r];
        memcpy(hp, v.data(), v.size() * sizeof(phos_copy_t));
        // not by the copy engines: an upload would queue behind the DMA legs
        phos_status rp = push_small(dp, hp, h_ring_dev[r] + ring_pos[r],
                                    v.size() * sizeof(phos_copy_t), s);
        if (rp) return rp;
        ring_pos[r] += v.size();
        return phos_copy(t, dp, (uint32_t)v.size(), d.d_staging, d.staging_bytes, img, img_bytes,
                         nullptr, d_status, s);
    }

    void admit() {
        for (auto it = queue.begin(); it != queue.end() && active.size() < d.max_slots;) {
            Req &q = reqs[*it];
            const phos_table *t = q.r.table;
            q.img_bytes = t->image_bytes;
            if (q.r.kind == PHOS_REQ_CHECKPOINT && q.img_bytes) {
                uint64_t off;
                if (!stg_alloc(align_up(q.img_bytes, 256), &off)) {
                    ++it;                      // waits for staging; restores may pass
                    if (d.max_slots == 1) break;
                    continue;
                }
                q.stg_off = off;
                // snapshot: every buffer live -> staging at its image offset
                std::vector<phos_copy_t> v(t->n);
                for (uint32_t i = 0; i < t->n; ++i)
                    v[i] = phos_copy_t{0, off + t->img_off[i], t->size[i], i,
                                       PHOS_COPY_LIVE_TO_STAGING};
                phos_status e = launch(0, s_snap, t, v, nullptr, 0);
                q.snap_ev = get_ev();
                cudaEventRecord(q.snap_ev, s_snap);
                if (e) q.res.status = e;
            }
            q.res.state = 1;
            q.res.t_admit_ns = now_ns();
            active.push_back(q.ticket);
            it = queue.erase(it);
        }
    }

    // One host-leg batch for a direction: pieces of the admitted requests of
    // that direction, oldest first, up to `batch` bytes.
    void issue(bool d2h) {
        std::deque<Issue> &inf = d2h ? inflight_d2h : inflight_h2d;
        if (inf.size() >= 2) return;           // keep at most two batches queued
        if ((d.flags & PHOS_SERVER_APP_PRIORITY) && app_busy()) {
            ++st.paused_turns;                 // an application transfer goes first
            return;
        }
        const uint64_t batch = d.window ? std::max(d.chunk, d.window / 2)
                                        : std::max<uint64_t>(d.chunk * 8, 64ull << 20);
        std::vector<Req *> cand;
        for (uint64_t tk : active) {
            Req &q = reqs[tk];
            if (q.res.state != 1 || q.res.status || q.cancel) continue;
            if (d2h && q.r.kind == PHOS_REQ_CHECKPOINT && q.issued < q.img_bytes) {
                if (!q.snap_done) {
                    if (cudaEventQuery(q.snap_ev) != cudaSuccess) continue;
                    q.snap_done = true;
                }
                cand.push_back(&q);
            } else if (!d2h && q.r.kind == PHOS_REQ_RESTORE && q.issued < q.img_bytes) {
                cand.push_back(&q);
            }
        }
        if (cand.empty()) return;
        Issue is;
        uint64_t used = 0, pieces = 0;
        std::vector<std::vector<phos_copy_t>> lists(cand.size());
        // oldest admitted request first: a batch takes its pieces, then the
        // next request's, so small requests behind a large one still start
        // as soon as the large one's remaining bytes fit in a batch, and
        // the other direction is never held up
        for (size_t c = 0; c < cand.size() && used < batch && pieces < 1024; ++c) {
            Req &q = *cand[c];
            const phos_table *t = q.r.table;
            while (q.issued < q.img_bytes && used < batch && pieces < 1024) {
                // pieces of the next buffer with bytes left (never across a
                // buffer, so the image's padding is left alone)
                while (q.buf < t->n && q.buf_off >= t->size[q.buf]) {
                    ++q.buf;
                    q.buf_off = 0;
                }
                if (q.buf < t->n) {
                    const uint64_t take = std::min(d.chunk, t->size[q.buf] - q.buf_off);
                    const uint64_t io = t->img_off[q.buf] + q.buf_off;
                    if (d2h)        // staging holds the image layout
                        lists[c].push_back(phos_copy_t{q.stg_off + io, io, take, q.buf,
                                                       PHOS_COPY_STAGING_TO_IMAGE});
                    else
                        lists[c].push_back(phos_copy_t{io, q.buf_off, take, q.buf,
                                                       PHOS_COPY_IMAGE_TO_LIVE});
                    q.buf_off += take;
                    used += take;
                    ++pieces;
                }
                while (q.buf < t->n && q.buf_off >= t->size[q.buf]) {
                    ++q.buf;
                    q.buf_off = 0;
                }
                if (q.buf >= t->n) {
                    q.issued = q.img_bytes;
                    is.finishing.push_back(q.ticket);
                }
            }
        }
        cudaStream_t s = d2h ? s_d2h : s_h2d;
        for (size_t c = 0; c < cand.size(); ++c) {
            if (lists[c].empty()) continue;
            Req &q = *cand[c];
            is.members.push_back(q.ticket);
            ++q.inflight;
            const phos_table *t = q.r.table;
            std::vector<phos_copy_t> kern;
            // Runs of pieces that are contiguous on both sides (adjacent
            // buffers whose sizes are multiples of 256, and for a restore
            // adjacent in the address space too) move as one DMA copy once
            // the run reaches dma_min; shorter runs go to the SM kernel
            // piece by piece.
            const std::vector<phos_copy_t> &L = lists[c];
            size_t k = 0;
            while (k < L.size()) {
                auto ptrs = [&](const phos_copy_t &p, const uint8_t **src, uint8_t **dst) {
                    if (d2h) {
                        *src = static_cast<const uint8_t *>(d.d_staging) + p.src_off;
                        *dst = static_cast<uint8_t *>(q.r.host) + p.dst_off;
                    } else {
                        *src = static_cast<const uint8_t *>(q.r.host) + p.src_off;
                        *dst = reinterpret_cast<uint8_t *>(t->base[p.buf] + p.dst_off);
                    }
                };
                const uint8_t *s0;
                uint8_t *d0;
                ptrs(L[k], &s0, &d0);
                uint64_t run = L[k].len;
                size_t e = k + 1;
                while (e < L.size() && run < kMaxRun) {
                    const uint8_t *s1;
                    uint8_t *d1;
                    ptrs(L[e], &s1, &d1);
                    if (s1 != s0 + run || d1 != d0 + run) break;
                    run += L[e].len;
                    ++e;
                }
                if (d.dma_min && run >= d.dma_min) {
                    cudaError_t ce = cudaMemcpyAsync(d0, s0, run, cudaMemcpyDefault, s);
                    if (ce != cudaSuccess) q.res.status = PHOS_ECUDA;
                } else {
                    kern.insert(kern.end(), L.begin() + k, L.begin() + e);
                }
                k = e;
            }
            phos_status e = launch(d2h ? 1 : 2, s, q.r.table, kern, q.r.host, q.r.host_bytes);
            if (e) q.res.status = e;
        }
        is.ev = get_ev();
        cudaEventRecord(is.ev, s);
        inf.push_back(std::move(is));
        ++st.batches;
    }

    // True while an application transfer is being issued or has not
    // completed (retire_app runs first in each turn).
    bool app_busy() const {
        return app_pending[0] || app_pending[1] || !app_inflight.empty();
    }
    void retire_app() {
        for (size_t k = 0; k < app_inflight.size();) {
            if (cudaEventQuery(app_inflight[k].ev) == cudaSuccess) {
                ev_pool.push_back(app_inflight[k].ev);
                app_inflight.erase(app_inflight.begin() + k);
            } else {
                ++k;
            }
        }
    }

    void retire(std::deque<Issue> &inf) {
        while (!inf.empty() && cudaEventQuery(inf.front().ev) == cudaSuccess) {
            Issue &is = inf.front();
            const uint64_t t = now_ns();
            for (uint64_t tk : is.members) --reqs[tk].inflight;
            for (uint64_t tk : is.finishing) {
                Req &q = reqs[tk];
                q.res.state = q.res.status ? 3 : 2;
                q.res.t_done_ns = t;
                q.res.bytes = q.img_bytes;
                if (q.r.kind == PHOS_REQ_CHECKPOINT && q.img_bytes)
                    stg_release(q.stg_off, align_up(q.img_bytes, 256));
                if (q.snap_ev) ev_pool.push_back(q.snap_ev);
                q.snap_ev = nullptr;
                active.erase(std::find(active.begin(), active.end(), tk));
            }
            ev_pool.push_back(is.ev);
            inf.pop_front();
        }
    }

    // Admitted requests cancelled before their last piece was issued end
    // once none of their pieces is in flight (and a checkpoint's snapshot
    // has landed, so its staging can be reused).
    void retire_cancelled() {
        for (size_t k = 0; k < active.size();) {
            Req &q = reqs[active[k]];
            if (q.cancel && q.res.state == 1 && q.issued < q.img_bytes && q.inflight == 0 &&
                (!q.snap_ev || cudaEventQuery(q.snap_ev) == cudaSuccess)) {
                q.res.state = 4;
                q.res.t_done_ns = now_ns();
                if (q.r.kind == PHOS_REQ_CHECKPOINT && q.img_bytes)
                    stg_release(q.stg_off, align_up(q.img_bytes, 256));
                if (q.snap_ev) ev_pool.push_back(q.snap_ev);
                q.snap_ev = nullptr;
                ++st.cancelled;
                active.erase(active.begin() + k);
            } else {
                ++k;
            }
        }
    }

    void loop() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            retire(inflight_d2h);
            retire(inflight_h2d);
            retire_app();
            retire_cancelled();
            admit();
            issue(true);
            issue(false);
            // empty restores / zero-byte checkpoints complete at once
            for (size_t k = 0; k < active.size();) {
                Req &q = reqs[active[k]];
                if (q.img_bytes == 0 && q.res.state == 1) {
                    q.res.state = 2;
                    q.res.t_done_ns = now_ns();
                    active.erase(active.begin() + k);
                } else {
                    ++k;
                }
            }
            if (stop && queue.empty() && active.empty()) break;
            const bool idle = queue.empty() && active.empty() && app_inflight.empty();
            if (idle) {
                cv.wait_for(lk, std::chrono::milliseconds(5));
            } else {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            }
        }
    }
};

extern "C" phos_status phos_server_start(const phos_server_desc_t *d, phos_server_t **out) {
    if (!d || !out) return fail(PHOS_EINVAL, "server_start: NULL argument");
    *out = nullptr;
    if (d->max_slots == 0 || d->chunk == 0 || d->chunk % 256)
        return fail(PHOS_EINVAL, "server_start: max_slots >= 1, chunk a multiple of 256");
    if (d->staging_bytes && !d->d_staging)
        return fail(PHOS_EINVAL, "server_start: staging budget without a staging area");
    phos_server *S = new phos_server();
    S->d = *d;
    cudaGetDevice(&S->device);
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&S->s_snap, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&S->s_d2h, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&S->s_h2d, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaMalloc(&S->d_status, 256)) != cudaSuccess ||
        (e = cudaMemset(S->d_status, 0, 256)) != cudaSuccess) {
        delete S;
        return cuda_fail(e, "server_start");
    }
    for (int r = 0; r < 3; ++r) {
        if ((e = cudaHostAlloc(&S->h_ring[r], S->ring_cap * sizeof(phos_copy_t),
                               cudaHostAllocMapped)) != cudaSuccess ||
            (e = cudaHostGetDevicePointer((void **)&S->h_ring_dev[r], S->h_ring[r], 0)) !=
                cudaSuccess ||
            (e = cudaMalloc(&S->d_ring[r], S->ring_cap * sizeof(phos_copy_t))) != cudaSuccess) {
            delete S;
            return cuda_fail(e, "server_start: rings");
        }
    }
    if (d->staging_bytes) S->free_stg.push_back({0, d->staging_bytes});
    S->th = std::thread([S] { S->loop(); });
    *out = S;
    return PHOS_OK;
}

extern "C" phos_status phos_server_submit(phos_server_t *S, const phos_request_t *r,
                                          uint64_t *ticket) {
    if (!S || !r || !r->table || !ticket) return fail(PHOS_EINVAL, "server_submit: NULL argument");
    if (r->kind != PHOS_REQ_CHECKPOINT && r->kind != PHOS_REQ_RESTORE)
        return fail(PHOS_EINVAL, "server_submit: kind %u", r->kind);
    if (r->host_bytes < r->table->image_bytes || (!r->host && r->table->image_bytes))
        return fail(PHOS_EINVAL, "server_submit: host image smaller than the table's image");
    // callers may submit from any thread: bind the server's device first
    PHOS_CUDA(cudaSetDevice(S->device));
    void *dv = nullptr;
    phos_status st = device_view(r->host, &dv);
    if (st) return st;
    if (r->kind == PHOS_REQ_CHECKPOINT && align_up(r->table->image_bytes, 256) > S->d.staging_bytes)
        return fail(PHOS_EBUDGET, "server_submit: image of %llu bytes exceeds the staging budget",
                    (unsigned long long)r->table->image_bytes);
    std::lock_guard<std::mutex> g(S->mu);
    Req q;
    q.ticket = S->next_ticket++;
    q.r = *r;
    q.r.host = dv;
    memset(&q.res, 0, sizeof q.res);
    q.res.t_submit_ns = now_ns();
    S->reqs[q.ticket] = q;
    S->queue.push_back(q.ticket);
    *ticket = q.ticket;
    S->cv.notify_one();
    return PHOS_OK;
}

extern "C" phos_status phos_server_cancel(phos_server_t *S, uint64_t ticket) {
    if (!S) return fail(PHOS_EINVAL, "server_cancel: NULL server");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(PHOS_EINVAL, "server_cancel: unknown ticket");
    Req &q = it->second;
    if (q.res.state == 0) {
        auto qi = std::find(S->queue.begin(), S->queue.end(), ticket);
        if (qi != S->queue.end()) S->queue.erase(qi);
        q.res.state = 4;
        q.res.t_done_ns = now_ns();
        ++S->st.cancelled;
    } else if (q.res.state == 1) {
        q.cancel = true;
    }
    S->cv.notify_one();
    return PHOS_OK;
}

extern "C" phos_status phos_server_poll(phos_server_t *S, uint64_t ticket, phos_result_t *out) {
    if (!S || !out) return fail(PHOS_EINVAL, "server_poll: NULL argument");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(PHOS_EINVAL, "server_poll: unknown ticket");
    *out = it->second.res;
    return PHOS_OK;
}

static bool host_side(const void *p, bool *ok) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        *ok = false;
        return false;
    }
    *ok = a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeDevice ||
          a.type == cudaMemoryTypeManaged;
    return a.type == cudaMemoryTypeHost;
}

extern "C" phos_status phos_server_app_copy(phos_server_t *S, void *dst, const void *src,
                                            uint64_t bytes, cudaStream_t stream) {
    if (!S || !dst || !src) return fail(PHOS_EINVAL, "server_app_copy: NULL argument");
    PHOS_CUDA(cudaSetDevice(S->device));
    bool ok_d, ok_s;
    const bool hd = host_side(dst, &ok_d), hs = host_side(src, &ok_s);
    if (!ok_d || !ok_s)
        return fail(PHOS_EINVAL, "server_app_copy: pageable or unknown memory (pin the host side)");
    if (hd == hs)
        return fail(PHOS_EINVAL, "server_app_copy: one side must be pinned host memory and the "
                                 "other device memory");
    const bool d2h = hd;
    cudaEvent_t ev;
    {
        // registered before the copy is issued, so no C/R batch issued from
        // here on gets ahead of it
        std::lock_guard<std::mutex> g(S->mu);
        ev = S->get_ev();
        ++S->app_pending[d2h];
    }
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev, stream);
    std::lock_guard<std::mutex> g(S->mu);
    --S->app_pending[d2h];
    if (e != cudaSuccess) {
        S->ev_pool.push_back(ev);
        return cuda_fail(e, "server_app_copy");
    }
    S->app_inflight.push_back(AppCopy{ev, d2h});
    ++S->st.app_copies;
    S->st.app_bytes += bytes;
    S->cv.notify_one();
    return PHOS_OK;
}

extern "C" phos_status phos_server_stats(phos_server_t *S, phos_server_stats_t *out) {
    if (!S || !out) return fail(PHOS_EINVAL, "server_stats: NULL argument");
    std::lock_guard<std::mutex> g(S->mu);
    *out = S->st;
    return PHOS_OK;
}

extern "C" phos_status phos_server_drain(phos_server_t *S, uint32_t timeout_ms) {
    if (!S) return fail(PHOS_EINVAL, "server_drain: NULL server");
    const uint64_t t_end = now_ns() + (uint64_t)timeout_ms * 1000000ull;
    while (true) {
        {
            std::lock_guard<std::mutex> g(S->mu);
            if (S->queue.empty() && S->active.empty()) return PHOS_OK;
        }
        if (now_ns() > t_end) return fail(PHOS_ETIMEDOUT, "server_drain: timed out");
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

extern "C" phos_status phos_server_stop(phos_server_t *S) {
    if (!S) return PHOS_OK;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        S->cv.notify_one();
    }
    S->th.join();
    for (const AppCopy &a : S->app_inflight) {
        cudaEventSynchronize(a.ev);
        cudaEventDestroy(a.ev);
    }
    cudaStreamSynchronize(S->s_snap);
    cudaStreamSynchronize(S->s_d2h);
    cudaStreamSynchronize(S->s_h2d);
    for (auto &kv : S->reqs)
        if (kv.second.snap_ev) cudaEventDestroy(kv.second.snap_ev);
    for (cudaEvent_t e : S->ev_pool) cudaEventDestroy(e);
    for (int r = 0; r < 3; ++r) {
        cudaFreeHost(S->h_ring[r]);
        cudaFree(S->d_ring[r]);
    }
    cudaFree(S->d_status);
    cudaStreamDestroy(S->s_snap);
    cudaStreamDestroy(S->s_d2h);
    cudaStreamDestroy(S->s_h2d);
    delete S;
    return PHOS_OK;
}
