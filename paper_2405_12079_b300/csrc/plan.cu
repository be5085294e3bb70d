// Batched plan: the validation traces and copy lists of many process
// images in one persistent launch, replayed as a CUDA graph (the batched
// form of the data plane; the paper checkpoints each process of a
// multi-process application separately after a global quiesce, Sec. 7
// "Fault tolerance", so many images are independent work).
//
// B300 design
//   * One CTA per SM, 1024 threads.  Phase 1: the validation batches (1024
//     records) of every item are one index space; each CTA takes a
//     contiguous range, which touches one or two items; per item it stages
//     that item's table, permissions and victim bitmaps in shared memory,
//     runs the batched-leader word classification of phos_validate, and
//     folds its counts and victims into per-item accumulators.  Phase 2:
//     the copy tiles of every item are one index space, walked grid-stride;
//     a CTA that finishes validating starts copying while others still
//     validate, so the two HBM streams overlap.
//   * Descriptors are resolved and scanned once, at plan creation, on the
//     host; a launch carries no prologue kernel.  The tile size is the
//     autotuned parameter (64 KiB .. 4 MiB).
//   * The last CTA out writes every item's counts and victim bitmaps and
//     re-zeroes the accumulators, so a plan can be replayed as a graph with
//     no memset node.
#include <string.h>

#include <algorithm>
#include <vector>

#include "copy_dev.cuh"
#include "internal.h"
#include "validate_dev.cuh"

namespace phos {

struct PlanRes {
    const uint8_t *src;
    uint8_t *dst;
    uint64_t len;
};

struct PlanItemDev {
    const uint64_t *base, *size;
    const uint8_t *perm;
    const uint64_t *trace;
    uint64_t n_rec;
    uint32_t *bitmap;
    uint64_t *count;
    uint32_t *victim, *victim_st;
    uint64_t batch0;    // first global validation batch of the item
    uint64_t vacc_off;  // u32 offset of the item's victim accumulators
    uint32_t n, w;
};

struct PlanDev {
    const PlanItemDev *items;
    uint32_t n_items;
    uint64_t vbatches;
    const PlanRes *res;
    const uint64_t *prefix;  // [n_desc + 1] tile prefix
    uint32_t n_desc;
    uint64_t tile;
    unsigned long long *cnt_acc;  // [n_items][4]
    uint32_t *vacc;
    uint32_t *ticket;
    uint32_t *status;
    uint32_t max_n;
};

constexpr uint32_t kPlanThreads = 1024;

__global__ void __launch_bounds__(kPlanThreads, 1) k_plan(const PlanDev P) {
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t nwarps = blockDim.x >> 5;
    Lead *leads = reinterpret_cast<Lead *>(smem);
    uint8_t *cur = smem + sizeof(Lead) * 32 * nwarps;
    unsigned long long *red = reinterpret_cast<unsigned long long *>(cur);
    uint32_t *s_misc = reinterpret_cast<uint32_t *>(cur + 24);  // [0] last, [1] bad
    cur += 32;
    uint64_t *tb = reinterpret_cast<uint64_t *>(cur);
    uint64_t *tl = tb + P.max_n;
    uint8_t *perm = reinterpret_cast<uint8_t *>(tl + P.max_n);
    uint32_t *sv = reinterpret_cast<uint32_t *>(perm + ((P.max_n + 15) & ~15u));
    const uint32_t max_nvw = (P.max_n + 31) / 32;
    uint32_t *svs = sv + max_nvw;
    const uint64_t G = gridDim.x, c = blockIdx.x;
    if (tid == 0) {
        red[0] = red[1] = red[2] = 0;
        s_misc[1] = 0;
    }

    // ---------------- phase 1: validation
    const uint64_t vb0 = P.vbatches * c / G, vb1 = P.vbatches * (c + 1) / G;
    uint32_t j = 0;
    {
        uint32_t lo = 0, cnt = P.n_items;  // last item with batch0 <= vb0
        while (cnt > 0) {
            const uint32_t half = cnt >> 1;
            if (P.items[lo + half].batch0 <= vb0) {
                lo += half + 1;
                cnt -= half + 1;
            } else {
                cnt = half;
            }
        }
        j = lo ? lo - 1 : 0;
    }
    Lead *mine = leads + 32 * warp;
    for (uint64_t bt0 = vb0; bt0 < vb1 && j < P.n_items; ++j) {
        const PlanItemDev it = P.items[j];
        const uint64_t nb_item = (it.n_rec + kBatch - 1) / kBatch;
        const uint64_t seg_end = min(vb1, it.batch0 + nb_item);
        if (seg_end <= bt0) continue;
        const uint32_t n = it.n, nvw = (n + 31) / 32;
        __syncthreads();
        for (uint32_t i = tid; i < n; i += blockDim.x) {
            tb[i] = __ldg(it.base + i);
            const uint64_t sz = __ldg(it.size + i);
            tl[i] = sz >= it.w ? sz - it.w + 1 : 0;
            perm[i] = it.perm[i];
        }
        for (uint32_t i = tid; i < nvw; i += blockDim.x) sv[i] = svs[i] = 0;
        __syncthreads();
        Look L;
        L.n = n;
        L.nf1 = (n + 31) >> 5;
        L.w = it.w;
        L.base = tb;
        L.lim = tl;
        L.size = it.size;
        L.f1 = nullptr;
        L.f2 = nullptr;
        L.perm = perm;
        L.rf = 0;
        Acc acc;
        for (uint64_t bt = bt0 + warp; bt < seg_end; bt += nwarps) {
            const uint64_t lb = bt - it.batch0;
            const uint64_t r0 = lb * kBatch;
            const uint64_t nb = min((uint64_t)kBatch, it.n_rec - r0);
            const uint64_t *recs = it.trace + r0;
            mine[lane] = make_lead(
                L, lane * 32 < nb ? L.lane_search(recs[lane * 32] & PHOS_REC_ADDR_MASK) : -1,
                true);
            __syncwarp();
            uint32_t *bm = it.bitmap + (r0 >> 5);
            if (nb == kBatch)
                batch_pairs<true>(L, recs, 32, lane, mine, bm, sv, svs, acc);
            else
                batch_words<true, false>(L, recs, nb, 32, lane, mine, bm, sv, svs, acc);
            __syncwarp();
        }
        if (__any_sync(0xffffffffu, acc.bad) && lane == 0) s_misc[1] = 1;
        if (lane == 0 && (acc.c0 | acc.c1 | acc.c2)) {
            atomicAdd(&red[0], (unsigned long long)acc.c0);
            atomicAdd(&red[1], (unsigned long long)acc.c1);
            atomicAdd(&red[2], (unsigned long long)acc.c2);
        }
        __syncthreads();
        if (tid == 0) {
            if (red[0]) atomicAdd(&P.cnt_acc[4 * j + 0], red[0]);
            if (red[1]) atomicAdd(&P.cnt_acc[4 * j + 1], red[1]);
            if (red[2]) atomicAdd(&P.cnt_acc[4 * j + 2], red[2]);
            red[0] = red[1] = red[2] = 0;
        }
        for (uint32_t i = tid; i < nvw; i += blockDim.x) {
            if (sv[i]) atomicOr(&P.vacc[it.vacc_off + i], sv[i]);
            if (svs[i]) atomicOr(&P.vacc[it.vacc_off + nvw + i], svs[i]);
        }
        bt0 = seg_end;
    }

    // ---------------- phase 2: copies
    __shared__ uint32_t s_d;
    const uint64_t total = P.prefix[P.n_desc];
    for (uint64_t t = c; t < total; t += G) {
        __syncthreads();
        if (tid == 0) {
            uint32_t lo = 0, cnt = P.n_desc + 1;
            while (cnt > 0) {
                const uint32_t half = cnt >> 1;
                if (P.prefix[lo + half] <= t) {
                    lo += half + 1;
                    cnt -= half + 1;
                } else {
                    cnt = half;
                }
            }
            s_d = lo - 1;
        }
        __syncthreads();
        const PlanRes r = P.res[s_d];
        const uint64_t off = (t - P.prefix[s_d]) * P.tile;
        const uint64_t len = off < r.len ? min(P.tile, r.len - off) : 0;
        copy_block(r.dst + off, r.src + off, len);
    }

    // ---------------- last CTA: publish per-item results
    __syncthreads();
    if (tid == 0 && s_misc[1]) set_status(P.status, PHOS_EINVAL);
    __threadfence();
    __syncthreads();
    if (tid == 0) s_misc[0] = (atomicAdd(P.ticket, 1u) == (uint32_t)(G - 1)) ? 1u : 0u;
    __syncthreads();
    if (!s_misc[0]) return;
    __threadfence();
    for (uint32_t q = warp; q < P.n_items; q += nwarps) {
        const PlanItemDev it = P.items[q];
        const uint32_t nvw = (it.n + 31) / 32;
        if (lane < 3) {
            it.count[lane] = __ldcg(&P.cnt_acc[4 * q + lane]);
            P.cnt_acc[4 * q + lane] = 0;
        }
        for (uint32_t i = lane; i < nvw; i += 32) {
            const uint32_t v = __ldcg(&P.vacc[it.vacc_off + i]);
            const uint32_t vs = __ldcg(&P.vacc[it.vacc_off + nvw + i]);
            if (it.victim) it.victim[i] = v;
            if (it.victim_st) it.victim_st[i] = vs;
            P.vacc[it.vacc_off + i] = 0;
            P.vacc[it.vacc_off + nvw + i] = 0;
        }
    }
    if (tid == 0) *P.ticket = 0;
}

}  // namespace phos

using namespace phos;

struct phos_plan {
    int device = 0;
    std::vector<PlanItemDev> items;
    std::vector<PlanRes> res;
    std::vector<uint64_t> prefix;
    PlanItemDev *d_items = nullptr;
    PlanRes *d_res = nullptr;
    uint64_t *d_prefix = nullptr;
    unsigned long long *d_cnt = nullptr;
    uint32_t *d_vacc = nullptr;
    uint32_t *d_ticket = nullptr;
    uint32_t *d_status = nullptr;
    uint64_t vbatches = 0, vacc_words = 0, tile = 256 * 1024;
    uint32_t max_n = 0;
    size_t smem = 0;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t copy_bytes = 0, records = 0;

    ~phos_plan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
        cudaFree(d_items);
        cudaFree(d_res);
        cudaFree(d_prefix);
        cudaFree(d_cnt);
        cudaFree(d_vacc);
        cudaFree(d_ticket);
        cudaFree(d_status);
    }

    phos_status upload_prefix() {
        prefix.assign(res.size() + 1, 0);
        for (size_t d = 0; d < res.size(); ++d)
            prefix[d + 1] = prefix[d] + (res[d].len + tile - 1) / tile;
        if (!d_prefix) PHOS_CUDA(cudaMalloc(&d_prefix, 8 * prefix.size()));
        PHOS_CUDA(cudaMemcpy(d_prefix, prefix.data(), 8 * prefix.size(), cudaMemcpyHostToDevice));
        return PHOS_OK;
    }

    PlanDev dev() const {
        PlanDev P;
        P.items = d_items;
        P.n_items = (uint32_t)items.size();
        P.vbatches = vbatches;
        P.res = d_res;
        P.prefix = d_prefix;
        P.n_desc = (uint32_t)res.size();
        P.tile = tile;
        P.cnt_acc = d_cnt;
        P.vacc = d_vacc;
        P.ticket = d_ticket;
        P.status = d_status;
        P.max_n = max_n;
        return P;
    }

    phos_status capture() {
        if (exec) {
            cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
        if (graph) {
            cudaGraphDestroy(graph);
            graph = nullptr;
        }
        if (!cap) PHOS_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        PHOS_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        const unsigned G = (unsigned)sm_count(device);
        k_plan<<<G, kPlanThreads, smem, cap>>>(dev());
        cudaError_t le = cudaGetLastError();
        cudaError_t ee = cudaStreamEndCapture(cap, &graph);
        if (le != cudaSuccess) return cuda_fail(le, "plan: kernel launch during capture");
        if (ee != cudaSuccess) return cuda_fail(ee, "plan: cudaStreamEndCapture");
        PHOS_CUDA(cudaGraphInstantiate(&exec, graph, 0));
        return PHOS_OK;
    }
};

extern "C" phos_status phos_plan_create(const phos_plan_item_t *items, uint32_t n_items,
                                        phos_plan_t **out) {
    if (!out || (n_items && !items)) return fail(PHOS_EINVAL, "plan_create: NULL argument");
    *out = nullptr;
    phos_plan *P = new phos_plan();
    cudaGetDevice(&P->device);
    std::vector<phos_copy_t> h;
    uint64_t batch = 0, vacc = 0;
    for (uint32_t q = 0; q < n_items; ++q) {
        const phos_plan_item_t &it = items[q];
        const phos_table *t = it.table;
        if (!t) {
            delete P;
            return fail(PHOS_EINVAL, "plan_create: item %u has no table", q);
        }
        if (it.n_rec && (!it.d_trace || !it.d_bitmap || ((uintptr_t)it.d_trace & 15) ||
                         it.access_bytes == 0 || (t->n && !it.d_perm) || !it.d_count)) {
            delete P;
            return fail(PHOS_EINVAL, "plan_create: item %u validation arguments", q);
        }
        PlanItemDev d;
        d.base = t->view.base;
        d.size = t->view.size;
        d.perm = it.d_perm;
        d.trace = it.d_trace;
        d.n_rec = it.n_rec;
        d.bitmap = it.d_bitmap;
        d.count = it.d_count;
        d.victim = it.d_victim;
        d.victim_st = it.d_victim_st;
        d.batch0 = batch;
        d.vacc_off = vacc;
        d.n = t->n;
        d.w = it.access_bytes ? it.access_bytes : 1;
        if (!it.d_count) {
            delete P;
            return fail(PHOS_EINVAL, "plan_create: item %u has no count output", q);
        }
        batch += (it.n_rec + kBatch - 1) / kBatch;
        vacc += 2ull * ((t->n + 31) / 32);
        P->max_n = std::max(P->max_n, t->n);
        P->records += it.n_rec;
        P->items.push_back(d);
        // resolve the item's copies on the host
        if (it.n_copy) {
            if (!it.d_list) {
                delete P;
                return fail(PHOS_EINVAL, "plan_create: item %u has copies but no list", q);
            }
            h.resize(it.n_copy);
            cudaError_t e = cudaMemcpy(h.data(), it.d_list, sizeof(phos_copy_t) * it.n_copy,
                                       cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                delete P;
                return cuda_fail(e, "plan_create: reading a copy list");
            }
            void *stg = nullptr, *img = nullptr;
            phos_status r = device_view(it.staging, &stg);
            if (!r) r = device_view(it.image, &img);
            if (r) {
                delete P;
                return r;
            }
            for (uint32_t k = 0; k < it.n_copy; ++k) {
                const phos_copy_t &c = h[k];
                const uint32_t dir = c.flags & PHOS_COPY_DIR_MASK;
                auto live_ok = [&](uint64_t off) {
                    return c.buf < t->n && off <= t->size[c.buf] && c.len <= t->size[c.buf] - off;
                };
                auto area_ok = [&](const void *p, uint64_t bytes, uint64_t off) {
                    return p && off <= bytes && c.len <= bytes - off;
                };
                PlanRes pr{nullptr, nullptr, c.len};
                bool ok = (c.flags & ~(uint32_t)PHOS_COPY_DIR_MASK) == 0;
                switch (dir) {
                    case PHOS_COPY_LIVE_TO_STAGING:
                        ok = ok && live_ok(c.src_off) && area_ok(stg, it.staging_bytes, c.dst_off);
                        if (ok) {
                            pr.src = (const uint8_t *)(t->base[c.buf] + c.src_off);
                            pr.dst = (uint8_t *)stg + c.dst_off;
                        }
                        break;
                    case PHOS_COPY_LIVE_TO_IMAGE:
                        ok = ok && live_ok(c.src_off) && area_ok(img, it.image_bytes, c.dst_off);
                        if (ok) {
                            pr.src = (const uint8_t *)(t->base[c.buf] + c.src_off);
                            pr.dst = (uint8_t *)img + c.dst_off;
                        }
                        break;
                    case PHOS_COPY_STAGING_TO_IMAGE:
                        ok = ok && area_ok(stg, it.staging_bytes, c.src_off) &&
                             area_ok(img, it.image_bytes, c.dst_off);
                        if (ok) {
                            pr.src = (const uint8_t *)stg + c.src_off;
                            pr.dst = (uint8_t *)img + c.dst_off;
                        }
                        break;
                    case PHOS_COPY_IMAGE_TO_LIVE:
                        ok = ok && area_ok(img, it.image_bytes, c.src_off) && live_ok(c.dst_off);
                        if (ok) {
                            pr.src = (const uint8_t *)img + c.src_off;
                            pr.dst = (uint8_t *)(t->base[c.buf] + c.dst_off);
                        }
                        break;
                    default:
                        ok = false;
                }
                if (!ok) {
                    delete P;
                    return fail(PHOS_EINVAL, "plan_create: item %u descriptor %u is invalid "
                                             "(bounds, direction, or a flag the plan lacks)",
                                q, k);
                }
                if (pr.len) {
                    P->res.push_back(pr);
                    P->copy_bytes += pr.len;
                }
            }
        }
    }
    P->vbatches = batch;
    P->vacc_words = vacc;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device);
    const uint32_t mn = P->max_n, nvw = (mn + 31) / 32;
    P->smem = sizeof(Lead) * kPlanThreads + 32 + 16ull * mn + ((mn + 15) & ~15u) + 8ull * nvw;
    cudaFuncAttributes fa;
    size_t static_smem = 0;
    if (cudaFuncGetAttributes(&fa, (const void *)k_plan) == cudaSuccess) static_smem = fa.sharedSizeBytes;
    if (P->smem + static_smem > (size_t)(optin > 0 ? optin : 227 * 1024)) {
        delete P;
        return fail(PHOS_EINVAL, "plan_create: a table of %u buffers does not fit the plan's "
                                 "shared memory", mn);
    }
    cudaError_t e;
    const size_t ni = std::max<size_t>(P->items.size(), 1), nr = std::max<size_t>(P->res.size(), 1);
    if ((e = cudaMalloc(&P->d_items, sizeof(PlanItemDev) * ni)) != cudaSuccess ||
        (e = cudaMalloc(&P->d_res, sizeof(PlanRes) * nr)) != cudaSuccess ||
        (e = cudaMalloc(&P->d_cnt, 32 * ni)) != cudaSuccess ||
        (e = cudaMalloc(&P->d_vacc, 4 * std::max<uint64_t>(vacc, 1))) != cudaSuccess ||
        (e = cudaMalloc(&P->d_ticket, 256)) != cudaSuccess ||
        (e = cudaMalloc(&P->d_status, 256)) != cudaSuccess) {
        delete P;
        return fail(PHOS_ENOMEM, "plan_create: cudaMalloc: %s", cudaGetErrorString(e));
    }
    if ((e = cudaMemcpy(P->d_items, P->items.data(), sizeof(PlanItemDev) * P->items.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(P->d_res, P->res.data(), sizeof(PlanRes) * P->res.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(P->d_cnt, 0, 32 * ni)) != cudaSuccess ||
        (e = cudaMemset(P->d_vacc, 0, 4 * std::max<uint64_t>(vacc, 1))) != cudaSuccess ||
        (e = cudaMemset(P->d_ticket, 0, 256)) != cudaSuccess ||
        (e = cudaMemset(P->d_status, 0, 256)) != cudaSuccess) {
        delete P;
        return cuda_fail(e, "plan_create: upload");
    }
    phos_status r = P->upload_prefix();
    if (!r) {
        cudaError_t ae = cudaFuncSetAttribute((const void *)k_plan,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)P->smem);
        if (ae != cudaSuccess) r = cuda_fail(ae, "plan_create: cudaFuncSetAttribute");
    }
    if (!r) r = P->capture();
    if (r) {
        delete P;
        return r;
    }
    *out = P;
    return PHOS_OK;
}

extern "C" phos_status phos_plan_launch(phos_plan_t *P, phos_stream_t stream) {
    if (!P) return fail(PHOS_EINVAL, "plan_launch: NULL plan");
    PHOS_CUDA(cudaGraphLaunch(P->exec, static_cast<cudaStream_t>(stream)));
    count_launch();
    return PHOS_OK;
}

extern "C" phos_status phos_plan_set_tile(phos_plan_t *P, uint64_t tile_bytes) {
    if (!P) return fail(PHOS_EINVAL, "plan_set_tile: NULL plan");
    if (tile_bytes < 4096 || tile_bytes % 4096 || tile_bytes > (16ull << 20))
        return fail(PHOS_EINVAL, "plan_set_tile: %llu", (unsigned long long)tile_bytes);
    PHOS_CUDA(cudaDeviceSynchronize());
    P->tile = tile_bytes;
    phos_status r = P->upload_prefix();
    if (r) return r;
    return P->capture();
}

extern "C" phos_status phos_plan_autotune(phos_plan_t *P, phos_stream_t stream,
                                          uint64_t *best_tile, float *best_ms) {
    if (!P) return fail(PHOS_EINVAL, "plan_autotune: NULL plan");
    static const uint64_t cand[] = {64ull << 10, 128ull << 10, 256ull << 10, 512ull << 10,
                                    1ull << 20,  2ull << 20,   4ull << 20};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t a, b;
    PHOS_CUDA(cudaEventCreate(&a));
    PHOS_CUDA(cudaEventCreate(&b));
    uint64_t bt = P->tile;
    float bm = 1e30f;
    phos_status r = PHOS_OK;
    for (uint64_t tile : cand) {
        if ((r = phos_plan_set_tile(P, tile))) break;
        for (int w = 0; w < 2 && !r; ++w) r = phos_plan_launch(P, stream);
        if (r) break;
        float best = 1e30f;
        for (int rep = 0; rep < 5; ++rep) {
            cudaEventRecord(a, s);
            if ((r = phos_plan_launch(P, stream))) break;
            cudaEventRecord(b, s);
            cudaEventSynchronize(b);
            float ms = 0;
            cudaEventElapsedTime(&ms, a, b);
            best = std::min(best, ms);
        }
        if (r) break;
        if (best < bm) {
            bm = best;
            bt = tile;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (r) return r;
    r = phos_plan_set_tile(P, bt);
    if (best_tile) *best_tile = bt;
    if (best_ms) *best_ms = bm;
    return r;
}

extern "C" phos_status phos_plan_info(const phos_plan_t *P, uint64_t *records, uint64_t *copy_bytes,
                                      uint64_t *tile_bytes, uint32_t *status_out) {
    if (!P) return fail(PHOS_EINVAL, "plan_info: NULL plan");
    if (records) *records = P->records;
    if (copy_bytes) *copy_bytes = P->copy_bytes;
    if (tile_bytes) *tile_bytes = P->tile;
    if (status_out) PHOS_CUDA(cudaMemcpy(status_out, P->d_status, 4, cudaMemcpyDeviceToHost));
    return PHOS_OK;
}

extern "C" phos_status phos_plan_destroy(phos_plan_t *P) {
    if (P) {
        cudaDeviceSynchronize();
        delete P;
    }
    return PHOS_OK;
}
