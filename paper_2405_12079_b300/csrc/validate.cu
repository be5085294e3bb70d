// Access validation (PhoenixOS Sec. 4.1 "Runtime validation"; the read
// check of Sec. 6): every recorded load/store address is looked up in the
// sorted buffer table and checked against the permission speculated for
// its buffer.
//
// B300 design
//   * Persistent grid, one CTA per SM (148), each owning a contiguous range
//     of 2048-record tiles (16 KiB).  Tiles stream HBM -> shared memory with
//     one-dimensional bulk copies (TMA engine) into a ring of 2..6 stages,
//     completion tracked by mbarriers: the only HBM traffic is the trace
//     read once (8 B/record) plus the bitmap written once (1/8 B/record).
//   * The table (base, per-call access limit, two fence levels), the
//     permission bytes and the victim bitmaps sit in shared memory when
//     they fit (tables of up to ~11k buffers); larger tables are read
//     through L1/L2.
//   * Lookup is warp-cooperative: the 32 lanes of a warp hold 32
//     consecutive records; one 32-ary search (top level held in registers,
//     then fence1 and base in shared memory, one ballot per level,
//     conflict-free reads) finds the interval of lane 0's record, every
//     lane checks its own record against that interval with one unsigned
//     compare, and only lanes that miss fall back to a private binary
//     search.  Coalesced traces (a warp's 32 accesses in one buffer)
//     therefore cost one search per 32 records.
//   * Stages are released per warp: the last warp to finish a stage
//     refills it, so warps never wait for each other inside the loop.
//   * Results: ballot -> one bitmap word per warp; popc -> per-warp counts;
//     shared-memory atomics for victims; one last-block reduction writes
//     the counts and victim bitmaps (overwriting the outputs, no memset).
//   * The ascending index list is a second, optional launch: each CTA takes
//     the exclusive prefix of the per-CTA violation counts and compacts its
//     own bitmap words with a block scan, so the order is deterministic.
#include <stdio.h>

#include "internal.h"
#include "ptx.cuh"
#include "validate_dev.cuh"

namespace phos {

constexpr uint32_t kTileRec = 2048;
constexpr uint32_t kTileBytes = kTileRec * 8;
constexpr uint32_t kValThreads = 1024;
constexpr uint32_t kMaxStages = 8;
constexpr uint32_t kWaitLimit = 1u << 24;   // probes before a tile wait gives up

struct ValParams {
    ProtoRule rule{};   // kind 0: none (see ProtoRule)
    TableDev tab;
    const uint8_t *perm;
    const uint64_t *trace;
    uint64_t n_rec;
    uint64_t tiles;
    uint32_t *bitmap;
    uint64_t *count;
    uint32_t *victim;
    uint32_t *victim_st;
    uint32_t *status;
    // scratch
    uint64_t *cta_cnt;  // [grid][4]
    uint32_t *vacc;     // [2][nvw], zero between calls
    uint32_t *ticket;   // zero between calls
    unsigned long long *next;  // batched variant: next batch to take, zero between calls
    uint32_t w;
    uint32_t nvw;
    uint32_t stages;
    uint32_t wpb;       // batched variant: bitmap words per warp batch
    uint32_t wait_limit;  // ring variant: probes of a staged tile's mbarrier
};

// Classify the 32 records of one bitmap word (one per lane) and write the
// word.  kFull: every lane holds a record.
template <bool kFull, bool kSmemLim>
__device__ __forceinline__ void word(const Look &L, uint64_t rec, bool valid, uint32_t lane,
                                     uint32_t *bm_word, uint32_t *sv, uint32_t *svs, Acc &acc) {
    if (kFull) valid = true;
    const uint64_t a = rec & PHOS_REC_ADDR_MASK;
    const uint32_t hi = (uint32_t)(rec >> 32);
    const bool st = (int32_t)hi < 0;
    const bool bad = (hi & 0x7E000000u) != 0;
    // leader: lane 0's address (any choice is correct; lanes that miss fall
    // back to their own search)
    const uint64_t x = __shfl_sync(0xffffffffu, a, 0);
    const int i0 = L.search(x, lane);
    int bi = i0;
    uint32_t pm = 0;
    bool hit = false;
    if (i0 >= 0) {
        const uint64_t b0 = L.base[i0];
        const uint64_t l0 = L.limit(i0, kSmemLim);
        pm = L.perm[i0];
        hit = (a - b0) < l0;
    }
    hit = hit && !bad && valid;
    const bool miss = valid && !bad && !hit;
    if (__ballot_sync(0xffffffffu, miss)) {
        if (miss) {
            const int ii = L.lane_search(a);
            if (ii >= 0 && (a - L.base[ii]) < L.limit(ii, kSmemLim)) {
                hit = true;
                bi = ii;
                pm = L.perm[ii];
            }
        }
    }
    const bool viol = valid && !(hit && (pm & (st ? 2u : 1u)));
    const uint32_t vw = __ballot_sync(0xffffffffu, viol);
    if (lane == 0) *bm_word = vw;
    if (vw) {
        const uint32_t sw = __ballot_sync(0xffffffffu, viol && st);
        const uint32_t uw = __ballot_sync(0xffffffffu, valid && !hit);
        if (lane == 0) {
            acc.c0 += __popc(vw);
            acc.c1 += __popc(sw);
            acc.c2 += __popc(uw);
        }
        if (viol && hit) {
            atomicOr(&sv[bi >> 5], 1u << (bi & 31));
            if (st) atomicOr(&svs[bi >> 5], 1u << (bi & 31));
        }
        acc.bad |= bad;
    }
}

// Last CTA: sum the per-CTA counts.  Warp 0 alone, lane-strided loads and
// a shuffle reduction: every thread adding into shared 64-bit counters
// instead serialised for ~12 us with 148 CTAs.
__device__ __forceinline__ void sum_cta_counts(const uint64_t *cta_cnt, uint64_t G, uint32_t tid,
                                               unsigned long long *red) {
    if (tid >= 32) return;
    unsigned long long a0 = 0, a1 = 0, a2 = 0;
    for (uint64_t q = tid; q < G; q += 32) {
        a0 += __ldcg(cta_cnt + q * 4 + 0);
        a1 += __ldcg(cta_cnt + q * 4 + 1);
        a2 += __ldcg(cta_cnt + q * 4 + 2);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_down_sync(0xffffffffu, a0, o);
        a1 += __shfl_down_sync(0xffffffffu, a1, o);
        a2 += __shfl_down_sync(0xffffffffu, a2, o);
    }
    if (tid == 0) {
        red[0] = a0;
        red[1] = a1;
        red[2] = a2;
    }
}

template <bool kSmemTable>
__global__ void __launch_bounds__(kValThreads, 1) k_validate(const ValParams p) {
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t nwarps = blockDim.x >> 5;
    const uint32_t S = p.stages, n = p.tab.n, nvw = p.nvw;
    uint64_t *ring = reinterpret_cast<uint64_t *>(smem);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + (size_t)S * kTileBytes);
    uint32_t *used = reinterpret_cast<uint32_t *>(mbar + kMaxStages);
    uint32_t *issued = used + kMaxStages;
    uint8_t *cur = reinterpret_cast<uint8_t *>(issued + kMaxStages);
    unsigned long long *red = reinterpret_cast<unsigned long long *>(cur);
    uint32_t *flag = reinterpret_cast<uint32_t *>(cur + 24);
    uint32_t *last = flag + 1;
    cur += 32;
    const uint32_t nf1 = (n + 31) >> 5, nf2 = (n + 1023) >> 10;
    Look L;
    L.n = n;
    L.nf1 = nf1;
    L.w = p.w;
    L.base = p.tab.base;
    L.size = p.tab.size;
    L.lim = nullptr;
    L.f1 = p.tab.fence1;
    L.f2 = p.tab.fence2;
    if (kSmemTable) {
        uint64_t *tb = reinterpret_cast<uint64_t *>(cur);
        uint64_t *tl = tb + n, *t1 = tl + n, *t2 = t1 + nf1;
        const uint32_t w = p.w;
        for (uint32_t i = tid; i < n; i += blockDim.x) {
            tb[i] = __ldg(p.tab.base + i);
            const uint64_t sz = __ldg(p.tab.size + i);
            tl[i] = sz >= w ? sz - w + 1 : 0;
        }
        for (uint32_t i = tid; i < nf1; i += blockDim.x) t1[i] = __ldg(p.tab.fence1 + i);
        for (uint32_t i = tid; i < nf2; i += blockDim.x) t2[i] = __ldg(p.tab.fence2 + i);
        L.base = tb;
        L.lim = tl;
        L.f1 = t1;
        L.f2 = t2;
        cur += 8ull * (2 * n + nf1 + nf2);
    }
    uint8_t *perm = cur;
    cur += (n + 15) & ~15u;
    uint32_t *sv = reinterpret_cast<uint32_t *>(cur);
    uint32_t *svs = sv + nvw;
    L.perm = perm;

    for (uint32_t i = tid; i < n; i += blockDim.x) perm[i] = p.perm[i];
    for (uint32_t i = tid; i < nvw; i += blockDim.x) sv[i] = svs[i] = 0;
    if (tid == 0) {
        for (uint32_t q = 0; q < S; ++q) {
            mbar_init(&mbar[q], 1);
            used[q] = 0;
            issued[q] = ~0u;
        }
        fence_mbar_init();
        red[0] = red[1] = red[2] = 0;
        *flag = 0;
    }
    __syncthreads();
    // top search level in registers: base (n <= 32), fence1 (n <= 1024) or
    // fence2 (larger tables), one entry per lane
    {
        const uint64_t kMax = ~0ull;
        if (n <= 32)
            L.rf = lane < n ? L.base[lane] : kMax;
        else if (n <= 1024)
            L.rf = lane < nf1 ? L.f1[lane] : kMax;
        else
            L.rf = lane < nf2 ? L.f2[lane] : kMax;
    }

    const uint64_t G = gridDim.x, c = blockIdx.x;
    const uint64_t t0 = p.tiles * c / G, t1 = p.tiles * (c + 1) / G;
    const uint32_t ntl = (uint32_t)(t1 - t0);

    auto issue = [&](uint32_t j) {
        const uint32_t s = j % S;
        const uint64_t r0 = (t0 + j) * kTileRec;
        const uint64_t cnt = min((uint64_t)kTileRec, p.n_rec - r0);
        const uint32_t bytes = (uint32_t)(cnt * 8);
        const uint32_t bulk = bytes & ~15u;
        uint64_t *dst = ring + (size_t)s * kTileRec;
        if (bytes & 8) dst[cnt - 1] = p.trace[r0 + cnt - 1];
        mbar_arrive_expect_tx(&mbar[s], bulk);
        if (bulk) bulk_g2s(dst, p.trace + r0, bulk, &mbar[s]);
    };

    if (tid == 0)
        for (uint32_t j = 0; j < ntl && j < S; ++j) {
            issued[j] = j;
            issue(j);
        }
    __syncthreads();

    // Every warp walks all of the CTA's tiles, taking words warp and
    // warp + 32 of each; warps run independently (no block barrier per
    // tile).  The last warp to finish a stage refills it with the tile S
    // ahead.
    Acc acc;
    uint32_t s = 0, par = 0;
    uint64_t r0 = t0 * kTileRec;
    for (uint32_t j = 0; j < ntl; ++j) {
        if (!mbar_wait_bounded(&mbar[s], par, p.wait_limit)) {
            if (lane == 0) atomicOr(flag, 1u);
            break;
        }
        const uint32_t cnt = (uint32_t)min((uint64_t)kTileRec, p.n_rec - r0);
        const uint64_t *tile = ring + (size_t)s * kTileRec;
        uint32_t *bmw = p.bitmap + (r0 >> 5);
        if (cnt == kTileRec) {
            for (uint32_t wi = warp; wi < kTileRec / 32; wi += nwarps)
                word<true, kSmemTable>(L, tile[wi * 32 + lane], true, lane, bmw + wi, sv, svs,
                                       acc);
        } else {
            const uint32_t nw = (cnt + 31) >> 5;
            for (uint32_t wi = warp; wi < nw; wi += nwarps) {
                const uint32_t rl = wi * 32 + lane;
                const bool valid = rl < cnt;
                word<false, kSmemTable>(L, valid ? tile[rl] : 0ull, valid, lane, bmw + wi, sv,
                                        svs, acc);
            }
        }
        // release the stage; the last warp out refills it
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            if (atomicAdd(&used[s], 1u) == nwarps - 1) {
                used[s] = 0;
                const uint32_t nj = j + S;
                if (nj < ntl) {
                    issued[s] = nj;
                    fence_proxy_async_smem();
                    issue(nj);
                } else {
                    issued[s] = ~0u;
                }
            }
        }
        r0 += kTileRec;
        if (++s == S) {
            s = 0;
            par ^= 1u;
        }
    }
    __syncthreads();
    if (*flag) {
        // a bulk copy did not complete in time: wait (bounded) for what is
        // still in flight before the CTA's shared memory is released
        if (tid == 0) {
            for (uint32_t q = 0; q < S; ++q)
                if (issued[q] != ~0u) mbar_wait_bounded(&mbar[q], (issued[q] / S) & 1u);
            set_status(p.status, PHOS_ETIMEDOUT);
        }
    }
    if (__any_sync(0xffffffffu, acc.bad) && lane == 0) set_status(p.status, PHOS_EINVAL);
    if (lane == 0 && (acc.c0 | acc.c1 | acc.c2)) {
        atomicAdd(&red[0], (unsigned long long)acc.c0);
        atomicAdd(&red[1], (unsigned long long)acc.c1);
        atomicAdd(&red[2], (unsigned long long)acc.c2);
    }
    __syncthreads();
    if (tid == 0) {
        p.cta_cnt[c * 4 + 0] = red[0];
        p.cta_cnt[c * 4 + 1] = red[1];
        p.cta_cnt[c * 4 + 2] = red[2];
    }
    for (uint32_t i = tid; i < nvw; i += blockDim.x) {
        if (sv[i]) atomicOr(&p.vacc[i], sv[i]);
        if (svs[i]) atomicOr(&p.vacc[nvw + i], svs[i]);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) *last = (atomicAdd(p.ticket, 1u) == (uint32_t)(G - 1)) ? 1u : 0u;
    __syncthreads();
    if (!*last) return;
    // last CTA: every other CTA has published its partials
    __threadfence();
    sum_cta_counts(p.cta_cnt, G, tid, red);
    for (uint32_t i = tid; i < nvw; i += blockDim.x) {
        const uint32_t v = __ldcg(p.vacc + i), vs = __ldcg(p.vacc + nvw + i);
        if (p.victim) p.victim[i] = v;
        if (p.victim_st) p.victim_st[i] = vs;
        p.vacc[i] = 0;
        p.vacc[nvw + i] = 0;
    }
    __syncthreads();
    if (tid == 0) {
        p.count[0] = red[0];
        p.count[1] = red[1];
        p.count[2] = red[2];
        *p.ticket = 0;
    }
}

template <bool kSmemTable, bool kDyn>
__global__ void __launch_bounds__(kValThreads, 1) k_validate_b(const ValParams p) {
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t nwarps = blockDim.x >> 5;
    const uint32_t n = p.tab.n, nvw = p.nvw;
    Lead *leads = reinterpret_cast<Lead *>(smem);             // [nwarps][2][32]
    uint8_t *cur = smem + sizeof(Lead) * 64 * nwarps;
    unsigned long long *red = reinterpret_cast<unsigned long long *>(cur);
    uint32_t *last = reinterpret_cast<uint32_t *>(cur + 24);
    cur += 32;
    const uint32_t nf1 = (n + 31) >> 5;
    Look L;
    L.n = n;
    L.nf1 = nf1;
    L.w = p.w;
    L.base = p.tab.base;
    L.size = p.tab.size;
    L.lim = nullptr;
    L.f1 = p.tab.fence1;
    L.f2 = p.tab.fence2;
    L.rf = 0;
    if (kSmemTable) {
        uint64_t *tb = reinterpret_cast<uint64_t *>(cur);
        uint64_t *tl = tb + n;
        const uint32_t w = p.w;
        for (uint32_t i = tid; i < n; i += blockDim.x) {
            tb[i] = __ldg(p.tab.base + i);
            const uint64_t sz = __ldg(p.tab.size + i);
            tl[i] = sz >= w ? sz - w + 1 : 0;
        }
        L.base = tb;
        L.lim = tl;
        cur += 16ull * n;
    }
    uint8_t *perm = cur;
    cur += (n + 15) & ~15u;
    uint32_t *sv = reinterpret_cast<uint32_t *>(cur);
    uint32_t *svs = sv + nvw;
    L.perm = perm;
    for (uint32_t i = tid; i < n; i += blockDim.x) perm[i] = p.perm[i];
    for (uint32_t i = tid; i < nvw; i += blockDim.x) sv[i] = svs[i] = 0;
    if (tid == 0) red[0] = red[1] = red[2] = 0;
    __syncthreads();

    const uint64_t G = gridDim.x, c = blockIdx.x;
    const uint32_t W = p.wpb;
    const uint64_t brec = 32ull * W;
    const uint64_t nbatch = (p.n_rec + brec - 1) / brec;
    // kDyn (traces of more batches than the grid has warps): warps take
    // batches from a shared counter, one batch ahead of the one they work
    // on, so fast warps take more.  A static assignment (each CTA a
    // contiguous range, or batches grid-stride) left warps finishing up to
    // 60 us apart on a 400 us launch (global-timer stamps per warp), and the
    // launch waits for the last one.  Otherwise batches go grid-stride by
    // the warp's index in the grid (CTA-minor), with no atomics: on a 1.3M-record trace
    // (one batch or none per warp) one atomic per warp on a single address
    // cost ~5 us.  Either way every batch is taken exactly once.
    const uint64_t b1 = nbatch;
    const uint64_t nfull = p.n_rec / brec;
    const uint64_t TW = G * (blockDim.x >> 5);
    Lead *mine = leads + 64 * warp;
    Acc acc;
    // CTA-minor: batch b goes to CTA b % G, so a trace of fewer batches
    // than warps spreads over every CTA instead of filling the first ones
    uint64_t bt = (uint64_t)warp * G + c;
    auto grab = [&]() -> uint64_t {
        if (!kDyn) return bt + TW;
        unsigned long long g = 0;
        if (lane == 0) g = atomicAdd(p.next, 1ull);
        return __shfl_sync(0xffffffffu, g, 0);
    };
    if (kDyn) bt = grab();
    // Full batches run as one stream per warp: the leader records of the
    // warp's next batch are loaded a batch ahead and the record ring runs on
    // into that batch's first pairs, so no batch begins with a load the warp
    // has to wait for.  Two leader sets per warp alternate.
    {
        const uint32_t npair = W >> 1;           // W is 8, 16 or 32
        const ulonglong2 z = make_ulonglong2(0, 0);
        ulonglong2 r[4];
        uint64_t xl = 0;
        if (bt < b1 && bt < nfull) {
            const uint64_t *rc = p.trace + bt * brec;
            xl = lane < W ? rc[lane * 32] : 0ull;
            const ulonglong2 *pc = reinterpret_cast<const ulonglong2 *>(rc) + lane;
#pragma unroll
            for (uint32_t u = 0; u < 3; ++u) r[u] = u < npair ? pc[u * 32] : z;
        }
        uint32_t sel = 0;
        const uint32_t half = lane >> 4;
        while (bt < nfull) {
            const uint64_t nt = grab();
            const bool more = nt < nfull;
            Lead *ldp = mine + 32 * sel;
            ldp[lane] = make_lead(L, lane < W ? L.lane_search(xl & PHOS_REC_ADDR_MASK) : -1,
                                  kSmemTable);
            const uint64_t *rn = p.trace + (more ? nt : bt) * brec;
            xl = (more && lane < W) ? rn[lane * 32] : 0ull;
            // the next batch into L2 while this one is worked on (one batch
            // ahead: two ahead thrashed L2 and measured 25 % slower)
            if (more && lane == 0)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(rn),
                             "r"((uint32_t)(brec * 8)) : "memory");
            __syncwarp();
            const ulonglong2 *pc = reinterpret_cast<const ulonglong2 *>(p.trace + bt * brec) + lane;
            const ulonglong2 *pn = reinterpret_cast<const ulonglong2 *>(rn) + lane;
            uint32_t myvw = 0;
#pragma unroll 1
            for (uint32_t q0 = 0; q0 < npair; q0 += 4) {
#pragma unroll
                for (uint32_t u = 0; u < 4; ++u) {
                    const uint32_t q = q0 + u, g = q + 3;
                    // streaming loads: every record is read once
                    r[(u + 3) & 3] = g < npair ? __ldcs(pc + g * 32)
                                               : (more ? __ldcs(pn + (g - npair) * 32) : z);
                    pair_step<kSmemTable>(L, r[u], ldp[2 * q + half], q, lane, sv, svs, acc,
                                          myvw);
                }
            }
            if (lane < W) p.bitmap[(bt * brec >> 5) + lane] = myvw;
            bt = nt;
            sel ^= 1;
        }
    }
    // the trace's last, partial batch (if this warp took it)
    if (bt < b1) {
        const uint64_t r0 = bt * brec;
        const uint64_t nb = min(brec, p.n_rec - r0);
        const uint64_t *recs = p.trace + r0;
        // leaders: lane j searches the first record of word j
        mine[lane] = make_lead(
            L, (lane < W && lane * 32 < nb) ? L.lane_search(recs[lane * 32] & PHOS_REC_ADDR_MASK)
                                            : -1,
            kSmemTable);
        __syncwarp();
        uint32_t *bm = p.bitmap + (r0 >> 5);
        if (nb == brec)
            batch_pairs<kSmemTable>(L, recs, W, lane, mine, bm, sv, svs, acc);
        else
            batch_words<kSmemTable, false>(L, recs, nb, W, lane, mine, bm, sv, svs, acc);
        __syncwarp();
    }
    if (__any_sync(0xffffffffu, acc.bad) && lane == 0) set_status(p.status, PHOS_EINVAL);
    if (lane == 0 && (acc.c0 | acc.c1 | acc.c2)) {
        atomicAdd(&red[0], (unsigned long long)acc.c0);
        atomicAdd(&red[1], (unsigned long long)acc.c1);
        atomicAdd(&red[2], (unsigned long long)acc.c2);
    }
    __syncthreads();
    if (tid == 0) {
        p.cta_cnt[c * 4 + 0] = red[0];
        p.cta_cnt[c * 4 + 1] = red[1];
        p.cta_cnt[c * 4 + 2] = red[2];
    }
    for (uint32_t i = tid; i < nvw; i += blockDim.x) {
        if (sv[i]) atomicOr(&p.vacc[i], sv[i]);
        if (svs[i]) atomicOr(&p.vacc[nvw + i], svs[i]);
    }
    // the CTA's writes are ordered before its ticket by the barrier and one
    // fence of the thread that takes the ticket (the grid-barrier pattern);
    // the last CTA's thread fences again before its CTA reads the others'
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        *last = (atomicAdd(p.ticket, 1u) == (uint32_t)(G - 1)) ? 1u : 0u;
        if (*last) __threadfence();
    }
    __syncthreads();
    if (!*last) return;
    sum_cta_counts(p.cta_cnt, G, tid, red);
    // the word after *last in dynamic shared memory (static shared memory
    // would cut into the 227 KB dynamic opt-in)
    volatile uint32_t *s_hit = last + 1;
    const uint32_t rk = p.rule.kind;
    if (rk) {
        if (tid == 0) *s_hit = 0;
        __syncthreads();
    }
    for (uint32_t i = tid; i < nvw; i += blockDim.x) {
        const uint32_t v = __ldcg(p.vacc + i), vs = __ldcg(p.vacc + nvw + i);
        if (p.victim) p.victim[i] = v;
        if (p.victim_st) p.victim_st[i] = vs;
        p.vacc[i] = 0;
        p.vacc[nvw + i] = 0;
        if (rk) {
            // the protocol's response to this validation (see ProtoRule)
            uint32_t m = rk == 3 ? v : vs;
            while (m) {
                const uint32_t b = i * 32 + (uint32_t)(__ffs(m) - 1);
                m &= m - 1;
                if (b >= n) break;
                if (rk == 1) {
                    if (p.rule.flags[b]) p.rule.dirty[b] = 1;
                } else if (!p.rule.flags[b]) {
                    *s_hit = 1;
                }
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        p.count[0] = red[0];
        p.count[1] = red[1];
        p.count[2] = red[2];
        *p.ticket = 0;
        *p.next = 0;
        if (rk) {
            uint64_t *acc = p.rule.acc;
            acc[3] += red[0];
            if (rk != 1 && *s_hit && (int64_t)acc[4] < 0) {
                acc[4] = (uint64_t)p.rule.round;
                *(volatile int64_t *)p.rule.h_flag = p.rule.round;
                __threadfence_system();
            }
        }
    }
}

// Ascending list of the first cap violating record indices, in two
// launches independent of how the validation kernel split the records:
// k_emit_count counts the violations of each CTA's contiguous range of
// bitmap words (cnt[4c + 3]), k_validate_emit takes the exclusive prefix of
// those counts and writes its range's indices with a block scan.
__global__ void __launch_bounds__(512) k_emit_count(const uint32_t *bitmap, uint64_t nwords,
                                                   uint64_t *cnt) {
    __shared__ unsigned long long s_n;
    const uint64_t G = gridDim.x, c = blockIdx.x;
    const uint64_t w0 = nwords * c / G, w1 = nwords * (c + 1) / G;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    unsigned long long n = 0;
    for (uint64_t w = w0 + threadIdx.x; w < w1; w += blockDim.x) n += __popc(bitmap[w]);
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(&s_n, n);
    __syncthreads();
    if (threadIdx.x == 0) cnt[4 * c + 3] = s_n;
}

__global__ void __launch_bounds__(512) k_validate_emit(const uint32_t *bitmap, uint64_t n_rec,
                                                       const uint64_t *cnt, uint64_t *idx,
                                                       uint64_t cap) {
    __shared__ unsigned long long s_pre;
    __shared__ uint32_t s_warp[16];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t G = gridDim.x, c = blockIdx.x;
    if (cnt[4 * c + 3] == 0) return;
    if (tid == 0) s_pre = 0;
    __syncthreads();
    unsigned long long pre = 0;
    for (uint64_t q = tid; q < c; q += blockDim.x) pre += cnt[4 * q + 3];
    if (pre) atomicAdd(&s_pre, pre);
    __syncthreads();
    uint64_t prefix = s_pre;
    if (prefix >= cap) return;
    const uint64_t nwords = (n_rec + 31) / 32;
    const uint64_t w0 = nwords * c / G, w1 = nwords * (c + 1) / G;
    for (uint64_t wb = w0; wb < w1; wb += blockDim.x) {
        const uint64_t wi = wb + tid;
        uint32_t v = wi < w1 ? bitmap[wi] : 0u;
        uint32_t pc = __popc(v);
        // block exclusive scan of pc
        uint32_t incl = pc;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        uint32_t woff = 0, total = 0;
        for (uint32_t q = 0; q < (blockDim.x >> 5); ++q) {
            if (q < warp) woff += s_warp[q];
            total += s_warp[q];
        }
        uint64_t pos = prefix + woff + incl - pc;
        while (v && pos < cap) {
            const uint32_t b = __ffs(v) - 1;
            idx[pos++] = wi * 32 + b;
            v &= v - 1;
        }
        prefix += total;
        __syncthreads();
        if (prefix >= cap) break;
    }
}

// Enqueue the index list (both launches) on s.
static phos_status emit_index_list(const uint32_t *d_bitmap, uint64_t n_rec, uint64_t G,
                                   uint64_t *cnt, uint64_t *d_idx, uint64_t cap,
                                   cudaStream_t s) {
    const uint64_t nwords = (n_rec + 31) / 32;
    k_emit_count<<<(unsigned)G, 512, 0, s>>>(d_bitmap, nwords, cnt);
    count_launch();
    PHOS_CUDA(cudaGetLastError());
    k_validate_emit<<<(unsigned)G, 512, 0, s>>>(d_bitmap, n_rec, cnt, d_idx, cap);
    count_launch();
    PHOS_CUDA(cudaGetLastError());
    return PHOS_OK;
}

struct ValPlan {
    bool smem_table;
    uint32_t stages;
    size_t smem;
};

static ValPlan plan_validate(uint32_t n, int device) {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (optin <= 0) optin = 227 * 1024;
    const uint32_t nvw = (n + 31) / 32, nf1 = (n + 31) / 32, nf2 = (n + 1023) / 1024;
    const size_t fixed = 32 + ((n + 15) & ~15u) + 8ull * nvw;
    const size_t tab = 8ull * (2 * n + nf1 + nf2);
    const size_t ctl = 16ull * kMaxStages;   // mbarriers, used[], issued[]
    for (uint32_t S = kMaxStages; S >= 2; --S) {
        size_t need = (size_t)S * kTileBytes + ctl + fixed + tab;
        if (need <= (size_t)optin) return {true, S, need};
    }
    uint32_t S = 6;
    size_t need = (size_t)S * kTileBytes + ctl + fixed;
    return {false, S, need};
}

static size_t plan_batched(uint32_t n, int device, bool *smem_table) {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (optin <= 0) optin = 227 * 1024;
    const uint32_t nvw = (n + 31) / 32;
    const size_t fixed = sizeof(Lead) * 64 * (kValThreads / 32) + 32 + ((n + 15) & ~15u) +
                         8ull * nvw;
    const size_t tab = 16ull * n;
    *smem_table = fixed + tab <= (size_t)optin;
    return *smem_table ? fixed + tab : fixed;
}

static uint32_t g_val_variant = 0;  // 0 auto, 1 TMA ring, 2 batched leaders
static uint32_t g_val_wait_limit = kWaitLimit;
static uint32_t g_val_ctas = 0;     // 0 auto (one per SM), else the grid size

// CTAs of a batched launch: one per 8 batches up to the SM count.  A CTA's
// prologue (table and perms into shared memory) and its part in the
// last-CTA reduction cost the same whether it has one busy warp or 32, and
// short traces are latency-bound per warp: a 65,536-record trace (256
// batches) measured 8.7 us on 32 CTAs against 10.3 us on 148.
static uint64_t batched_grid(uint64_t units, uint64_t ctas) {
    return std::max<uint64_t>(1, std::min<uint64_t>(ctas, (units + 7) / 8));
}

// Words per warp batch, W in {32, 16, 8}: the one that minimises the
// busiest warp's work, words x (W + 6) / W -- each batch costs its leader
// searches on top of its words, which makes an 8-word batch ~1.45x and a
// 16-word batch ~1.15x as dear per record as a 32-word one (measured:
// 260M records took 0.60 ms with 8-word batches, 0.41 ms with 32).  Small
// traces still spread over every warp; large ones keep W = 32 even where a
// smaller W would shave a partial batch off the tail.
static uint32_t words_per_batch(uint64_t n_rec, uint64_t ctas) {
    const uint64_t warps = ctas * (kValThreads / 32);
    uint32_t best = 32;
    double best_cost = 1e300;
    for (uint32_t W = 32; W >= 8; W /= 2) {
        const uint64_t nb = (n_rec + 32ull * W - 1) / (32ull * W);
        const uint64_t words = (nb + warps - 1) / warps * W;
        const double cost = (double)words * (W + 6) / W;
        if (cost < best_cost) {
            best_cost = cost;
            best = W;
        }
    }
    return best;
}

}  // namespace phos

using namespace phos;

namespace {

// always_attr: set the shared-memory opt-in on every call (the allocation-
// free entry point keeps no host-side state either).
template <bool T, bool D>
phos_status launch_b(uint64_t G, size_t smem, cudaStream_t s, const ValParams &p, bool always_attr) {
    if (always_attr) {
        PHOS_CUDA(cudaFuncSetAttribute((const void *)k_validate_b<T, D>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    } else {
        phos_status r = smem_optin_once((const void *)k_validate_b<T, D>);
        if (r) return r;
    }
    k_validate_b<T, D><<<(unsigned)G, kValThreads, smem, s>>>(p);
    return PHOS_OK;
}

}  // namespace

// The batched kernel with the table in shared memory or not, and batches
// from the shared counter when the trace has more batches than the grid
// has warps (else grid-stride, with no atomics).
static phos_status launch_validate_b(bool smem_table, uint64_t G, size_t smem, cudaStream_t s,
                                     const ValParams &p, bool always_attr) {
    const uint64_t brec = 32ull * p.wpb;
    const bool dyn = G * (kValThreads / 32) < (p.n_rec + brec - 1) / brec;
    if (smem_table)
        return dyn ? launch_b<true, true>(G, smem, s, p, always_attr)
                   : launch_b<true, false>(G, smem, s, p, always_attr);
    return dyn ? launch_b<false, true>(G, smem, s, p, always_attr)
               : launch_b<false, false>(G, smem, s, p, always_attr);
}

extern "C" phos_status phos_validate_config(uint32_t variant) {
    if (variant > 2) return fail(PHOS_EINVAL, "validate_config: variant %u", variant);
    g_val_variant = variant;
    return PHOS_OK;
}

extern "C" phos_status phos_validate_wait_limit(uint32_t probes) {
    g_val_wait_limit = probes;
    return PHOS_OK;
}

extern "C" phos_status phos_validate_grid(uint32_t ctas) {
    if (ctas > 4096) return fail(PHOS_EINVAL, "validate_grid: %u CTAs", ctas);
    g_val_ctas = ctas;
    return PHOS_OK;
}

phos_status phos::validate_impl(const phos_table_t *t, const uint8_t *d_perm,
                                const uint64_t *d_trace, uint64_t n_rec, uint32_t access_bytes,
                                uint32_t *d_bitmap, uint64_t *d_count, uint32_t *d_victim,
                                uint32_t *d_victim_st, uint64_t *d_idx, uint64_t idx_cap,
                                uint32_t *d_status, phos_stream_t stream, const ProtoRule *rule,
                                bool *rule_fused) {
    if (rule_fused) *rule_fused = false;
    if (!t) return fail(PHOS_EINVAL, "validate: table is NULL");
    if (!d_count) return fail(PHOS_EINVAL, "validate: d_count is NULL");
    if (access_bytes == 0) return fail(PHOS_EINVAL, "validate: access_bytes is 0");
    if (n_rec && (!d_trace || !d_bitmap))
        return fail(PHOS_EINVAL, "validate: NULL trace or bitmap");
    if (n_rec && ((uintptr_t)d_trace & 15))
        return fail(PHOS_EINVAL, "validate: trace must be 16-byte aligned");
    if (t->n && !d_perm) return fail(PHOS_EINVAL, "validate: d_perm is NULL");
    if (idx_cap && !d_idx) return fail(PHOS_EINVAL, "validate: idx_cap > 0 with NULL d_idx");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    phos_table *T = const_cast<phos_table *>(t);
    const uint32_t variant = g_val_variant == 0 ? 2u : g_val_variant;
    const int sms = g_val_ctas ? (int)g_val_ctas : sm_count(T->device);
    const uint32_t wpb = words_per_batch(n_rec, (uint64_t)sms);
    const uint64_t unit = variant == 1 ? kTileRec : 32ull * wpb;
    const uint64_t units = (n_rec + unit - 1) / unit;
    const uint64_t G = variant == 1 ? std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sms, units))
                                    : batched_grid(units, (uint64_t)sms);
    const uint32_t nvw = (t->n + 31) / 32;
    const size_t off_vacc = 256, off_cnt = align_up(off_vacc + 8ull * std::max(nvw, 1u), 256);
    const size_t need = off_cnt + 32ull * (size_t)sms;
    {
        std::lock_guard<std::mutex> g(T->mu);
        phos_status r = T->val_scratch.reserve(need);
        if (r) return r;
    }
    uint8_t *sc = static_cast<uint8_t *>(T->val_scratch.ptr);
    ValParams p;
    p.tab = t->view;
    p.perm = d_perm;
    p.trace = d_trace;
    p.n_rec = n_rec;
    p.tiles = (n_rec + kTileRec - 1) / kTileRec;
    p.bitmap = d_bitmap;
    p.count = d_count;
    p.victim = d_victim;
    p.victim_st = d_victim_st;
    p.status = d_status;
    p.ticket = reinterpret_cast<uint32_t *>(sc);
    p.next = reinterpret_cast<unsigned long long *>(sc + 8);
    p.vacc = reinterpret_cast<uint32_t *>(sc + off_vacc);
    p.cta_cnt = reinterpret_cast<uint64_t *>(sc + off_cnt);
    p.w = access_bytes;
    p.nvw = nvw;
    p.stages = 0;
    p.wpb = wpb;
    p.wait_limit = g_val_wait_limit;
    if (rule && variant != 1 && n_rec) {
        p.rule = *rule;
        if (rule_fused) *rule_fused = true;
    }
    auto attr = [&](const void *fn, int) -> phos_status { return smem_optin_once(fn); };
    phos_status r;
    if (variant == 1) {
        ValPlan pl = plan_validate(t->n, T->device);
        p.stages = pl.stages;
        if (pl.smem_table) {
            if ((r = attr((const void *)k_validate<true>, 0))) return r;
            k_validate<true><<<(unsigned)G, kValThreads, pl.smem, s>>>(p);
        } else {
            if ((r = attr((const void *)k_validate<false>, 1))) return r;
            k_validate<false><<<(unsigned)G, kValThreads, pl.smem, s>>>(p);
        }
    } else {
        bool smem_table;
        const size_t smem = plan_batched(t->n, T->device, &smem_table);
        if ((r = launch_validate_b(smem_table, G, smem, s, p, false))) return r;
    }
    count_launch();
    PHOS_CUDA(cudaGetLastError());
    if (d_idx && idx_cap && n_rec) {
        phos_status re = emit_index_list(d_bitmap, n_rec, G, p.cta_cnt, d_idx, idx_cap, s);
        if (re) return re;
    }
    return PHOS_OK;
}

extern "C" phos_status phos_validate(const phos_table_t *t, const uint8_t *d_perm,
                                     const uint64_t *d_trace, uint64_t n_rec,
                                     uint32_t access_bytes, uint32_t *d_bitmap,
                                     uint64_t *d_count, uint32_t *d_victim,
                                     uint32_t *d_victim_st, uint64_t *d_idx, uint64_t idx_cap,
                                     uint32_t *d_status, phos_stream_t stream) {
    return validate_impl(t, d_perm, d_trace, n_rec, access_bytes, d_bitmap, d_count, d_victim,
                         d_victim_st, d_idx, idx_cap, d_status, stream, nullptr, nullptr);
}

// ----------------------------------------------------------------------
// phos_validate_noalloc: phos_validate without any device allocation.
//
// Some callers cannot call cudaMalloc when they validate: the interposer
// that runs inside an application's intercepted CUDA call (where entering
// the allocator again can deadlock on the application's allocator lock or
// recurse into the interception layer), and callers that must not let an
// allocation's implicit device synchronisation stall the application's
// in-flight kernels during a concurrent checkpoint.  This entry point
// keeps its scratch (per-CTA counts, victim accumulators, completion
// ticket) in a fixed array inside the library instead of the table
// handle's growable scratch.
// ----------------------------------------------------------------------
namespace phos {

constexpr uint32_t kNoallocMaxCtas = 256;
constexpr uint32_t kNoallocMaxBuffers = 16384;
constexpr size_t kNoallocOffVacc = 256;
constexpr size_t kNoallocOffCnt = kNoallocOffVacc + 8ull * ((kNoallocMaxBuffers + 31) / 32);
constexpr size_t kNoallocBytes = kNoallocOffCnt + 32ull * kNoallocMaxCtas;

// Every GPU that loads the library holds this array until the process
// exits.  All calls share it.
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoallocBytes];

static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[64];

// Zero the ticket and the victim accumulators this call will use.
__global__ void k_noalloc_clear(uint8_t *scratch, uint32_t nvw) {
    uint32_t *ticket = reinterpret_cast<uint32_t *>(scratch);
    uint32_t *vacc = reinterpret_cast<uint32_t *>(scratch + kNoallocOffVacc);
    if (threadIdx.x == 0) {
        *ticket = 0;
        *reinterpret_cast<unsigned long long *>(scratch + 8) = 0;  // batch counter
    }
    for (uint32_t i = threadIdx.x; i < 2 * nvw; i += blockDim.x) vacc[i] = 0;
}

// Device address of the array on `device`, which the caller has checked is
// the current device; looked up once per device.
static phos_status noalloc_scratch(int device, void **out) {
    if (device < 0 || device >= 64) return fail(PHOS_EINVAL, "validate_noalloc: device %d", device);
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "validate_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[device] = p;
    }
    *out = g_noalloc_ptr[device];
    return PHOS_OK;
}

}  // namespace phos

extern "C" phos_status phos_validate_noalloc(const phos_table_t *t, const uint8_t *d_perm,
                                             const uint64_t *d_trace, uint64_t n_rec,
                                             uint32_t access_bytes, uint32_t *d_bitmap,
                                             uint64_t *d_count, uint32_t *d_victim,
                                             uint32_t *d_victim_st, uint64_t *d_idx,
                                             uint64_t idx_cap, uint32_t *d_status,
                                             phos_stream_t stream) {
    if (!t) return fail(PHOS_EINVAL, "validate_noalloc: table is NULL");
    if (!d_count) return fail(PHOS_EINVAL, "validate_noalloc: d_count is NULL");
    if (access_bytes == 0) return fail(PHOS_EINVAL, "validate_noalloc: access_bytes is 0");
    if (n_rec && (!d_trace || !d_bitmap))
        return fail(PHOS_EINVAL, "validate_noalloc: NULL trace or bitmap");
    if (n_rec && ((uintptr_t)d_trace & 15))
        return fail(PHOS_EINVAL, "validate_noalloc: trace must be 16-byte aligned");
    if (t->n && !d_perm) return fail(PHOS_EINVAL, "validate_noalloc: d_perm is NULL");
    if (idx_cap && !d_idx) return fail(PHOS_EINVAL, "validate_noalloc: idx_cap > 0 with NULL d_idx");
    if (t->n > kNoallocMaxBuffers)
        return fail(PHOS_EINVAL,
                    "validate_noalloc: table of %u buffers exceeds the fixed scratch limit of %u "
                    "buffers; use phos_validate",
                    t->n, kNoallocMaxBuffers);
    // The kernels launch on the calling thread's current device, so that
    // must be the device the table (and the array's address) belongs to.
    int cur = -1;
    PHOS_CUDA(cudaGetDevice(&cur));
    if (cur != t->device)
        return fail(PHOS_EINVAL,
                    "validate_noalloc: the table belongs to device %d but device %d is current; "
                    "make device %d current before the call",
                    t->device, cur, t->device);
    void *scr = nullptr;
    phos_status r = noalloc_scratch(t->device, &scr);
    if (r) return r;
    uint8_t *sc = static_cast<uint8_t *>(scr);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t ctas =
        std::min<uint64_t>((uint64_t)sm_count(t->device), kNoallocMaxCtas);
    const uint32_t wpb = words_per_batch(n_rec, ctas);
    const uint64_t units = (n_rec + 32ull * wpb - 1) / (32ull * wpb);
    const uint64_t G = batched_grid(units, ctas);
    const uint32_t nvw = (t->n + 31) / 32;
    ValParams p;
    p.tab = t->view;
    p.perm = d_perm;
    p.trace = d_trace;
    p.n_rec = n_rec;
    p.tiles = (n_rec + kTileRec - 1) / kTileRec;
    p.bitmap = d_bitmap;
    p.count = d_count;
    p.victim = d_victim;
    p.victim_st = d_victim_st;
    p.status = d_status;
    p.ticket = reinterpret_cast<uint32_t *>(sc);
    p.next = reinterpret_cast<unsigned long long *>(sc + 8);
    p.vacc = reinterpret_cast<uint32_t *>(sc + kNoallocOffVacc);
    p.cta_cnt = reinterpret_cast<uint64_t *>(sc + kNoallocOffCnt);
    p.w = access_bytes;
    p.nvw = nvw;
    p.stages = 0;
    p.wpb = wpb;
    p.wait_limit = kWaitLimit;
    k_noalloc_clear<<<1, 256, 0, s>>>(sc, nvw);
    count_launch();
    PHOS_CUDA(cudaGetLastError());
    bool smem_table;
    const size_t smem = plan_batched(t->n, t->device, &smem_table);
    if ((r = launch_validate_b(smem_table, G, smem, s, p, true))) return r;
    count_launch();
    PHOS_CUDA(cudaGetLastError());
    if (d_idx && idx_cap && n_rec) {
        r = emit_index_list(d_bitmap, n_rec, G, p.cta_cnt, d_idx, idx_cap, s);
        if (r) return r;
    }
    return PHOS_OK;
}
