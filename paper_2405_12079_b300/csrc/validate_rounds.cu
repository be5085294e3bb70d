// Validation of several protocol rounds in one launch (PhoenixOS Sec. 4.1
// "Runtime validation", with the protocols' responses of Sec. 4.2, 4.3 and
// 6).  A no-sync session whose after_kernel defers validation hands the
// traces of up to kMaxRounds kernel rounds to one launch; every round is
// checked against its own speculated permissions and answered with its own
// rule flags (the state of the protocol when that round ran), exactly as a
// launch per round would, so only the moment the host can learn of a
// mis-speculation moves.
//
// B300 design
//   * Short traces (a kernel round's trace is ~10^4-10^6 records) are
//     latency-bound per warp, so the work unit is the validation kernels'
//     8-word batch (256 records): lane j searches the first record of word
//     j, then the records are checked word by word against those leaders
//     (batch_words).  Batches never straddle two rounds; they are taken
//     grid-stride, CTA-minor, over the rounds' concatenated batch ranges.
//   * Rounds with long traces (the training step's 1.3M records per kernel)
//     take 32-word batches (1,024 records) instead: an 8-word batch pays its
//     leader searches on a quarter of the records, ~1.45x the cost per
//     record.  The host picks the width with the plain validation's cost
//     model, words x (W + 6) / W for the busiest warp.  16 rounds of 1.3M
//     records: 74.5-78.8 -> 60.8-64.2 us per launch (ncu durations).  What
//     the streaming kernel adds on top measured no faster here (CUDA events,
//     against 61.4-63.5 us): an L2 prefetch of each warp's next batch raised
//     DRAM reads to 1.29x the records' bytes (67.6 us), loading the next
//     batch's leader records ahead cost 67.6 us, one record stream across the
//     warp's batches 63.5 us, and batches from a shared counter instead of
//     grid-stride 62.8 us.
//   * Every round's permissions and victim bitmaps sit in shared memory
//     next to the table, so a batch only switches pointers.
//   * One last-CTA epilogue per launch applies each round's rule: recopy
//     marks store victims that the copier had touched dirty; CoW and
//     restore record the first round (in round order) with a victim its
//     flags do not cover.  Results need no per-round bitmap or count, so
//     none is written.
#include <stdio.h>

#include <algorithm>

#include "internal.h"
#include "validate_dev.cuh"

namespace phos {

constexpr uint32_t kRoundThreads = 512;
constexpr uint32_t kRoundWShort = 8;   // words per batch: short rounds
constexpr uint32_t kRoundWLong = 32;   // long rounds

struct RoundsParams {
    TableDev tab;
    uint32_t w;                     // access width
    uint32_t nvw;                   // victim words per round
    uint32_t k;                     // rounds in this launch
    uint32_t rule;                  // 1 recopy, 2 CoW, 3 restore (see ProtoRule)
    uint32_t W;                     // words per batch: kRoundWShort or kRoundWLong
    const uint64_t *trace[kMaxRounds];
    const uint8_t *perm[kMaxRounds];
    const uint8_t *flags[kMaxRounds];
    int64_t round[kMaxRounds];
    uint64_t n_rec[kMaxRounds];
    uint64_t bstart[kMaxRounds + 1];  // first batch of each round; [k] = all batches
    uint8_t *dirty;
    uint64_t *acc;
    int64_t *h_flag;
    uint32_t *status;
    uint32_t *vacc;                 // [k][2][nvw], zero between calls
    unsigned long long *cnt;        // violations, zero between calls
    uint32_t *ticket;               // zero between calls
};

static size_t rounds_fixed_smem(uint32_t W) {
    const uint32_t nw = kRoundThreads / 32;
    return sizeof(Lead) * W * nw + 4ull * W * nw + 128;
}

// Each round's permissions sit at a 16-byte aligned stride in shared memory.
static size_t rounds_smem(uint32_t n, uint32_t k, bool table, uint32_t W) {
    const uint32_t nvw = std::max((n + 31) / 32, 1u);
    return rounds_fixed_smem(W) + (table ? 16ull * n : 0) + (uint64_t)k * align_up(n, 16) +
           8ull * k * nvw;
}

template <bool kSmemTable>
__global__ void __launch_bounds__(kRoundThreads, 2)
    k_validate_rounds(const __grid_constant__ RoundsParams p) {
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t nwarps = blockDim.x >> 5;
    const uint32_t n = p.tab.n, nvw = p.nvw, K = p.k, W = p.W;
    const uint64_t brec = 32ull * W;                               // records per batch
    Lead *leads = reinterpret_cast<Lead *>(smem);                  // [nwarps][W]
    uint8_t *cur = smem + sizeof(Lead) * W * nwarps;
    uint32_t *words = reinterpret_cast<uint32_t *>(cur);           // [nwarps][W], unread
    cur += 4ull * W * nwarps;
    unsigned long long *red = reinterpret_cast<unsigned long long *>(cur);
    volatile uint32_t *fw = reinterpret_cast<volatile uint32_t *>(cur + 8);  // last, hit[K]
    cur += 128;
    Look L;
    L.n = n;
    L.nf1 = (n + 31) >> 5;
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
        for (uint32_t i = tid; i < n; i += blockDim.x) {
            tb[i] = __ldg(p.tab.base + i);
            const uint64_t sz = __ldg(p.tab.size + i);
            tl[i] = sz >= p.w ? sz - p.w + 1 : 0;
        }
        L.base = tb;
        L.lim = tl;
        cur += 16ull * n;
    }
    const uint32_t np = (n + 15) & ~15u;                         // per-round stride
    uint8_t *perms = cur;                                          // [K][np]
    cur += (uint64_t)K * np;
    uint32_t *sv = reinterpret_cast<uint32_t *>(cur);              // [K][2][nvw]
    for (uint32_t s = 0; s < K; ++s) {
        // 16-byte copies where the round's slot allows (upload slots are
        // 256-byte aligned), bytes for the rest
        const uint8_t *src = p.perm[s];
        uint8_t *dst = perms + (size_t)s * np;
        uint32_t done = 0;
        if (((uintptr_t)src & 15) == 0) {
            const uint32_t nv = n / 16;
            for (uint32_t i = tid; i < nv; i += blockDim.x)
                reinterpret_cast<uint4 *>(dst)[i] = reinterpret_cast<const uint4 *>(src)[i];
            done = nv * 16;
        }
        for (uint32_t i = done + tid; i < n; i += blockDim.x) dst[i] = src[i];
    }
    for (uint32_t i = tid; i < 2 * K * nvw; i += blockDim.x) sv[i] = 0;
    if (tid == 0) red[0] = 0;
    if (tid <= kMaxRounds) fw[tid] = 0;
    __syncthreads();

    const uint64_t G = gridDim.x, c = blockIdx.x, TW = G * nwarps;
    const uint64_t total = p.bstart[K];
    Lead *mine = leads + W * warp;
    Acc acc;
    // a warp's batches ascend, so the round index only moves forward
    uint32_t s = 0;
    for (uint64_t b = (uint64_t)warp * G + c; b < total; b += TW) {
        while (s + 1 < K && p.bstart[s + 1] <= b) ++s;
        const uint64_t r0 = (b - p.bstart[s]) * brec;
        const uint64_t nb = min(brec, p.n_rec[s] - r0);
        const uint64_t *recs = p.trace[s] + r0;
        L.perm = perms + (size_t)s * np;
        uint32_t *svr = sv + (size_t)s * 2 * nvw;
        if (lane < W)
            mine[lane] = make_lead(
                L, lane * 32 < nb ? L.lane_search(recs[lane * 32] & PHOS_REC_ADDR_MASK) : -1,
                kSmemTable);
        __syncwarp();
        // a full batch two words per step (one 16-byte load per lane:
        // traces are 16-byte aligned and batches start at 256-record
        // boundaries), a partial one word by word
        if (nb == brec)
            batch_pairs<kSmemTable>(L, recs, W, lane, mine, words + W * warp, svr, svr + nvw,
                                    acc);
        else
            batch_words<kSmemTable, false>(L, recs, nb, W, lane, mine, words + W * warp, svr,
                                           svr + nvw, acc);
        __syncwarp();
    }
    if (__any_sync(0xffffffffu, acc.bad) && lane == 0) set_status(p.status, PHOS_EINVAL);
    if (lane == 0 && acc.c0) atomicAdd(red, (unsigned long long)acc.c0);
    __syncthreads();
    if (tid == 0 && red[0]) atomicAdd(p.cnt, red[0]);
    for (uint32_t i = tid; i < 2 * K * nvw; i += blockDim.x)
        if (sv[i]) atomicOr(p.vacc + i, sv[i]);
    // ordered before the ticket by the barrier and one fence (grid-barrier
    // pattern); the last CTA's thread fences again before the reads
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        fw[0] = (atomicAdd(p.ticket, 1u) == (uint32_t)(G - 1)) ? 1u : 0u;
        if (fw[0]) __threadfence();
    }
    __syncthreads();
    if (!fw[0]) return;
    // the last CTA: each round's rule against that round's flags
    for (uint32_t i = tid; i < K * nvw; i += blockDim.x) {
        const uint32_t s = i / nvw, wd = i - s * nvw;
        uint32_t *va = p.vacc + (size_t)s * 2 * nvw;
        const uint32_t v = __ldcg(va + wd), vs = __ldcg(va + nvw + wd);
        va[wd] = 0;
        va[nvw + wd] = 0;
        uint32_t m = p.rule == 3 ? v : vs;
        const uint8_t *fl = p.flags[s];
        while (m) {
            const uint32_t bi = wd * 32 + (uint32_t)(__ffs(m) - 1);
            m &= m - 1;
            if (bi >= n) break;
            if (p.rule == 1) {
                if (fl[bi]) p.dirty[bi] = 1;
            } else if (!fl[bi]) {
                fw[1 + s] = 1;
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        p.acc[3] += __ldcg(p.cnt);
        *p.cnt = 0;
        *p.ticket = 0;
        if (p.rule != 1 && (int64_t)p.acc[4] < 0) {
            for (uint32_t s = 0; s < K; ++s) {
                if (fw[1 + s]) {
                    p.acc[4] = (uint64_t)p.round[s];
                    *(volatile int64_t *)p.h_flag = p.round[s];
                    __threadfence_system();
                    break;
                }
            }
        }
    }
}

// CTAs of a launch over b batches: one warp per batch, two CTAs per SM at
// most.
static uint64_t rounds_grid(uint64_t b, uint64_t max_ctas) {
    const uint64_t warps_per_cta = kRoundThreads / 32;
    return std::max<uint64_t>(1,
                              std::min<uint64_t>(max_ctas, (b + warps_per_cta - 1) / warps_per_cta));
}

// Batch width of a launch: the one whose busiest warp has the least work,
// counting each batch's leader searches as six words on top of its W words
// (the plain validation's cost model).  Ties keep the short batches.
static uint32_t rounds_width(const RoundSeg *seg, uint32_t k, uint64_t max_ctas) {
    uint32_t best = kRoundWShort;
    uint64_t best_cost = ~0ull;
    for (uint32_t W : {kRoundWShort, kRoundWLong}) {
        const uint64_t brec = 32ull * W;
        uint64_t b = 0;
        for (uint32_t i = 0; i < k; ++i) b += (seg[i].n_rec + brec - 1) / brec;
        const uint64_t warps = rounds_grid(b, max_ctas) * (kRoundThreads / 32);
        const uint64_t cost = (b + warps - 1) / warps * (W + 6);
        if (cost < best_cost) {
            best_cost = cost;
            best = W;
        }
    }
    return best;
}

uint32_t rounds_cap(uint32_t n, int device) {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (optin <= 0) optin = 227 * 1024;
    for (uint32_t k = kMaxRounds; k >= 2; --k)
        if (rounds_smem(n, k, false, kRoundWShort) <= (size_t)optin) return k;
    return 0;
}

size_t rounds_scratch_bytes(uint32_t n, uint32_t k) {
    const uint32_t nvw = std::max((n + 31) / 32, 1u);
    return 256 + 8ull * k * nvw;
}

phos_status validate_rounds(const phos_table_t *t, const RoundSeg *seg, uint32_t k,
                            uint32_t access_bytes, uint32_t rule, uint8_t *d_dirty,
                            uint64_t *d_acc, int64_t *d_flag, uint32_t *d_status,
                            void *d_scratch, cudaStream_t s) {
    if (k == 0) return PHOS_OK;
    if (k > kMaxRounds) return fail(PHOS_EINVAL, "validate_rounds: %u rounds", k);
    RoundsParams p;
    p.tab = t->view;
    p.w = access_bytes;
    p.nvw = std::max((t->n + 31) / 32, 1u);
    p.k = k;
    p.rule = rule;
    int optin = 0;
    PHOS_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, t->device));
    if (optin <= 0) optin = 227 * 1024;
    const uint64_t max_ctas = 2ull * sm_count(t->device);
    const uint32_t W = rounds_width(seg, k, max_ctas);
    // the wider batches' leader slots must fit next to the rounds' state
    p.W = rounds_smem(t->n, k, false, W) <= (size_t)optin ? W : kRoundWShort;
    const uint64_t brec = 32ull * p.W;
    uint64_t b = 0;
    for (uint32_t i = 0; i < k; ++i) {
        p.trace[i] = seg[i].trace;
        p.perm[i] = seg[i].perm;
        p.flags[i] = seg[i].flags;
        p.round[i] = seg[i].round;
        p.n_rec[i] = seg[i].n_rec;
        p.bstart[i] = b;
        b += (seg[i].n_rec + brec - 1) / brec;
    }
    for (uint32_t i = k; i < kMaxRounds; ++i) {
        p.trace[i] = nullptr;
        p.perm[i] = nullptr;
        p.flags[i] = nullptr;
        p.round[i] = 0;
        p.n_rec[i] = 0;
        p.bstart[i] = b;
    }
    p.bstart[kMaxRounds] = b;
    p.bstart[k] = b;
    p.dirty = d_dirty;
    p.acc = d_acc;
    p.h_flag = d_flag;
    p.status = d_status;
    uint8_t *sc = static_cast<uint8_t *>(d_scratch);
    p.cnt = reinterpret_cast<unsigned long long *>(sc);
    p.ticket = reinterpret_cast<uint32_t *>(sc + 8);
    p.vacc = reinterpret_cast<uint32_t *>(sc + 256);
    const bool table = rounds_smem(t->n, k, true, p.W) <= (size_t)optin;
    const size_t smem = rounds_smem(t->n, k, table, p.W);
    const uint64_t G = rounds_grid(b, max_ctas);
    if (table) {
        phos_status r = smem_optin_once((const void *)k_validate_rounds<true>);
        if (r) return r;
        k_validate_rounds<true><<<(unsigned)G, kRoundThreads, smem, s>>>(p);
    } else {
        phos_status r = smem_optin_once((const void *)k_validate_rounds<false>);
        if (r) return r;
        k_validate_rounds<false><<<(unsigned)G, kRoundThreads, smem, s>>>(p);
    }
    count_launch();
    PHOS_CUDA(cudaGetLastError());
    return PHOS_OK;
}

}  // namespace phos
