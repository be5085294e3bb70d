// Device-side lookup and word classification shared by the validation
// kernels and the batched plan (PhoenixOS Sec. 4.1 "Runtime validation").
#pragma once
#include <stdint.h>

#include "../../include/phos.h"

namespace phos {

// Table view used by the lookup.  lim[i] = number of valid start offsets
// of a w-byte access in buffer i (size - w + 1, or 0 if size < w), so that
// [a, a+w) lies in buffer i  <=>  a - base[i] < lim[i]  (unsigned; a below
// base wraps to a huge value).
struct Look {
    const uint64_t *base;
    const uint64_t *lim;     // shared-memory path
    const uint64_t *size;    // global path: lim computed on the fly
    const uint64_t *f1;
    const uint64_t *f2;
    const uint8_t *perm;
    uint32_t n, nf1, w;
    uint64_t rf;             // this lane's entry of the top search level

    __device__ __forceinline__ uint64_t limit(int i, bool smem_lim) const {
        if (smem_lim) return lim[i];
        const uint64_t s = size[i];
        return s >= w ? s - w + 1 : 0;
    }

    // Warp-uniform x: index of the last buffer with base <= x, or -1.
    // One ballot per level; the top level lives in registers.
    __device__ __forceinline__ int search(uint64_t x, uint32_t lane) const {
        const uint64_t kMax = ~0ull;
        uint32_t c = __popc(__ballot_sync(0xffffffffu, rf <= x));
        if (n <= 32) return (int)c - 1;
        if (c == 0) return -1;
        uint32_t blk = c - 1;
        if (n > 1024) {
            const uint32_t idx = blk * 32 + lane;
            const uint64_t v = idx < nf1 ? f1[idx] : kMax;
            blk = blk * 32 + __popc(__ballot_sync(0xffffffffu, v <= x)) - 1;
        }
        const uint32_t idx = blk * 32 + lane;
        const uint64_t v = idx < n ? base[idx] : kMax;
        return (int)(blk * 32 + __popc(__ballot_sync(0xffffffffu, v <= x)) - 1);
    }

    // Per-lane binary search (divergent fallback).
    __device__ __forceinline__ int lane_search(uint64_t a) const {
        uint32_t lo = 0, cnt = n;
        while (cnt > 0) {
            const uint32_t half = cnt >> 1;
            if (base[lo + half] <= a) {
                lo += half + 1;
                cnt -= half + 1;
            } else {
                cnt = half;
            }
        }
        return (int)lo - 1;
    }
};

struct Acc {
    uint64_t c0 = 0, c1 = 0, c2 = 0;
    bool bad = false;
};

// Batched-leader variant.  A warp takes W consecutive bitmap words (32 * W
// records, W = 32 for large traces, 16 or 8 for small ones so that every
// warp gets work) at a time.  Lane j loads the first record of word j and
// runs its own binary search for it, so the W searches of a batch run in
// parallel across the lanes; the interval found for word j (base, limit,
// permission) is parked in the warp's shared-memory slot.  Then, word by
// word, every lane checks its record against that interval with one
// unsigned compare (broadcast reads), lanes that miss run their own
// search, and the batch's W bitmap words leave in one coalesced store.
// batch_words takes one word per step (records four words ahead) and
// serves the trace's last, partial batch; full batches take two words per
// step (batch_pairs, or the validation kernel's cross-batch stream).
constexpr uint32_t kBatch = 1024;   // records of a full 32-word batch

// The leader of a word, folded with its permission into one test: a record
// rec (store bit 63, address bits 0..56, reserved bits 57..62) lies in the
// leader's buffer with an admitted access iff
//     ((rec - kb) & (km:0xffffffff)) < kl.
// With base b and limit l (valid start offsets of a w-byte access):
//   R and W  kb = b, km = 0x7fffffff: the store bit drops out of the
//            difference, so loads and stores in range pass
//   R only   kb = b, km = ~0: a store's difference is >= 2^63 > l
//   W only   kb = b | 2^63, km = ~0: a load's difference is >= 2^63
//   neither, or no leader: kl = 0
// An address below b wraps to >= 2^63 - 2^57 > l either way; reserved
// bits make the difference >= 2^57 > l (b + l <= 2^57 for any table).
struct __align__(16) Lead {
    uint64_t kb, kl;
    uint32_t km;
    int32_t i;         // leader's table index, -1 if none
    uint64_t pad;
};

__device__ __forceinline__ bool lead_ok(const Lead &ld, uint64_t rec) {
    const uint64_t m = ((uint64_t)ld.km << 32) | 0xffffffffull;
    return ((rec - ld.kb) & m) < ld.kl;
}

// Lead of table entry i (or of no entry, i < 0).
__device__ __forceinline__ Lead make_lead(const Look &L, int i, bool smem_lim) {
    Lead ld;
    ld.kb = 0;
    ld.kl = 0;
    ld.km = 0xffffffffu;
    ld.i = i;
    ld.pad = 0;
    if (i >= 0) {
        const uint64_t b = L.base[i];
        const uint32_t pm = L.perm[i] & 3u;
        ld.kb = pm == 2u ? (b | PHOS_REC_STORE) : b;
        ld.kl = pm ? L.limit(i, smem_lim) : 0;
        ld.km = pm == 3u ? 0x7fffffffu : 0xffffffffu;
    }
    return ld;
}

// Full classification of one record: the interval of its word's leader
// (table entry ld.i) when the address lies in it, else the lane's own
// search.  hit: the access lies inside some buffer; bi, pm: that buffer
// and its permission; bad: a reserved bit is set.
template <bool kSmemTable>
__device__ __forceinline__ void classify(const Look &L, uint64_t rec, const Lead &ld, bool &hit,
                                         int &bi, uint32_t &pm, bool &bad) {
    const uint64_t a = rec & ~PHOS_REC_STORE;
    hit = false;
    bi = -1;
    pm = 0;
    bad = false;
    if (ld.i >= 0 && (a - L.base[ld.i]) < L.limit(ld.i, kSmemTable)) {
        hit = true;
        bi = ld.i;
        pm = L.perm[ld.i];
        return;
    }
    bad = a > PHOS_REC_ADDR_MASK;
    if (!bad) {
        const int ii = L.lane_search(a);
        if (ii >= 0 && (a - L.base[ii]) < L.limit(ii, kSmemTable)) {
            hit = true;
            bi = ii;
            pm = L.perm[ii];
        }
    }
}

// Classify one record against its word's leader interval.  The store bit
// is cleared but the reserved bits are kept, so a malformed record lies
// above the 57-bit space and can never fall inside an interval: it misses
// and is sorted out on the (rare) fallback path.
template <bool kSmemTable, bool kFull>
__device__ __forceinline__ void one_word(const Look &L, uint64_t rec, bool valid, uint32_t j,
                                         uint32_t lane, const Lead &ld, uint32_t &myvw,
                                         uint32_t *sv, uint32_t *svs, Acc &acc) {
    if (kFull) valid = true;
    const uint32_t st = (uint32_t)(rec >> 63);
    bool viol = false, hit = true, bad = false;
    const bool slow = valid && !lead_ok(ld, rec);
    if (__ballot_sync(0xffffffffu, slow)) {
        if (slow) {
            int bi;
            uint32_t pm;
            classify<kSmemTable>(L, rec, ld, hit, bi, pm, bad);
            viol = !(hit && ((pm >> st) & 1u));
            if (viol && hit) {
                atomicOr(&sv[bi >> 5], 1u << (bi & 31));
                if (st) atomicOr(&svs[bi >> 5], 1u << (bi & 31));
            }
        }
    }
    const uint32_t vw = __ballot_sync(0xffffffffu, viol);
    myvw = (lane == j) ? vw : myvw;
    if (vw) {
        const uint32_t sw = __ballot_sync(0xffffffffu, viol && st);
        const uint32_t uw = __ballot_sync(0xffffffffu, viol && !hit);
        if (lane == 0) {
            acc.c0 += __popc(vw);
            acc.c1 += __popc(sw);
            acc.c2 += __popc(uw);
        }
        acc.bad |= bad;
    }
}

// The W words (W = 8, 16 or 32) of one batch, records loaded four words
// ahead of use.  kFull: the batch holds 32 * W records.
template <bool kSmemTable, bool kFull>
__device__ __forceinline__ void batch_words(const Look &L, const uint64_t *recs, uint64_t nb,
                                            uint32_t W, uint32_t lane, const Lead *lead,
                                            uint32_t *bm, uint32_t *sv, uint32_t *svs,
                                            Acc &acc) {
    uint32_t myvw = 0;
    uint64_t r[4], n[4];
#pragma unroll
    for (uint32_t u = 0; u < 4; ++u) {
        const uint32_t k = u * 32 + lane;
        r[u] = (kFull || k < nb) ? recs[k] : 0ull;
    }
#pragma unroll 1
    for (uint32_t j0 = 0; j0 < W; j0 += 4) {
        if (j0 + 4 < W) {
#pragma unroll
            for (uint32_t u = 0; u < 4; ++u) {
                const uint32_t k = (j0 + 4 + u) * 32 + lane;
                n[u] = (kFull || k < nb) ? recs[k] : 0ull;
            }
        }
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u) {
            const uint32_t j = j0 + u;
            one_word<kSmemTable, kFull>(L, r[u], kFull || (j * 32 + lane) < nb, j, lane, lead[j],
                                        myvw, sv, svs, acc);
        }
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u) r[u] = n[u];
    }
    if (lane < W && (kFull || lane * 32 < nb)) bm[lane] = myvw;
}

// Bits 0..15 of x to the even bit positions 0, 2, .., 30.
__device__ __forceinline__ uint32_t spread16(uint32_t x) {
    x &= 0xFFFFu;
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

// General path of one record of a pair (a lane's element e); victims are
// marked here.
template <bool kSmemTable>
__device__ __forceinline__ bool pair_record(const Look &L, uint64_t rec, const Lead &ld,
                                            uint32_t *sv, uint32_t *svs, bool &hit,
                                            bool &bad) {
    const uint32_t st = (uint32_t)(rec >> 63);
    int bi;
    uint32_t pm;
    classify<kSmemTable>(L, rec, ld, hit, bi, pm, bad);
    const bool viol = !(hit && ((pm >> st) & 1u));
    if (viol && hit) {
        atomicOr(&sv[bi >> 5], 1u << (bi & 31));
        if (st) atomicOr(&svs[bi >> 5], 1u << (bi & 31));
    }
    return viol;
}

// One pair of a full batch (see batch_pairs): x = this lane's two records,
// ld = the leader of its word, q = the pair's index in the batch.
template <bool kSmemTable>
__device__ __forceinline__ void pair_step(const Look &L, ulonglong2 x, const Lead &ld,
                                          uint32_t q, uint32_t lane, uint32_t *sv,
                                          uint32_t *svs, Acc &acc, uint32_t &myvw) {
    const uint64_t x0 = x.x, x1 = x.y;
    const bool ok0 = lead_ok(ld, x0), ok1 = lead_ok(ld, x1);
    if (__ballot_sync(0xffffffffu, !(ok0 && ok1))) {
        bool h0, h1, bad0, bad1;
        const bool v0 = pair_record<kSmemTable>(L, x0, ld, sv, svs, h0, bad0);
        const bool v1 = pair_record<kSmemTable>(L, x1, ld, sv, svs, h1, bad1);
        const uint32_t b0 = __ballot_sync(0xffffffffu, v0);
        const uint32_t b1 = __ballot_sync(0xffffffffu, v1);
        const uint32_t s0 = __ballot_sync(0xffffffffu, v0 && (x0 >> 63));
        const uint32_t s1 = __ballot_sync(0xffffffffu, v1 && (x1 >> 63));
        const uint32_t u0 = __ballot_sync(0xffffffffu, !h0);
        const uint32_t u1 = __ballot_sync(0xffffffffu, !h1);
        if (lane == 0) {
            acc.c0 += __popc(b0) + __popc(b1);
            acc.c1 += __popc(s0) + __popc(s1);
            acc.c2 += __popc(u0) + __popc(u1);
        }
        acc.bad |= bad0 || bad1;
        const uint32_t lo = spread16(b0) | (spread16(b1) << 1);
        const uint32_t hi = spread16(b0 >> 16) | (spread16(b1 >> 16) << 1);
        myvw = lane == 2 * q ? lo : (lane == 2 * q + 1 ? hi : myvw);
    }
}

// A full batch two bitmap words at a time: lane l loads records 2l and
// 2l+1 of the pair with one 16-byte load, so lanes 0-15 cover the first
// word and lanes 16-31 the second.  When every record of the pair lies in
// its word's leader interval and the leader's permission admits it (the
// common case), the pair costs one ballot; otherwise the general path
// classifies each record, and the two words' bits are put back in record
// order (record k of a word is element k & 1 of lane k >> 1).  Pairs are
// loaded three ahead.  recs: 16-byte aligned, 32 * W records, W even.
template <bool kSmemTable>
__device__ __forceinline__ void batch_pairs(const Look &L, const uint64_t *recs, uint32_t W,
                                            uint32_t lane, const Lead *lead, uint32_t *bm,
                                            uint32_t *sv, uint32_t *svs, Acc &acc) {
    uint32_t myvw = 0;
    const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(recs) + lane;
    const uint32_t npair = W >> 1;
    // ring of four pairs: pair q sits in slot q % 4, pair q + 3 is loaded
    // into the slot pair q - 1 left
    ulonglong2 r[4];
#pragma unroll
    for (uint32_t u = 0; u < 3; ++u) r[u] = u < npair ? p[u * 32] : make_ulonglong2(0, 0);
    const uint32_t half = lane >> 4;
#pragma unroll 1
    for (uint32_t q0 = 0; q0 < npair; q0 += 4) {
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u) {
            const uint32_t q = q0 + u;
            if (q >= npair) break;
            r[(u + 3) & 3] = q + 3 < npair ? p[(q + 3) * 32] : make_ulonglong2(0, 0);
            pair_step<kSmemTable>(L, r[u], lead[2 * q + half], q, lane, sv, svs, acc, myvw);
        }
    }
    if (lane < W) bm[lane] = myvw;
}

}  // namespace phos
