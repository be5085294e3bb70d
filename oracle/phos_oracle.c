/*
 * Plain CPU oracle for the PhOS data plane -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the slow, obviously correct definition that the CUDA path is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or
 * constant generator with the CUDA library; every function below is written
 * from the paper's statement of the method (PhoenixOS, SOSP'25,
 * arXiv 2405.12079) or from the published definition it names.
 *
 * Conventions (fixed readings of the paper, shared by both sides only as
 * prose, never as code):
 *   - buffer table: n buffers, base[i] ascending, size[i] > 0, disjoint,
 *     half-open [base, base + size)                       (Section 4.1)
 *   - perm byte per buffer: bit 0 = may read, bit 1 = may write;
 *     R = 1, RW = 3                                       (Sections 4.1, 6)
 *   - trace record: bit 63 = store, bits 57..62 reserved (must be 0),
 *     bits 0..56 = address; every access is w bytes wide   (Section 4.1)
 *
 * Build: gcc -O2 -shared -fPIC -o liboracle.so phos_oracle.c
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>

#define ORC_ADDR_MASK ((1ull << 57) - 1ull)
#define ORC_RSVD_MASK (0x3Full << 57)
#define ORC_GOLDEN 0x9E3779B97F4A7C15ull

/* ---------------------------------------------------------------------
 * SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014; finaliser constants as in Vigna's public
 * splitmix64.c).  orc_mix64 is the output function; orc_sm(x) is the value
 * produced by a generator whose state was x before one step.
 * ------------------------------------------------------------------- */
uint64_t orc_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t orc_sm(uint64_t x) { return orc_mix64(x + ORC_GOLDEN); }

/* ---------------------------------------------------------------------
 * Buffer table check (Section 4.1: the OS knows every buffer the process
 * allocated; each buffer is one contiguous virtual range).
 * Returns 0 if sorted, disjoint, non-empty and inside the 57-bit space.
 * ------------------------------------------------------------------- */
int orc_table_check(const uint64_t *base, const uint64_t *size, uint32_t n) {
    for (uint32_t i = 0; i < n; i++) {
        if (size[i] == 0) return 1;
        if (base[i] > ORC_ADDR_MASK || size[i] > ORC_ADDR_MASK + 1 - base[i]) return 2;
        if (i > 0 && base[i - 1] + size[i - 1] > base[i]) return 3;
    }
    return 0;
}

/* ---------------------------------------------------------------------
 * Argument-based speculation (Section 4.1 "Tracing with speculation on GPU
 * API arguments"; read-set extension in Section 6).
 *
 * Every argument value v that falls inside a buffer, base <= v < base+size,
 * marks the whole buffer.  kind: 0 scalar (ignored), 1 const pointer (read),
 * 2 mutable pointer (write, which also reads), 3 opaque struct: every
 * 8-byte little-endian chunk at offsets 0, 8, ... is treated as a possible
 * mutable pointer; a trailing partial chunk is ignored.
 * args[j] points at the argument's bytes, arg_size[j] is its byte size.
 * perm_out[n] is OR-accumulated (caller zeroes it).  Linear scan.
 * ------------------------------------------------------------------- */
static void orc_mark(const uint64_t *base, const uint64_t *size, uint32_t n,
                     uint64_t v, uint8_t p, uint8_t *perm) {
    for (uint32_t i = 0; i < n; i++)
        if (base[i] <= v && v - base[i] < size[i]) perm[i] |= p;
}

void orc_speculate(const uint64_t *base, const uint64_t *size, uint32_t n,
                   const void *const *args, const uint32_t *arg_size,
                   const uint8_t *kind, uint32_t nargs, uint8_t *perm_out) {
    for (uint32_t j = 0; j < nargs; j++) {
        const uint8_t *b = (const uint8_t *)args[j];
        if (kind[j] == 1 || kind[j] == 2) {
            uint64_t v = 0;
            uint32_t m = arg_size[j] < 8 ? arg_size[j] : 8;
            for (uint32_t t = 0; t < m; t++) v |= (uint64_t)b[t] << (8 * t);
            orc_mark(base, size, n, v, kind[j] == 1 ? 1 : 3, perm_out);
        } else if (kind[j] == 3) {
            for (uint32_t off = 0; off + 8 <= arg_size[j]; off += 8) {
                uint64_t v = 0;
                for (uint32_t t = 0; t < 8; t++) v |= (uint64_t)b[off + t] << (8 * t);
                orc_mark(base, size, n, v, 3, perm_out);
            }
        }
    }
}

/* Type-1 API rule (Section 4.1, memory moves): a copy that writes
 * [addr, addr+len) marks every buffer that range overlaps with perm p. */
void orc_speculate_region(const uint64_t *base, const uint64_t *size, uint32_t n,
                          uint64_t addr, uint64_t len, uint8_t p, uint8_t *perm_out) {
    if (len == 0) return;
    for (uint32_t i = 0; i < n; i++)
        if (base[i] < addr + len && addr < base[i] + size[i]) perm_out[i] |= p;
}

/* ---------------------------------------------------------------------
 * Runtime validation (Section 4.1 "Runtime validation"; reads too in
 * Section 6 "Handling mis-speculation").
 *
 * For record r: a = address, s = store bit.  Look for a buffer i with
 * base_i <= a and a + w <= base_i + size_i (linear scan).
 *   none                      -> violation, unmapped (count[2])
 *   perm_i lacks R (load)     -> violation, victim i
 *   perm_i lacks W (store)    -> violation, victim i
 * A store violation also counts in count[1].  A record with a reserved bit
 * set is malformed: counted as an unmapped violation and reported by the
 * return value (1).  bitmap bit r (word r>>5, bit r&31) is set for every
 * violation; idx receives the first idx_cap violating r in ascending order.
 * victim marks every buffer named by a violating access, victim_st only
 * those named by a violating store (the ones that matter for Sections 4.2
 * and 4.3).  Outputs are overwritten.  victim / victim_st / idx may be NULL.
 * ------------------------------------------------------------------- */
int orc_validate(const uint64_t *base, const uint64_t *size, const uint8_t *perm,
                 uint32_t n, const uint64_t *trace, uint64_t nrec, uint32_t w,
                 uint32_t *bitmap, uint64_t *count, uint32_t *victim,
                 uint32_t *victim_st, uint64_t *idx, uint64_t idx_cap) {
    int malformed = 0;
    uint64_t nwords = (nrec + 31) / 32;
    memset(bitmap, 0, nwords * sizeof(uint32_t));
    count[0] = count[1] = count[2] = 0;
    if (victim) memset(victim, 0, ((n + 31) / 32) * sizeof(uint32_t));
    if (victim_st) memset(victim_st, 0, ((n + 31) / 32) * sizeof(uint32_t));
    uint64_t nidx = 0;
    for (uint64_t r = 0; r < nrec; r++) {
        uint64_t rec = trace[r];
        uint64_t a = rec & ORC_ADDR_MASK;
        int store = (int)(rec >> 63);
        int viol = 0, unmapped = 0;
        long hit = -1;
        if (rec & ORC_RSVD_MASK) {
            malformed = 1;
            viol = 1; unmapped = 1;
        } else {
            for (uint32_t i = 0; i < n; i++)
                if (base[i] <= a && a + w <= base[i] + size[i]) { hit = (long)i; break; }
            if (hit < 0) { viol = 1; unmapped = 1; }
            else if (!(perm[hit] & (store ? 2 : 1))) {
                viol = 1;
                if (victim) victim[hit >> 5] |= 1u << (hit & 31);
                if (victim_st && store) victim_st[hit >> 5] |= 1u << (hit & 31);
            }
        }
        if (viol) {
            bitmap[r >> 5] |= 1u << (r & 31);
            count[0]++;
            if (store) count[1]++;
            if (unmapped) count[2]++;
            if (idx && nidx < idx_cap) idx[nidx++] = r;
        }
    }
    return malformed;
}

/* ---------------------------------------------------------------------
 * Order-independent 64-bit buffer digest (harness, not in the paper):
 * D = sum_j mix64(word_j + j * GOLDEN) mod 2^64, word_j the little-endian
 * 8-byte word at byte 8j, the last word zero-padded.
 * ------------------------------------------------------------------- */
uint64_t orc_digest(const uint8_t *p, uint64_t len) {
    uint64_t acc = 0;
    for (uint64_t j = 0; 8 * j < len; j++) {
        uint64_t wv = 0;
        for (uint64_t t = 0; t < 8 && 8 * j + t < len; t++)
            wv |= (uint64_t)p[8 * j + t] << (8 * t);
        acc += orc_mix64(wv + j * ORC_GOLDEN);
    }
    return acc;
}

/* The digest's partial sum over a piece of a buffer whose first byte is
 * the first byte of the buffer's word j0 (so a buffer's digest is the
 * mod-2^64 sum of its pieces' partial sums when every piece but the last
 * is a whole number of words). */
uint64_t orc_digest_at(const uint8_t *p, uint64_t len, uint64_t j0) {
    uint64_t acc = 0;
    for (uint64_t j = 0; 8 * j < len; j++) {
        uint64_t wv = 0;
        for (uint64_t t = 0; t < 8 && 8 * j + t < len; t++)
            wv |= (uint64_t)p[8 * j + t] << (8 * t);
        acc += orc_mix64(wv + (j0 + j) * ORC_GOLDEN);
    }
    return acc;
}

/* ---------------------------------------------------------------------
 * Word stream of the harness fill (not in the paper): the byte stream
 * whose 8-byte little-endian word j is sm(key ^ j).  orc_words writes its
 * bytes [byte_off, byte_off + len) to out.  The mutator's fill of buffer
 * w is this stream with key = sm(s_k ^ sm(w)) from byte 0; the initial
 * fill of a memory arena is this stream with the arena's key.
 * ------------------------------------------------------------------- */
void orc_words(uint8_t *out, uint64_t len, uint64_t key, uint64_t byte_off) {
    uint64_t q = 0;
    while (q < len) {
        uint64_t b = byte_off + q;
        uint64_t v = orc_sm(key ^ (b >> 3));
        for (uint64_t t = b & 7; t < 8 && q < len; t++, q++)
            out[q] = (uint8_t)(v >> (8 * t));
    }
}

/* ---------------------------------------------------------------------
 * Mutator kernel k (harness standing in for an application kernel).
 *   s_k  = sm(seed ^ sm(k)); then s_k = sm(s_k ^ D(r)) for each read buffer
 *          r in ascending table order (the write depends on what was read)
 *   key  = sm(s_k ^ sm(w)) for written buffer w
 *   fill : 8-byte word j of w is sm(key ^ j), little-endian, tail truncated
 * orc_mutator_seed returns s_k from the digests of the read buffers.
 * ------------------------------------------------------------------- */
uint64_t orc_mutator_seed(uint64_t seed, uint64_t k, const uint64_t *rdig, uint32_t nr) {
    uint64_t s = orc_sm(seed ^ orc_sm(k));
    for (uint32_t t = 0; t < nr; t++) s = orc_sm(s ^ rdig[t]);
    return s;
}

uint64_t orc_mutator_key(uint64_t s_k, uint32_t w) { return orc_sm(s_k ^ orc_sm((uint64_t)w)); }

void orc_mutator_fill(uint8_t *p, uint64_t len, uint64_t s_k, uint32_t w) {
    uint64_t key = orc_mutator_key(s_k, w);
    for (uint64_t j = 0; 8 * j < len; j++) {
        uint64_t v = orc_sm(key ^ j);
        for (uint64_t t = 0; t < 8 && 8 * j + t < len; t++)
            p[8 * j + t] = (uint8_t)(v >> (8 * t));
    }
}

/* Value of the stray 4-byte store made by trace record r of kernel k. */
uint32_t orc_stray_value(uint64_t seed, uint64_t k, uint64_t r) {
    return (uint32_t)orc_sm(orc_sm(seed ^ k) ^ r);
}
