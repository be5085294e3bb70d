/*
 * phos_harness.h -- test and benchmark harness kernels of the PhOS data
 * plane library.  Not part of the method: these stand in for the
 * application whose memory is checkpointed (the paper's evaluation runs
 * real training and inference jobs, Table 4), and give an exact,
 * order-independent fingerprint of memory so that images can be compared
 * without copying them back.
 *
 * Definitions (SplitMix64 of Steele, Lea & Flood, OOPSLA 2014:
 * mix64 = its output function, sm(x) = mix64(x + 0x9E3779B97F4A7C15)):
 *   digest   D(bytes) = sum over 8-byte little-endian words j of
 *            mix64(word_j + j * 0x9E3779B97F4A7C15) mod 2^64, the last word
 *            zero-padded.
 *   mutator  kernel k reading buffers r (ascending) and writing buffers w:
 *            s_k = sm(seed ^ sm(k)), then s_k = sm(s_k ^ D(r)) per read;
 *            word j of each written buffer w = sm(sm(s_k ^ sm(w)) ^ j),
 *            little-endian, tail truncated; then each stray store (record
 *            index r, address a) writes the low 32 bits of
 *            sm(sm(seed ^ k) ^ r) at a, in list order.
 * All calls are asynchronous on the stream and return PHOS_* codes.
 */
#ifndef PHOS_HARNESS_H
#define PHOS_HARNESS_H

#include "phos.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Digest n regions: ptrs[j] (device-accessible address; pinned host memory
 * is translated), lens[j] bytes (host arrays).  d_out: device u64[n],
 * overwritten. */
phos_status phos_harness_digest(const uint64_t *ptrs, const uint64_t *lens, uint32_t n,
                                uint64_t *d_out, phos_stream_t stream);

/* Run mutator kernel k over the table's buffers: reads (ascending table
 * indices, host array, the written buffers included) and writes (host
 * array), then ns stray stores d_strays[2*q] = record index,
 * d_strays[2*q + 1] = address (device array).  Each stray must lie inside
 * a table buffer (4 bytes). */
phos_status phos_harness_mutate(const phos_table_t *t, uint64_t seed, uint64_t k,
                                const uint32_t *reads, uint32_t nr, const uint32_t *writes,
                                uint32_t nw, const uint64_t *d_strays, uint32_t ns,
                                phos_stream_t stream);

/* One application kernel of the stand-in, as the native driver below runs
 * it: its launch arguments (for speculation, phos_speculate's layout), the
 * mutator's read and write sets and stray stores (phos_harness_mutate's),
 * and its recorded access trace (device, 16-byte aligned). */
typedef struct {
    const void *const *args;
    const uint32_t *arg_size;
    const uint8_t *kind;
    uint32_t nargs;
    uint32_t nr;
    const uint32_t *reads;
    const uint32_t *writes;
    uint32_t nw;
    uint32_t ns;
    const uint64_t *d_strays;
    const uint64_t *d_trace;
    uint64_t n_rec;
} phos_harness_kernel_t;

/* Drive a checkpoint session natively through kernels [0, n) of the stand-in,
 * one round per kernel in the order the session defines: copier advance by
 * quota bytes (stop when it reports done), speculation of the kernel's
 * arguments and before_kernel, the mutator as the kernel (seed, index k),
 * after_kernel on its trace (stop after a reported mis-speculation).  The
 * session is not finished.  *kernels_run = rounds run.  Host work per round
 * is the library's own: no interpreter between the calls. */
phos_status phos_harness_drive_ckpt(phos_ckpt_t *c, const phos_table_t *t, uint64_t seed,
                                    uint64_t quota, const phos_harness_kernel_t *ks, uint32_t n,
                                    phos_stream_t stream, uint32_t *kernels_run);

/* Fill [ptr, ptr + len) (device address) with bytes of sm(key ^ j) words:
 * used to give live memory and arenas a reproducible initial content. */
phos_status phos_harness_fill(uint64_t ptr, uint64_t len, uint64_t key, phos_stream_t stream);

/* Test hooks on a table handle.
 * phos_harness_table_rebind records `device` as the device the table
 * belongs to (the previous value in *old_device, nullable); nothing is
 * moved, so the table is only usable again once the true device is
 * recorded back.  It lets a one-GPU test reach the device-mismatch
 * rejection of calls that must not switch devices.
 * phos_harness_table_scratch reports the bytes of the table's growable
 * validation scratch (0 until a call has needed it). */
phos_status phos_harness_table_rebind(phos_table_t *t, int device, int *old_device);
phos_status phos_harness_table_scratch(const phos_table_t *t, uint64_t *val_bytes);

/* Deferred validation of several kernel rounds in one launch, as a no-sync
 * checkpoint or restore session with PHOS_CKPT_DEFER runs it (Sec. 4.1
 * "Runtime validation" with the response of Sec. 4.3, 4.2 or 6), exposed so
 * that tests and benchmarks can reach the launch directly.  Round i checks
 * d_trace[0, n_rec) (device, 16-byte aligned; access width access_bytes)
 * against its own d_perm (device, n bytes) and answers with its own d_flags
 * (device, n bytes):
 *   rule 1 (recopy):  every store victim b with d_flags[b] != 0 gets
 *                     d_dirty[b] = 1;
 *   rule 2 (CoW):     a store victim b with d_flags[b] == 0 makes the round a
 *                     mis-speculation;
 *   rule 3 (restore): any victim b with d_flags[b] == 0 does.
 * d_acc (device u64[8]): d_acc[3] += the violations of all rounds; if
 * (int64)d_acc[4] < 0 and some round mis-speculated, d_acc[4] and *d_flag
 * (device-accessible int64, e.g. mapped pinned memory) become the `round`
 * of the first such round in the array's order.  d_status as for
 * phos_validate.  d_scratch: phos_harness_rounds_scratch bytes of device
 * memory, zeroed once by the caller; each launch leaves it zeroed, and
 * launches that overlap on the GPU must not share it.  k <= 16; EINVAL if
 * the table is too large for k rounds in one launch. */
typedef struct {
    const uint64_t *d_trace;
    uint64_t n_rec;
    const uint8_t *d_perm;
    const uint8_t *d_flags;
    int64_t round;
} phos_harness_round_t;
phos_status phos_harness_validate_rounds(const phos_table_t *t, const phos_harness_round_t *rounds,
                                         uint32_t k, uint32_t access_bytes, uint32_t rule,
                                         uint8_t *d_dirty, uint64_t *d_acc, int64_t *d_flag,
                                         uint32_t *d_status, void *d_scratch,
                                         phos_stream_t stream);
/* Bytes of the scratch above for the table (any k), and the most rounds one
 * launch takes for it (0: the table is too large for deferred validation). */
phos_status phos_harness_rounds_scratch(const phos_table_t *t, uint64_t *bytes,
                                        uint32_t *max_rounds);

#ifdef __cplusplus
}
#endif
#endif /* PHOS_HARNESS_H */
