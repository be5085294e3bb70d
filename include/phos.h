/*
 * phos.h -- C ABI of the PhOS data plane on B300 (sm_103a).
 *
 * The data plane of concurrent GPU checkpoint/restore with validated
 * speculation (PhoenixOS, SOSP'25, arXiv 2405.12079):
 *   - argument-based speculation of a kernel's read/write buffers (Sec. 4.1,
 *     read set in Sec. 6), host side;
 *   - access validation of recorded load/store addresses against the
 *     speculated buffers (Sec. 4.1 "Runtime validation"), CUDA;
 *   - the copy engine behind soft copy-on-write (Sec. 4.2), soft recopy
 *     (Sec. 4.3, chunked per Sec. 5) and soft on-demand restore (Sec. 6),
 *     CUDA;
 *   - the protocol state machines that drive them (phos_ckpt_*,
 *     phos_restore_*), host C++.
 *
 * Conventions for every call
 *   - Return value: PHOS_OK or one of the error codes below; the message of
 *     the last failure on the calling thread is phos_last_error().
 *   - Device work is asynchronous on the caller's stream (a cudaStream_t
 *     passed as phos_stream_t; NULL = legacy default stream).  Errors found
 *     on the device are written to a caller-owned uint32_t status word
 *     (d_status, device or mapped memory, zeroed once by the caller): the
 *     first error code sticks, later calls never clear it.  Read it after
 *     synchronising the stream.
 *   - Ownership: the caller owns every buffer passed in (live memory,
 *     staging, image, traces, outputs); the library never frees caller
 *     memory and never synchronises, except where a call says so.  The
 *     library owns only its opaque handles and their scratch memory.
 *   - "image" pointers may be pinned host memory (cudaHostAlloc or
 *     cudaHostRegister; the kernels reach it through its mapped device
 *     address) or device memory; pageable host memory is rejected.
 *   - Calls that use the same table handle and run concurrently on
 *     different streams race on the handle's scratch; order them.
 *   - Device work goes to the calling thread's current CUDA device, which
 *     must be the device that was current when the handle was created (a
 *     table records it).  Only phos_validate_noalloc checks this
 *     (PHOS_EINVAL).  The server is the exception: its own thread, and
 *     phos_server_submit and phos_server_app_copy on the caller's thread,
 *     make the server's device current.
 */
#ifndef PHOS_H
#define PHOS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t phos_status;
enum {
    PHOS_OK = 0,
    PHOS_EINVAL = 1,     /* bad argument, table, descriptor or record      */
    PHOS_ENOMEM = 2,     /* library scratch allocation failed              */
    PHOS_EBUDGET = 3,    /* staging budget exhausted and no fallback       */
    PHOS_ECUDA = 4,      /* a CUDA runtime call failed                     */
    PHOS_ETIMEDOUT = 5,  /* a bounded device-side wait gave up             */
    PHOS_ECORRUPT = 6,   /* digest mismatch in a checkpoint image          */
    PHOS_EMISSPEC = 7    /* validation found a mis-speculation that needed
                            the stop-the-world fallback                    */
};

typedef void *phos_stream_t;             /* a cudaStream_t */

/* One buffer of the process (Sec. 2.1: a contiguous virtual range per
 * allocation; Sec. 4.1: the OS learns them by intercepting allocation). */
typedef struct {
    uint64_t base;                        /* first byte                    */
    uint64_t size;                        /* bytes, > 0                    */
} phos_buf_t;

/* Speculated permission per buffer (Sec. 4.1 write set, Sec. 6 read set).
 * A mutable pointer argument both reads and writes its buffer.           */
enum { PHOS_PERM_NONE = 0, PHOS_PERM_R = 1, PHOS_PERM_W = 2, PHOS_PERM_RW = 3 };

/* Kind of a launch argument (Sec. 4.1: the kernel signature tells pointer
 * from scalar and const from mutable; an opaque struct is scanned in
 * 8-byte chunks, each a possible mutable pointer).                      */
enum { PHOS_ARG_SCALAR = 0, PHOS_ARG_CONST_PTR = 1, PHOS_ARG_MUT_PTR = 2,
       PHOS_ARG_STRUCT = 3 };

/* Trace record: bit 63 = store, bits 57..62 reserved (must be 0),
 * bits 0..56 = the accessed address.                                     */
#define PHOS_REC_STORE (1ull << 63)
#define PHOS_REC_ADDR_MASK ((1ull << 57) - 1ull)

/* Copy descriptor: one (buffer, offset, len) region (Sec. 4.2 CoW copy,
 * Sec. 4.3 recopy, Sec. 5 4 MB chunks, Sec. 6 restore).  A live endpoint is
 * (table index buf, offset inside that buffer); a staging or image
 * endpoint is a byte offset into the staging or image area of the call.  */
typedef struct {
    uint64_t src_off;
    uint64_t dst_off;
    uint64_t len;
    uint32_t buf;
    uint32_t flags;                       /* PHOS_COPY_* direction | marks  */
} phos_copy_t;
enum {
    PHOS_COPY_LIVE_TO_STAGING = 1,        /* CoW: buffer -> device staging  */
    PHOS_COPY_LIVE_TO_IMAGE = 2,          /* checkpoint / recopy            */
    PHOS_COPY_STAGING_TO_IMAGE = 3,       /* drain a CoW shadow             */
    PHOS_COPY_IMAGE_TO_LIVE = 4,          /* restore                        */
    PHOS_COPY_DIR_MASK = 0xff,
    PHOS_COPY_MARK_PRESENT = 0x100        /* set bit buf of the present
                                             bitmap once these bytes landed */
};

const char *phos_last_error(void);
const char *phos_status_name(phos_status s);

/* Number of CUDA kernels this library has launched in the process so far
 * (diagnostics: lets a caller count launches inside a timed region). */
uint64_t phos_launch_count(void);

/* ---------------------------------------------------------------- table */

typedef struct phos_table phos_table_t;

/* Copy n buffers (host array, sorted by base, disjoint, size > 0, inside
 * the 57-bit address space) into a device-resident table.  Synchronous.
 * At most 32,768 buffers (the validation kernels' three-level search).
 * EINVAL if the rules are broken, checked on the host before any device
 * work; n may be 0 (every access then fails validation as unmapped).  The
 * table keeps a host copy for speculation. */
phos_status phos_table_create(const phos_buf_t *bufs, uint32_t n, phos_table_t **out);
phos_status phos_table_destroy(phos_table_t *t);
uint32_t phos_table_size(const phos_table_t *t);

/* ----------------------------------------------------------- speculate */

/* Argument-based speculation (Sec. 4.1, Sec. 6), host side.
 * args[j] points at the bytes of argument j (arg_size[j] bytes, little
 * endian), kind[j] is PHOS_ARG_*.  Pointer arguments use their first 8
 * bytes (zero-extended if shorter); a struct is scanned at offsets 0, 8,
 * ... and a trailing partial chunk is ignored.  Every value v with
 * base <= v < base + size marks that buffer R (const) or RW (mutable,
 * struct).  perm_out (host, n bytes) is OR-accumulated: zero it first. */
phos_status phos_speculate(const phos_table_t *t, const void *const *args,
                           const uint32_t *arg_size, const uint8_t *kind,
                           uint32_t nargs, uint8_t *perm_out);

/* The same speculation on the device, for many launches at once (the
 * batched form: a queue of launches of one process image).  The caller
 * flattens the arguments into 8-byte words: a pointer argument is one word
 * (its first 8 bytes, zero-extended), a struct one word per full 8-byte
 * chunk, scalars may be left out.  d_words: device u64[total words];
 * d_kind: u8 PHOS_ARG_* of the argument each word came from (a kind above
 * PHOS_ARG_STRUCT sets d_status to PHOS_EINVAL and the word is ignored);
 * d_launch_off: u64[n_launch + 1], launch l owns words [off[l], off[l+1])
 * (a decreasing pair sets PHOS_EINVAL and the launch is skipped); d_perm:
 * device u8[n_launch][n], row l for launch l, OR-accumulated (zero it
 * first).  d_status may be NULL.  Asynchronous on stream. */
phos_status phos_speculate_device(const phos_table_t *t, const uint64_t *d_words,
                                  const uint8_t *d_kind, const uint64_t *d_launch_off,
                                  uint32_t n_launch, uint8_t *d_perm, uint32_t *d_status,
                                  phos_stream_t stream);

/* Type-1 APIs (Sec. 4.1, memory moves): a call that reads or writes
 * [addr, addr + len) marks every buffer the range overlaps with perm. */
phos_status phos_speculate_region(const phos_table_t *t, uint64_t addr, uint64_t len,
                                  uint8_t perm, uint8_t *perm_out);

/* ------------------------------------------------------------ validate */

/* Access validation (Sec. 4.1 "Runtime validation"; reads too, Sec. 6).
 * For each record r of d_trace (n_rec records, 16-byte aligned device
 * array): find the buffer i with base_i <= a and a + access_bytes <=
 * base_i + size_i.  Outcomes:
 *   no such buffer (gap, straddle, or reserved bits set) -> violation,
 *       counted in d_count[2] ("unmapped"; reserved bits also make the
 *       status word PHOS_EINVAL)
 *   load and !(d_perm[i] & R), or store and !(d_perm[i] & W)
 *       -> violation; bit i set in d_victim, and in d_victim_st if a store
 * d_bitmap (u32[ceil(n_rec/32)]): bit r&31 of word r>>5 set per violation,
 *   padding bits 0.  d_count (u64[3]): violations, store violations,
 *   unmapped violations.  d_victim, d_victim_st (u32[ceil(n/32)]) and d_idx
 *   (the first idx_cap violating r, ascending) may be NULL.
 * All outputs are overwritten.  d_perm: device u8[n].  access_bytes >= 1.
 * Asynchronous on stream; uses the table handle's scratch. */
phos_status phos_validate(const phos_table_t *t, const uint8_t *d_perm,
                          const uint64_t *d_trace, uint64_t n_rec, uint32_t access_bytes,
                          uint32_t *d_bitmap, uint64_t *d_count, uint32_t *d_victim,
                          uint32_t *d_victim_st, uint64_t *d_idx, uint64_t idx_cap,
                          uint32_t *d_status, phos_stream_t stream);

/* phos_validate for callers that cannot allocate device memory.  The paper
 * has no counterpart: it exists for this library's users.  Examples are an
 * interposer validating from inside an application's intercepted CUDA call
 * (allocating there can re-enter the interception layer or deadlock on the
 * application's allocator lock) and callers that must not let cudaMalloc's
 * implicit device synchronisation stall the application's kernels during a
 * concurrent checkpoint.
 * Same arguments, results and error behaviour as phos_validate, but the
 * call allocates nothing: its scratch (per-CTA counts, victim accumulators,
 * a completion ticket; 12.5 KB) is a fixed array inside the library that
 * every GPU which loads the library holds until the process exits.
 * Limits: tables of at most 16384 buffers (larger ones get PHOS_EINVAL and
 * a message; use phos_validate for them) and at most 256 CTAs per launch
 * (the call never launches more).  The process-wide settings of
 * phos_validate_config and phos_validate_grid do not apply here: this call
 * always runs the batched-leader kernel on min(SMs, 256) CTAs (same
 * results, possibly different timing).  The table's device must be the
 * calling thread's current device (else PHOS_EINVAL, nothing launched):
 * the call never switches devices.  The first call on a device looks up
 * the array's address there; make that first call before any stream
 * capture.
 * Every call clears the parts of the array it uses, then launches; all
 * calls share the one array, so calls that overlap on the GPU (concurrent
 * streams, or several host threads) race and must be ordered by the
 * caller. */
phos_status phos_validate_noalloc(const phos_table_t *t, const uint8_t *d_perm,
                                  const uint64_t *d_trace, uint64_t n_rec,
                                  uint32_t access_bytes, uint32_t *d_bitmap, uint64_t *d_count,
                                  uint32_t *d_victim, uint32_t *d_victim_st, uint64_t *d_idx,
                                  uint64_t idx_cap, uint32_t *d_status, phos_stream_t stream);

/* Kernel variant of phos_validate (process-wide; the autotuner sets it):
 * 0 = default, 1 = bulk-copy ring with one warp-cooperative search per
 * 32 records, 2 = batched leaders (each lane searches the first record of
 * one of 32 words, the warp checks all 32 words against them).  Results
 * are identical; only speed differs. */
phos_status phos_validate_config(uint32_t variant);
/* Bound on the waits of the bulk-copy ring variant (variant 1) for a staged
 * trace tile: the number of mbarrier probes before the wait gives up
 * (default 2^24, far beyond any copy's latency).  A wait that gives up makes
 * the CTA stop validating, wait (with the default bound) for its copies
 * still in flight, and set PHOS_ETIMEDOUT in d_status; the outputs of that
 * launch are then undefined and the device stays usable.  0 makes every
 * such wait give up at once: a deterministic test of that path.
 * Process-wide. */
phos_status phos_validate_wait_limit(uint32_t probes);
/* Grid of phos_validate: 0 (default) = one CTA per SM, else that many CTAs
 * (at most 4096; each CTA stages the table once).  Process-wide. */
phos_status phos_validate_grid(uint32_t ctas);

/* --------------------------------------------------------- copy engine */

/* Gather-copy n descriptors (d_list: device array) between live buffers,
 * the staging area and the image.  Bounds: live off + len <= size[buf];
 * staging / image off + len <= their byte sizes.  A descriptor that breaks
 * a rule, or whose direction the entry point does not allow, moves nothing
 * and sets PHOS_EINVAL in d_status; the others still run.  Source and
 * destination must not overlap.  Asynchronous on stream.
 *
 * phos_cow_copy            live -> staging only (Sec. 4.2 copy-on-write)
 * phos_recopy              live -> image only (Sec. 4.3 recopy; also the
 *                          bulk checkpoint copy of Sec. 4.2/5)
 * phos_restore_on_demand   image -> live only (Sec. 6); descriptors with
 *                          PHOS_COPY_MARK_PRESENT set bit buf of d_present
 *                          (u32[ceil(n/32)], device) after their bytes land
 * phos_copy                any direction, mixed in one launch (the
 *                          background copier: shadow or live -> image) */
phos_status phos_cow_copy(const phos_table_t *t, const phos_copy_t *d_list, uint32_t n,
                          void *d_staging, uint64_t staging_bytes, uint32_t *d_status,
                          phos_stream_t stream);
phos_status phos_recopy(const phos_table_t *t, const phos_copy_t *d_list, uint32_t n,
                        void *image, uint64_t image_bytes, uint32_t *d_status,
                        phos_stream_t stream);
phos_status phos_restore_on_demand(const phos_table_t *t, const phos_copy_t *d_list, uint32_t n,
                                   const void *image, uint64_t image_bytes,
                                   uint32_t *d_present, uint32_t *d_status,
                                   phos_stream_t stream);
phos_status phos_copy(const phos_table_t *t, const phos_copy_t *d_list, uint32_t n,
                      void *d_staging, uint64_t staging_bytes, void *image,
                      uint64_t image_bytes, uint32_t *d_present, uint32_t *d_status,
                      phos_stream_t stream);

/* Launch shape of the copy engine: tile_bytes per CTA work item (multiple
 * of 4096, 4 KiB..16 MiB) and CTAs per SM (1..8).  Process-wide; the
 * autotuner sets it.  0 leaves a field unchanged. */
phos_status phos_copy_config(uint64_t tile_bytes, uint32_t ctas_per_sm);

/* Image layout used by the protocols: buffer i at img_off[i] = sum of
 * align256(size) of the buffers before it; returns the total bytes. */
uint64_t phos_image_bytes(const phos_table_t *t);
phos_status phos_image_offsets(const phos_table_t *t, uint64_t *img_off_out);

/* Checkpoint frequency for fault tolerance (Appendix A.1): N GPUs, each
 * failing F times per hour, checkpoint overhead O hours, restore time R
 * hours, job length T hours.  Wasted GPU hours at f checkpoints per hour:
 *   W(f) = N F T (R + N / (2 f)) + N O f T
 * (the paper's formula, taken as printed), minimised at f* = sqrt(N F / (2 O)).
 * Writes f* and W(f*); EINVAL unless N, F, O > 0 and R, T >= 0. */
phos_status phos_ckpt_frequency(double n_gpus, double fail_per_hour, double overhead_h,
                                double restore_h, double hours, double *f_opt,
                                double *wasted_at_opt);

/* ---------------------------------------------------------- batched plan
 *
 * Many process images' validation traces and copy lists in one persistent
 * launch, replayed as a CUDA graph.  Per item, the results are exactly those
 * of phos_validate (no index list) and phos_copy on the same arguments.
 * Items are independent images: no item's copies may write what another
 * item reads or writes.  Present marks (restore) are not supported here. */

typedef struct phos_plan phos_plan_t;

typedef struct {
    const phos_table_t *table;   /* the item's buffer table                  */
    const uint8_t *d_perm;       /* device u8[n], speculated permissions      */
    const uint64_t *d_trace;     /* device, 16-byte aligned; n_rec records    */
    uint64_t n_rec;
    uint32_t access_bytes;       /* >= 1 when n_rec > 0                       */
    uint32_t n_copy;             /* descriptors in d_list                     */
    uint32_t *d_bitmap;          /* outputs as in phos_validate; d_count is   */
    uint64_t *d_count;           /* required, the victim bitmaps may be NULL  */
    uint32_t *d_victim;
    uint32_t *d_victim_st;
    const phos_copy_t *d_list;   /* device descriptors, read once at create   */
    void *staging;               /* the item's staging area and image         */
    uint64_t staging_bytes;
    void *image;
    uint64_t image_bytes;
} phos_plan_item_t;

/* Resolve and check every descriptor (host side, once; synchronous), size
 * the plan's shared memory for its largest table (EINVAL if it does not
 * fit) and capture the launch as a CUDA graph.  The plan keeps the item
 * pointers: the caller keeps that memory alive and unchanged in place
 * (contents may change between launches: traces, permissions and the
 * bytes being copied are read at launch time). */
phos_status phos_plan_create(const phos_plan_item_t *items, uint32_t n_items,
                             phos_plan_t **out);
/* One graph launch on the stream: validation of every item, then every
 * copy; outputs overwritten. */
phos_status phos_plan_launch(phos_plan_t *p, phos_stream_t stream);
/* Copy work-item size (multiple of 4 KiB, 4 KiB .. 16 MiB); re-captures. */
phos_status phos_plan_set_tile(phos_plan_t *p, uint64_t tile_bytes);
/* Autotuner: times the plan at tile sizes 64 KiB .. 4 MiB (two warm-up and
 * five timed launches each, best of five) and keeps the fastest.  The
 * launches really run: outputs and copies are produced each time. */
phos_status phos_plan_autotune(phos_plan_t *p, phos_stream_t stream, uint64_t *best_tile,
                               float *best_ms);
/* Totals of the plan and its device status word (synchronous copy). */
phos_status phos_plan_info(const phos_plan_t *p, uint64_t *records, uint64_t *copy_bytes,
                           uint64_t *tile_bytes, uint32_t *status_out);
phos_status phos_plan_destroy(phos_plan_t *p);

/* ------------------------------------------------------------ serving
 *
 * Continuous batching of checkpoint and restore requests (Sec. 7: periodic
 * checkpoints for fault tolerance, restore-mostly serverless startups).  A
 * scheduler thread admits requests as slots and the staging budget free up
 * (a checkpoint needs staging for its whole image, a restore none, so a
 * restore may pass a checkpoint that waits), snapshots checkpoints into
 * staging at HBM speed, and moves every admitted request's host leg in
 * pieces, oldest request first, device->host and host->device at the same
 * time.  Pieces of >= dma_min bytes go to the DMA engines, smaller
 * ones to the SM copy kernel.  Requests must be independent: no two
 * requests in flight may share a table handle or overlapping memory. */

typedef struct phos_server phos_server_t;
enum { PHOS_REQ_CHECKPOINT = 1, PHOS_REQ_RESTORE = 2 };
/* Server flags. */
enum { PHOS_SERVER_APP_PRIORITY = 1 };

typedef struct {
    uint32_t max_slots;      /* requests on the device at once (1 = one at a
                                time, strictly in arrival order)            */
    uint32_t flags;          /* PHOS_SERVER_*                               */
    void *d_staging;         /* device staging area (checkpoint snapshots)  */
    uint64_t staging_bytes;  /* admission budget                            */
    uint64_t chunk;          /* host-leg piece size, multiple of 256        */
    uint64_t dma_min;        /* pieces >= this go to the DMA engines; 0 = none */
    uint64_t window;         /* host-leg bytes queued on the GPU per direction,
                                at most (two batches of window/2, each at
                                least one chunk); 0 = two batches of
                                max(8 chunks, 64 MiB).  With APP_PRIORITY it
                                bounds how long an application transfer can
                                wait behind C/R pieces already issued.      */
} phos_server_desc_t;

typedef struct {
    uint32_t kind;                /* PHOS_REQ_*                              */
    uint32_t reserved;
    const phos_table_t *table;    /* the process image (live device buffers) */
    void *host;                   /* pinned image: destination of a checkpoint,
                                     source of a restore (phos_image_offsets
                                     layout), >= phos_image_bytes(table)     */
    uint64_t host_bytes;
} phos_request_t;

typedef struct {
    uint32_t state;               /* 0 queued, 1 admitted, 2 done, 3 failed,
                                     4 cancelled                             */
    phos_status status;
    uint64_t bytes;               /* image bytes moved                       */
    uint64_t t_submit_ns;         /* CLOCK_MONOTONIC                         */
    uint64_t t_admit_ns;
    uint64_t t_done_ns;           /* the last byte is at its destination     */
} phos_result_t;

phos_status phos_server_start(const phos_server_desc_t *d, phos_server_t **out);
/* Thread-safe; returns a ticket.  EBUDGET if the image can never fit the
 * staging budget. */
phos_status phos_server_submit(phos_server_t *s, const phos_request_t *r, uint64_t *ticket);
/* Non-blocking. */
phos_status phos_server_poll(phos_server_t *s, uint64_t ticket, phos_result_t *out);
/* Cancel a request (one of the failures a serving loop must survive; the
 * other requests are not affected).  Queued: it leaves the queue at once
 * (state 4).  Admitted: no further piece of it is issued; it ends (state 4)
 * once its pieces already on the GPU have landed, and a checkpoint's
 * staging is then released.  A request whose last piece was already issued
 * completes normally (state 2), as does a finished one.  A cancelled
 * checkpoint leaves its host image partly written, a cancelled restore its
 * live buffers partly restored.  Non-blocking, thread-safe; EINVAL for an
 * unknown ticket. */
phos_status phos_server_cancel(phos_server_t *s, uint64_t ticket);
/* Wait until nothing is queued or in flight (ETIMEDOUT after timeout_ms). */
phos_status phos_server_drain(phos_server_t *s, uint32_t timeout_ms);
/* Finish what was submitted, then stop the scheduler and free its streams. */
phos_status phos_server_stop(phos_server_t *s);

/* An application transfer that the server's C/R traffic yields to (Sec. 5,
 * "Prioritized application PCIe transfer": the checkpoint is copied in
 * chunks and, after each one, pauses while an application transfer is
 * pending or running).  Copies `bytes` from src to dst on the caller's
 * `stream` (cudaMemcpyAsync, so the application keeps its own stream
 * order) and registers the transfer with the server.  One side must be
 * pinned host memory and the other device memory; the direction follows
 * from the pointers.  With PHOS_SERVER_APP_PRIORITY the scheduler issues
 * no C/R piece, in either direction (a copy engine may serve both), from
 * the moment of this call until the transfer completes, so it waits at
 * most for the C/R bytes already queued (desc.window per direction);
 * without the flag the transfer is only counted.  Thread-safe.  EINVAL: NULL pointers, pageable host memory, or
 * both sides on the device / on the host. */
phos_status phos_server_app_copy(phos_server_t *s, void *dst, const void *src, uint64_t bytes,
                                 cudaStream_t stream);

typedef struct {
    uint64_t app_copies;          /* application transfers registered        */
    uint64_t app_bytes;
    uint64_t paused_turns;        /* scheduler turns in which a direction's C/R
                                     issue was held back for an application
                                     transfer                                */
    uint64_t batches;             /* C/R host-leg batches issued             */
    uint64_t cancelled;           /* requests ended by phos_server_cancel    */
} phos_server_stats_t;
phos_status phos_server_stats(phos_server_t *s, phos_server_stats_t *out);

/* Host legs of the protocol drivers below: pieces that cross PCIe (to or
 * from the image) and are at least dma_min_bytes long go to the DMA copy
 * engines (cudaMemcpyAsync, one call per piece, as the paper's prototype
 * copies, Sec. 5) instead of the SM copy kernel; 0 keeps every piece on
 * the SM copy kernel.  Default 256 KiB: the engines move 57 GB/s of
 * payload over this link against 53 GB/s for SM stores, and a sub-MiB
 * piece left to the SM kernel costs a copy launch pair on the copier's
 * stream.  Process-wide. */
phos_status phos_host_copy_config(uint64_t dma_min_bytes);

/* ------------------------------------------------- protocol control plane
 *
 * Lockstep drivers of the three concurrent protocols.  The caller plays
 * the application: between phos_*_before_kernel and phos_*_after_kernel it
 * launches its kernel on the same stream.  A "round" is: advance (the
 * background copier moves up to quota bytes), before_kernel (the protocol
 * acts on the kernel's speculated buffers), the caller's kernel,
 * after_kernel (validation of the kernel's access trace and the
 * mis-speculation rules).  Copier order: ascending table index, pieces of
 * at most `chunk` bytes that never cross a buffer and are cut at the
 * remaining quota; each piece charges align256(len) against the quota.
 * Image layout: phos_image_offsets.  Only after_kernel, finish and the
 * fallbacks synchronise the stream. */

typedef struct phos_ckpt phos_ckpt_t;
typedef struct phos_restore phos_restore_t;

enum { PHOS_CKPT_COW = 1, PHOS_CKPT_RECOPY = 2 };
/* OR'ed into phos_ckpt_desc_t.mode: after_kernel does not wait for the
 * validation.  The protocol's response to it runs on the device instead
 * (recopy: store victims in flight or done become dirty; CoW: the first
 * round with a store victim neither done nor shadowed is recorded), so a
 * round is enqueue-only and the host may run ahead of the device.  A CoW
 * mis-speculation reaches the host through a mapped word: advance or
 * after_kernel report it once visible (advance: done; after_kernel:
 * *misspec = 1), and finish, which synchronises, copies every buffer
 * stop-the-world at that point (later than the synchronous mode's
 * fallback, which runs right after the kernel; both images are the memory
 * of one instant).  Copies issued between the mis-speculation and its
 * discovery are wasted but harmless.  stats and the dirty log synchronise
 * first in this mode.  Results without a mis-speculation are identical to
 * the synchronous mode's. */
enum { PHOS_CKPT_NO_SYNC = 0x100 };
/* OR'ed into mode (implies PHOS_CKPT_NO_SYNC): the background copier runs
 * on a stream of its own, concurrently with the caller's kernels, instead
 * of in lockstep on the caller's stream.  Each copier batch starts after
 * the work the caller had enqueued before that advance call; a CoW kernel
 * waits (stream event) only for the copier batches that still read a
 * buffer it may write, or a staging extent it reuses; recopy kernels never
 * wait (a buffer the copier touched and the kernel writes is dirty
 * anyway).  Every host decision, and so every result, is the lockstep
 * mode's. */
enum { PHOS_CKPT_CONCURRENT = 0x200 };
/* Copier window of PHOS_CKPT_CONCURRENT sessions (process-wide; 0, the
 * default, = none): before an advance issues the copier's next pieces, the
 * calling thread waits until at most `bytes` of earlier copier pieces are
 * still in flight.  Without a window the host may issue the whole image at
 * once, and a kernel that needs a buffer whose pieces sit deep in the
 * copier's queue waits for that queue; with one, such pieces are never far
 * from landing.  The pieces and every decision are unchanged (they depend
 * on rounds, not on timing); only when the host issues them changes. */
phos_status phos_copier_window(uint64_t bytes);
/* OR'ed into mode (CoW sessions) or restore flags (implies
 * PHOS_CKPT_NO_SYNC; not with PHOS_CKPT_CONCURRENT or a manifest): every
 * per-round decision is taken on the device from device-resident state --
 * the copier's pieces, the CoW set with its first-fit staging allocation
 * (or the direct copy when staging is full), the restore need set, and the
 * flags the validation rule reads -- so a round is a fixed sequence of
 * launches on the caller's stream and needs no host data: pass the round's
 * speculated permissions as a device array to *_before_kernel_dev (for
 * example rows of phos_speculate_device's output).  Every decision follows
 * the same rules as the host's, so lists and images are the lockstep
 * mode's.  The host does not learn when the copier finishes: advance
 * reports done only after a mis-speculation (restore: after its
 * roll-back), rounds after the end are no-ops for the protocol, and finish
 * drains the rest, then reads the device's logs (capacity fixed at begin;
 * PHOS_ENOMEM if exceeded).  Copies are all SM-issued (no DMA host legs:
 * the host does not see the pieces). */
enum { PHOS_CKPT_DEVICE = 0x400 };
/* OR'ed into mode or restore flags (implies PHOS_CKPT_NO_SYNC; not with
 * PHOS_CKPT_DEVICE): after_kernel does not launch the round's validation.
 * It queues the round, and up to 16 queued rounds are validated in one
 * launch -- each round's trace against that round's speculated
 * permissions, and the protocol's rule answered with that round's flags,
 * as the launch per round would -- when the queue is full, and before
 * anything that reads the rule's results or recycles the session's upload
 * arena (finish, stats, logs, begin_pass, a roll-back).  Results are the
 * no-sync mode's; a mis-speculation reaches the host up to 16 rounds later
 * (at the latest at finish).  A round's trace must stay unchanged in device
 * memory until it has been validated: until 16 more rounds have run, or
 * until finish.  A round whose trace is longer than 2^24 records, and every
 * round of a table too large for two rounds' permissions and victim sets
 * in one CTA's shared memory, is validated at once (after the queued
 * rounds). */
enum { PHOS_CKPT_DEFER = 0x800 };
/* Restore flags only, with PHOS_CKPT_CONCURRENT (Sec. 6 leaves the order
 * within a round open): each round fetches its kernel's missing buffers
 * first and moves the copier after -- per round: before_kernel(perm), then
 * advance(quota, &done), the kernel, after_kernel -- so the copier never
 * moves a buffer that round's kernel needs, the kernel never waits for its
 * own round's copier pieces, and the copier's pieces start after the
 * round's on-demand copies (which then have the link to themselves).
 * advance is allowed only there, once per round; done = 1 means every
 * buffer is restored (or a mis-speculation has been seen): the round's
 * kernel and after_kernel still belong to the session, and the caller
 * starts no further round.  EINVAL without PHOS_CKPT_CONCURRENT. */
enum { PHOS_RESTORE_ONDEMAND_FIRST = 0x1000 };

typedef struct {
    uint32_t mode;           /* PHOS_CKPT_COW (Sec. 4.2) or PHOS_CKPT_RECOPY
                                (Sec. 4.3)                                   */
    uint32_t access_bytes;   /* width of every traced access (>= 1)          */
    uint64_t chunk;          /* copier piece size, multiple of 256 (Sec. 5
                                uses 4 MiB)                                 */
    void *d_staging;         /* CoW staging area (device); may be NULL       */
    uint64_t staging_bytes;  /* CoW budget (Sec. 4.2 reserves up to 2 GB)    */
    void *image;             /* destination, >= phos_image_bytes(t) bytes    */
    uint64_t image_bytes;
} phos_ckpt_desc_t;

typedef struct {
    uint64_t kernels;        /* rounds begun (before_kernel calls)           */
    uint64_t copier_bytes;   /* bytes the background copier moved            */
    uint64_t cow_bytes;      /* CoW copies into staging                      */
    uint64_t direct_bytes;   /* CoW with no room: straight to the image      */
    uint64_t recopy_bytes;   /* recopy at t2                                 */
    uint64_t validated;      /* trace records validated                      */
    uint64_t violations;     /* of which violations                          */
    int64_t misspec_round;   /* round whose validation forced the
                                stop-the-world fallback, or -1               */
    uint32_t done;           /* 1 once the image is complete                 */
    uint32_t dirty;          /* recopy: size of the dirty set                */
    uint64_t passes;         /* recopy: extra concurrent passes started      */
} phos_ckpt_stats_t;

/* Start a checkpoint at t1 (the caller has quiesced: Sec. 4.2 phase 1).
 * Every buffer is pending.  Allocates the session's device and pinned
 * scratch. */
phos_status phos_ckpt_begin(const phos_table_t *t, const phos_ckpt_desc_t *d,
                            phos_stream_t stream, phos_ckpt_t **out);
/* Background copier: up to quota bytes (shadow if one exists, else live ->
 * image).  *done = 1 once every buffer is in the image. */
phos_status phos_ckpt_advance(phos_ckpt_t *c, uint64_t quota, int *done);
/* perm: host u8[n] speculated for the next kernel.  CoW: every speculated
 * write buffer that is neither done nor shadowed is copied whole to
 * staging (first fit, align256(size)) or, without room, its remaining
 * bytes go straight to the image (Sec. 4.2).  Recopy: speculated write
 * buffers that are in flight or done join the dirty set (Sec. 4.3). */
phos_status phos_ckpt_before_kernel(phos_ckpt_t *c, const uint8_t *perm);
/* Validate the kernel's trace (device, 16-byte aligned) against perm;
 * synchronises (PHOS_CKPT_NO_SYNC: enqueues and returns).  CoW: a store victim that was neither done nor shadowed
 * before the kernel discards the checkpoint and copies every buffer
 * stop-the-world now; *misspec = 1 and the session is complete.  Recopy:
 * store victims that were in flight or done join the dirty set. */
phos_status phos_ckpt_after_kernel(phos_ckpt_t *c, const uint64_t *d_trace, uint64_t n_rec,
                                   int *misspec);
/* PHOS_CKPT_DEVICE sessions: the round's CoW set from d_perm (device
 * u8[n], read when the round runs on the stream), decided on the device. */
phos_status phos_ckpt_before_kernel_dev(phos_ckpt_t *c, const uint8_t *d_perm);
/* Drain the rest; recopy: quiesce point t2, recopy the dirty set whole.
 * Synchronises. */
phos_status phos_ckpt_finish(phos_ckpt_t *c);
/* Iterative recopy (Sec. 4.3 "iteratively do the concurrent recopy"): when
 * a recopy session's copier has finished a pass (advance reported done),
 * start another concurrent pass over the current dirty set instead of
 * quiescing: those buffers become pending (copied from their start again)
 * and the dirty set empties; the dirty rule is unchanged.  *pass_bytes =
 * bytes of the new pass.  The caller decides when to stop (for instance
 * when the dirty bytes stop shrinking) and then calls phos_ckpt_finish,
 * which recopies the remaining dirty set stop-the-world. */
phos_status phos_ckpt_begin_pass(phos_ckpt_t *c, uint64_t *pass_bytes);
phos_status phos_ckpt_stats(const phos_ckpt_t *c, phos_ckpt_stats_t *out);
/* Event logs, 5 u64 per event (n_out = number of events available):
 *   0 CoW:     round, buffer, 1 = staging / 2 = direct, offset, len
 *   1 copier:  round, buffer, offset in buffer, len, 1 if from a shadow
 *   2 dirty:   buffer, 0, 0, 0, 0 (ascending)
 *   3 passes:  round, buffers, bytes, 0, 0 (one per phos_ckpt_begin_pass) */
phos_status phos_ckpt_log(const phos_ckpt_t *c, uint32_t kind, uint64_t *out, uint64_t cap,
                          uint64_t *n_out);
phos_status phos_ckpt_end(phos_ckpt_t *c);

typedef struct {
    uint32_t access_bytes;
    uint32_t flags;          /* PHOS_CKPT_NO_SYNC | PHOS_CKPT_CONCURRENT, as
                                for checkpoints: no wait per kernel (the
                                mis-speculation rule runs on the device and
                                the rollback happens when the host learns of
                                it, at the latest at finish; the caller then
                                replays every kernel it ran); the bulk
                                restore on a stream of its own, a kernel
                                waiting for the copier's pieces of the
                                buffers it is speculated to access.  With
                                the copier on its own stream, a buffer
                                counts as restored for the rule once it is
                                present and the caller's stream has waited
                                for its last piece.                          */
    uint64_t chunk;          /* multiple of 256                              */
    const void *image;       /* checkpoint image (pinned host or device)     */
    uint64_t image_bytes;
    uint32_t *d_present;     /* optional device u32[ceil(n/32)] kept in step
                                with the restored set (zeroed by begin)      */
    const uint64_t *d_manifest; /* optional device u64[n], the image's
                                manifest (phos_image_manifest): each buffer
                                is digested on the device as soon as its
                                last byte lands, before any kernel can use
                                it; a mismatch sets PHOS_ECORRUPT, which
                                the next call that synchronises returns
                                (an after_kernel of lockstep rounds, else
                                finish; stats.corrupt_buf names the lowest
                                damaged buffer found).  With a manifest, an
                                image shorter than phos_image_bytes is
                                PHOS_ECORRUPT at begin.                     */
} phos_restore_desc_t;

typedef struct {
    uint64_t kernels;
    uint64_t copier_bytes;   /* background bulk restore                      */
    uint64_t ondemand_bytes; /* copied before a kernel that needed them      */
    uint64_t validated;
    uint64_t violations;
    int64_t misspec_round;
    uint32_t done;           /* every buffer present                         */
    int32_t corrupt_buf;     /* lowest buffer found whose restored bytes
                                did not match the manifest, -1 if none (or
                                no manifest)                                */
} phos_restore_stats_t;

/* Manifest of a checkpoint image: d_digest[i] (device u64[n], overwritten)
 * = the digest of buffer i's bytes in the image (the definition in
 * phos_harness.h), for a later restore to verify against.  image: pinned
 * host (read through its mapped address, one pass over PCIe) or device.
 * PHOS_ECORRUPT if image_bytes is shorter than phos_image_bytes(t).
 * Asynchronous on stream. */
phos_status phos_image_manifest(const phos_table_t *t, const void *image, uint64_t image_bytes,
                                uint64_t *d_digest, phos_stream_t stream);

/* Concurrent restore (Sec. 6): nothing is present at begin. */
phos_status phos_restore_begin(const phos_table_t *t, const phos_restore_desc_t *d,
                               phos_stream_t stream, phos_restore_t **out);
/* Background bulk restore of up to quota bytes, skipping present buffers
 * and never writing one.  *done = 1 once every buffer is present.  Called
 * between rounds (before before_kernel), or, with
 * PHOS_RESTORE_ONDEMAND_FIRST, once inside each round after
 * before_kernel (EINVAL otherwise). */
phos_status phos_restore_advance(phos_restore_t *r, uint64_t quota, int *done);
/* Copy the not-yet-restored bytes of every buffer with perm != 0 before
 * the kernel runs (the kernel waits for them). */
phos_status phos_restore_before_kernel(phos_restore_t *r, const uint8_t *perm);
/* PHOS_CKPT_DEVICE sessions: the round's need set from d_perm (device
 * u8[n]), decided on the device. */
phos_status phos_restore_before_kernel_dev(phos_restore_t *r, const uint8_t *d_perm);
/* Validate; an access (load or store) to a buffer that was not present
 * before the kernel restores every buffer stop-the-world from the image
 * and sets *misspec = 1: the caller replays its kernels from the first
 * (Sec. 6 "roll back ... and perform a stop-the-world restore").
 * Synchronises (PHOS_CKPT_NO_SYNC: enqueues; *misspec = 1 only once the
 * host has seen the device's record; stats.misspec_round >= 0 after
 * finish says a rollback happened). */
phos_status phos_restore_after_kernel(phos_restore_t *r, const uint64_t *d_trace,
                                      uint64_t n_rec, int *misspec);
phos_status phos_restore_finish(phos_restore_t *r);
phos_status phos_restore_stats(const phos_restore_t *r, phos_restore_stats_t *out);
/* kind 0 on-demand: round, buffer, offset, len, 0;
 * kind 1 copier: round, buffer, offset, len, 0 */
phos_status phos_restore_log(const phos_restore_t *r, uint32_t kind, uint64_t *out,
                             uint64_t cap, uint64_t *n_out);
phos_status phos_restore_end(phos_restore_t *r);

#ifdef __cplusplus
}
#endif
#endif /* PHOS_H */
