// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/phos.h"

namespace phos {

// ---------------------------------------------------------------- errors
phos_status fail(phos_status code, const char *fmt, ...);
phos_status cuda_fail(cudaError_t e, const char *what);

#define PHOS_CUDA(call)                                          \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return phos::cuda_fail(e_, #call); \
    } while (0)

inline uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// Count kernel launches (phos_launch_count).
void count_launch(uint32_t k = 1);

// Device-side status word: first error sticks.
__device__ __forceinline__ void set_status(uint32_t *st, uint32_t code) {
    if (st) atomicCAS(st, 0u, code);
}

// ------------------------------------------------------------ scratch
// A growable device allocation owned by a handle.  Growth synchronises the
// device (cudaMalloc); size it before graph capture.
struct Scratch {
    void *ptr = nullptr;
    size_t bytes = 0;
    phos_status reserve(size_t need);
    ~Scratch();
};

// Device-resident view of the buffer table used by the kernels.
struct TableDev {
    const uint64_t *base;    // [n]
    const uint64_t *size;    // [n]
    const uint64_t *fence1;  // base[32 j],   j < ceil(n / 32)
    const uint64_t *fence2;  // base[1024 j], j < ceil(n / 1024)
    uint32_t n;
};

constexpr uint32_t kMaxTable = 32768;  // three-level warp search limit

// The protocol's response to one validation, applied by the validation
// kernel's last CTA (no-sync sessions): kind 1 recopy (store victims with
// flags[i] set become dirty[i] = 1), 2 CoW (a store victim with flags[i]
// clear is a mis-speculation), 3 restore (a victim of any access with
// flags[i] clear is one).  acc: u64[8] device words, [3] += violations,
// [4] = first mis-speculated round (-1 = none), also published to the
// mapped host word h_flag.  kind 0: no rule.
struct ProtoRule {
    const uint8_t *flags;
    uint8_t *dirty;
    uint64_t *acc;
    int64_t *h_flag;
    int64_t round;
    uint32_t kind;
};

// phos_validate with an optional ProtoRule; *rule_fused = true when the
// launched kernel applies it (otherwise the caller must).
phos_status validate_impl(const phos_table_t *t, const uint8_t *d_perm, const uint64_t *d_trace,
                          uint64_t n_rec, uint32_t access_bytes, uint32_t *d_bitmap,
                          uint64_t *d_count, uint32_t *d_victim, uint32_t *d_victim_st,
                          uint64_t *d_idx, uint64_t idx_cap, uint32_t *d_status,
                          phos_stream_t stream, const ProtoRule *rule, bool *rule_fused);

// Several rounds' validation in one launch (deferred no-sync sessions):
// round i's trace checked against its own perm, its rule answered with its
// own flags (rule kind as in ProtoRule; dirty, acc and h_flag as there).
constexpr uint32_t kMaxRounds = 16;
struct RoundSeg {
    const uint64_t *trace;
    uint64_t n_rec;
    const uint8_t *perm;
    const uint8_t *flags;
    int64_t round;
};
// Rounds one launch can take for a table of n buffers (0: none fit).
uint32_t rounds_cap(uint32_t n, int device);
// Bytes of zeroed device scratch a launch of up to k rounds needs (the
// kernel leaves it zeroed).
size_t rounds_scratch_bytes(uint32_t n, uint32_t k);
phos_status validate_rounds(const phos_table_t *t, const RoundSeg *seg, uint32_t k,
                            uint32_t access_bytes, uint32_t rule, uint8_t *d_dirty,
                            uint64_t *d_acc, int64_t *d_flag, uint32_t *d_status,
                            void *d_scratch, cudaStream_t s);

}  // namespace phos

struct phos_table;
namespace phos {
// Digest buffers bufs of live memory on the device and compare each with
// d_manifest[buf] (PHOS_ECORRUPT in d_status and the lowest bad index in
// *d_bad on a mismatch).  d_acc (u64[n]) and d_cnt (u32[n]) start zeroed
// and are left zeroed.  Asynchronous on s.
// Bytes of copy-engine scratch for a launch of n descriptors.
size_t copy_scratch_bytes(uint32_t n);
// Descriptors a table's copy scratch holds from creation on (a larger
// launch grows it, which synchronises the device).
constexpr uint32_t kCopyReserve = 1024;
// phos_copy whose descriptor count is read on the device (*d_n, at most
// cap): lists built by device-side decisions.
phos_status copy_device_count(const phos_table_t *t, const phos_copy_t *d_list, uint32_t cap,
                              const uint32_t *d_n, void *staging, uint64_t staging_bytes,
                              const void *image, uint64_t image_bytes, uint32_t *d_present,
                              uint32_t *d_status, phos_stream_t stream);
// Upload bytes from pinned host memory to device memory on s without the
// copy engines: up to 32 KB as kernel parameters (copied from h_src at the
// call), more by SM loads through h_src_dev (h_src's device-mapped
// address, which must stay unchanged until the upload has run).
phos_status push_small(void *d_dst, const void *h_src, const void *h_src_dev, uint64_t bytes,
                       cudaStream_t s);
phos_status verify_buffers(const phos_table *t, const std::vector<uint32_t> &bufs,
                           const uint64_t *d_manifest, unsigned long long *d_acc,
                           uint32_t *d_cnt, uint32_t *d_status, int *d_bad, cudaStream_t s);
// Device-decided protocol rounds (csrc/devround.cu): the copier's pieces
// and the CoW set / restore need set computed on the device each round.
struct DevRounds {
    const phos_table *t = nullptr;
    uint32_t mode = 0;            // 1 restore, 2 CoW
    void *mem = nullptr;          // every device array, one allocation
    uint32_t cap_c = 0;
    uint64_t cap_lc = 0;
    alignas(16) unsigned char dev[256];  // the kernels' view of the state
    phos_status init(const phos_table *t, uint32_t mode, uint64_t chunk,
                     uint64_t staging_bytes, bool mark_present, cudaStream_t s);
    // enqueue the copier's move of one round (k_dr_copier + copy engine)
    phos_status copier(uint64_t quota, uint64_t round, void *staging, uint64_t staging_bytes,
                       const void *image, uint64_t image_bytes, uint32_t *d_present,
                       uint32_t *d_status, cudaStream_t s);
    // enqueue the round's need set (restore) or CoW set (CoW) and its copies
    phos_status action(const uint8_t *d_perm, uint64_t round, void *staging,
                       uint64_t staging_bytes, const void *image, uint64_t image_bytes,
                       uint32_t *d_present, uint32_t *d_status, cudaStream_t s);
    // every buffer restored / done (after a stop-the-world fallback)
    phos_status mark_all(cudaStream_t s);
    const uint8_t *flags() const;
    // after a synchronisation: the logs (5 u64 per row) and counters
    // out[0..5] = copier rows, action rows, copier bytes, CoW bytes, direct
    // bytes, on-demand bytes
    phos_status collect(std::vector<uint64_t> &copier_log, std::vector<uint64_t> &act_log,
                        uint64_t out[6], std::vector<uint8_t> *state);
    ~DevRounds();
};

}  // namespace phos

struct phos_table {
    int device = 0;
    uint32_t n = 0;
    std::vector<uint64_t> base, size, img_off;
    uint64_t image_bytes = 0;
    void *dev = nullptr;         // one allocation: base | size | fence1 | fence2
    phos::TableDev view{};
    std::mutex mu;               // guards scratch growth
    phos::Scratch val_scratch;   // validate: per-CTA counts, victim acc, ticket
    phos::Scratch copy_scratch;  // copy engine: prefix, resolved descriptors
    phos::Scratch harness_scratch;
};

namespace phos {
// device SM count (cached per device)
int sm_count(int device);
// Opt kernel fn in to 227 KB of dynamic shared memory on the current device
// (once per kernel and device; thread-safe).
phos_status smem_optin_once(const void *fn);
// Resolve an image pointer to a device-accessible address (pinned host ->
// mapped device pointer; device -> itself).  EINVAL for pageable memory.
phos_status device_view(const void *p, void **out);
}  // namespace phos
