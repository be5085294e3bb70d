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
// Resolve an image pointer to a device-accessible address (pinned host ->
// mapped device pointer; device -> itself).  EINVAL for pageable memory.
phos_status device_view(const void *p, void **out);
}  // namespace phos
