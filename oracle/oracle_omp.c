/*
 * All-core timing driver of the CPU oracle -- TEST AND BASELINE
 * INFRASTRUCTURE ONLY (the benchmark's CPU-baseline leg).
 *
 * The oracle's own functions stay single-threaded and plain; this file
 * only runs them on several host threads at once, on independent parts of
 * the work, so that the baseline can state what the oracle does on all of
 * a host's cores:
 *   orc_validate_omp  the trace cut into contiguous ranges of whole 32-record
 *                     bitmap words, each range validated by orc_validate
 *                     (phos_oracle.c) into its own counts and victim
 *                     bitmaps, which are then summed and OR-ed
 *   orc_memcpy_omp    a byte copy cut into contiguous ranges, one memcpy each
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC -o liboracle_omp.so oracle_omp.c phos_oracle.c
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

int orc_validate(const uint64_t *base, const uint64_t *size, const uint8_t *perm,
                 uint32_t n, const uint64_t *trace, uint64_t nrec, uint32_t w,
                 uint32_t *bitmap, uint64_t *count, uint32_t *victim,
                 uint32_t *victim_st, uint64_t *idx, uint64_t idx_cap);

int orc_threads(void) { return omp_get_max_threads(); }

int orc_validate_omp(const uint64_t *base, const uint64_t *size, const uint8_t *perm,
                     uint32_t n, const uint64_t *trace, uint64_t nrec, uint32_t w,
                     uint32_t *bitmap, uint64_t *count, uint32_t *victim,
                     uint32_t *victim_st) {
    const uint64_t nwords = (nrec + 31) / 32;
    const uint32_t nv = (n + 31) / 32;
    int malformed = 0;
    count[0] = count[1] = count[2] = 0;
    memset(victim, 0, (size_t)nv * 4);
    memset(victim_st, 0, (size_t)nv * 4);
#pragma omp parallel reduction(| : malformed)
    {
        const uint64_t T = (uint64_t)omp_get_num_threads(), t = (uint64_t)omp_get_thread_num();
        const uint64_t w0 = nwords * t / T, w1 = nwords * (t + 1) / T;
        const uint64_t r0 = w0 * 32, r1 = w1 * 32 < nrec ? w1 * 32 : nrec;
        uint64_t c[3] = {0, 0, 0};
        uint32_t *v = calloc(nv ? nv : 1, 4), *vs = calloc(nv ? nv : 1, 4);
        if (r1 > r0)
            malformed |= orc_validate(base, size, perm, n, trace + r0, r1 - r0, w,
                                      bitmap + w0, c, v, vs, NULL, 0);
#pragma omp critical
        {
            count[0] += c[0];
            count[1] += c[1];
            count[2] += c[2];
            for (uint32_t q = 0; q < nv; q++) {
                victim[q] |= v[q];
                victim_st[q] |= vs[q];
            }
        }
        free(v);
        free(vs);
    }
    return malformed;
}

void orc_memcpy_omp(uint8_t *dst, const uint8_t *src, uint64_t len) {
#pragma omp parallel
    {
        const uint64_t T = (uint64_t)omp_get_num_threads(), t = (uint64_t)omp_get_thread_num();
        const uint64_t a = len * t / T, b = len * (t + 1) / T;
        if (b > a) memcpy(dst + a, src + a, b - a);
    }
}
