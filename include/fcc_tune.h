/*
 * fcc_tune.h -- tile-shape autotuner of the FP32 FCC kernel.
 *
 * The FP32 kernel's launch geometry (chunks of the bin-pair axis per pair
 * block, warps per group, groups per CTA, frames per stage and the depth of the
 * shared-memory ring) is chosen per plan by a heuristic at fcc_plan_create.
 * The autotuner times the best-scored candidates on the plan's own device, on
 * synthetic spectra larger than L2, and keeps the fastest; results are cached
 * in a JSON file keyed by device name, SM count, M, N, K_even + K_odd and I, so
 * a second plan with the same key (or a later process) skips the timing.  The
 * geometry changes only the order of the FP32 additions, never what is
 * computed (Sec. 3, Eqs. 7-9).
 */
#ifndef FCC_TUNE_GB300_H
#define FCC_TUNE_GB300_H

#include "fcc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Launch geometry of a plan's FP32 kernel. */
typedef struct {
    int C;            /* chunks of the bin-pair axis per 2x2 pair block */
    int warps_per_group;
    int groups;       /* groups per CTA, each with its own part of the ring */
    int frames_per_stage;
    int stages;       /* ring depth (a multiple of groups) */
    int threads;      /* threads per CTA of the single-plan launch */
    long long smem_bytes;
} fcc_geometry_t;

/* The plan's current FP32 geometry (all zero when N > 1024: no FP32 kernel).
 * Errors: INVALID_ARG (NULL). */
fcc_status_t fcc_plan_geometry(const fcc_plan_t *plan, fcc_geometry_t *out);

/*
 * Pick the plan's FP32 geometry by timing.  cache_path: JSON cache file (NULL:
 * the FCC_TUNE_CACHE environment variable, else no cache).  force != 0 times
 * the candidates even when the cache holds the key.  max_candidates <= 0 means
 * 8.  us_per_frame (may be NULL) receives the winner's time per frame in
 * microseconds (from the cache on a hit).  Synchronous; allocates about 256 MB
 * of device memory while timing and frees it before returning.  The plan must
 * not be in use on any stream.  FP32 plans only.
 * Errors: INVALID_ARG, UNSUPPORTED (no FP32 kernel for this plan), OOM, CUDA.
 */
fcc_status_t fcc_plan_autotune(fcc_plan_t *plan, const char *cache_path, int force, int max_candidates,
                               double *us_per_frame);

#ifdef __cplusplus
}
#endif
#endif /* FCC_TUNE_GB300_H */
