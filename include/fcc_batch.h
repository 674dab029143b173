/*
 * fcc_batch.h -- batched FCC: many independent microphone arrays, each with its
 * own geometry, frame size, sampling rate, lag grid and rank, in persistent
 * launches captured in one CUDA graph.
 *
 * Every array is an FP32 plan (fcc.h) evaluated exactly as fcc_tdoa does
 * (Sec. 2-3: per-microphone PHAT, cross-spectrum, fold, even/odd projection,
 * reconstruction on the lag grid, argmax, parabolic refinement); results are
 * identical, bit for bit, to fcc_tdoa on the same plan geometry.  Plans that
 * share (N, lag grid, K rule) share one basis construction.  Arrays are grouped
 * by kernel class (basis count per parity rounded up to 2/4/6/8, and N); each
 * class is one persistent launch whose CTAs take jobs (a run of one array's
 * frame tiles) from a counter, largest first.  The classes are independent
 * branches of the graph, so a class's tail overlaps the next class's start.
 *
 * Lifecycle: fcc_batch_create (plans, optional autotuning) -> fcc_batch_bind
 * (device buffers; builds the graph) -> fcc_batch_run (any number of times;
 * asynchronous) -> fcc_batch_sync (error word) -> fcc_batch_destroy.
 */
#ifndef FCC_BATCH_GB300_H
#define FCC_BATCH_GB300_H

#include "fcc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fcc_batch fcc_batch_t;

enum {
    FCC_BATCH_AUTOTUNE = 1,     /* time the tile shapes of every distinct (M, N, K, I) (see fcc_tune.h) */
    FCC_BATCH_SINGLE_LAUNCH = 2 /* the whole batch as one persistent launch instead of one per kernel class */
};

typedef struct {
    int n_arrays;
    int n_classes;       /* kernel classes (KH bases per parity, RS fold records per lane) among the arrays */
    int n_jobs;
    int n_bases;         /* distinct basis constructions (N, lag grid, K rule) */
    long long frames;    /* sum of T */
    long long pair_frames;
    double spectra_bytes; /* sum of T * M * (N/2+1) * 8: the bytes one run must read */
    double result_bytes;  /* sum of T * P * 8 (lag index + peak), plus 4 per pair-frame with tau_hat */
    int n_launches;       /* persistent kernel launches in the graph: n_classes, or 1 with FCC_BATCH_SINGLE_LAUNCH */
} fcc_batch_info_t;

/*
 * Create plans for n_arrays arrays (descs[a].prec must be FCC_PREC_FP32; the
 * device field of every desc is ignored: all plans live on `device`, -1 =
 * current) with T[a] >= 1 frames each.  flags: FCC_BATCH_AUTOTUNE,
 * FCC_BATCH_SINGLE_LAUNCH.  By default the arrays are grouped into kernel classes
 * (KH bases per parity, RS fold records per lane) and each class is one
 * persistent launch with its own warp count and register budget, the classes
 * being independent branches of one CUDA graph.  With FCC_BATCH_SINGLE_LAUNCH the
 * whole batch is one persistent launch: its CTAs take (array, tile run) jobs of
 * every array from one queue, largest first, and every array's tile geometry is
 * limited to that kernel's eight compute warps (keeping the chunk count of the
 * plan's own geometry).  Either way each array's results equal fcc_tdoa's on a
 * plan of the same geometry bit for bit.  tune_cache:
 * as fcc_plan_autotune (NULL: FCC_TUNE_CACHE or none).  Synchronous.
 * Errors: INVALID_ARG (the message names the array), UNSUPPORTED, OOM, CUDA,
 * NOT_CONVERGED.
 */
fcc_status_t fcc_batch_create(const fcc_plan_desc_t *descs, const long long *T, int n_arrays, int device,
                              int flags, const char *tune_cache, fcc_batch_t **out);

/* Synchronise the device and free the batch, its plans and its graph. */
void fcc_batch_destroy(fcc_batch_t *batch);

/* The batch's totals and classes into *info.  Errors: INVALID_ARG (NULL). */
fcc_status_t fcc_batch_info(const fcc_batch_t *batch, fcc_batch_info_t *info);

/* Sizes of array a's plan (P, I, K, ... as fcc_plan_info).
 * Errors: INVALID_ARG (NULL, a out of range). */
fcc_status_t fcc_batch_array_info(const fcc_batch_t *batch, int a, fcc_plan_info_t *info);

/*
 * Bind device buffers: host arrays of n_arrays device pointers each.
 * d_spectra[a]: complex64 [T[a]][M][N/2+1], 16-byte aligned; d_lag_idx[a],
 * d_peak[a]: [T[a]][P]; d_tau_hat: NULL (no refinement output) or an array
 * whose entries may be NULL.  Uploads the job tables and captures the graph.
 * Synchronous; no run may be in flight.  Errors: INVALID_ARG, CUDA, OOM.
 */
fcc_status_t fcc_batch_bind(fcc_batch_t *batch, const void *const *d_spectra, int *const *d_lag_idx,
                            float *const *d_peak, float *const *d_tau_hat);

/* Launch the bound graph on `stream` (asynchronous).  Errors: INVALID_ARG (not bound), CUDA. */
fcc_status_t fcc_batch_run(fcc_batch_t *batch, void *stream);

/* Synchronise `stream`, then read and clear the batch's device error word
 * (FCC_OK, FCC_ERR_NONFINITE or FCC_ERR_TIMEOUT).  Errors: INVALID_ARG (NULL), CUDA. */
fcc_status_t fcc_batch_sync(fcc_batch_t *batch, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FCC_BATCH_GB300_H */
