/*
 * fcc_doa.h -- direction-of-arrival search over candidate directions from the
 * pairs' FCC correlations: the step the paper's conclusion names after
 * per-pair TDoA estimation (use every pair's correlation and search for the
 * best DoA candidate).  The paper prints no formula; this is the steered
 * response power it refers to, read from FCC's lag grid:
 *
 *   tau_ij(u) = -(fs / c) (r_i - r_j) . u      (samples; t_i - t_j for a plane
 *                                               wave arriving from unit vector u)
 *   score(u)  = sum over pairs i < j of y_ij read at tau_ij(u) by linear
 *               interpolation on the grid tau_k = -L + k / den (Sec. 3), the
 *               grid position (tau + L) den clamped to [0, I - 1]
 *   per frame: the candidate with the highest score (lowest index on a tie).
 *
 * The grid positions are computed once, in FP64, when the search object is
 * created; the per-frame work is a gather and a sum per (candidate, pair).
 */
#ifndef FCC_DOA_GB300_H
#define FCC_DOA_GB300_H

#include "fcc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fcc_doa fcc_doa_t;

/*
 * plan: the FCC plan whose lag grid (L, den, I) and fs, c define the search;
 * it is borrowed and must stay alive while the object searches (destroying
 * the object afterwards is safe).  mic_xyz: host [M][3]
 * metres (M = the plan's microphones), copied.  dirs: host [n_dirs][3] unit
 * vectors (used as given), copied; n_dirs >= 1.  Synchronous (uploads a
 * table of P * n_dirs grid positions).
 * Errors: INVALID_ARG (null pointers, n_dirs < 1, non-finite input), OOM, CUDA.
 */
fcc_status_t fcc_doa_create(fcc_plan_t *plan, const double *mic_xyz, const double *dirs, int n_dirs,
                            fcc_doa_t **out);

/* Release a search object (NULL is ignored); safe after its plan was destroyed. */
void fcc_doa_destroy(fcc_doa_t *doa);

/*
 * The search over correlations already on the lag grid.  d_corr: float
 * [T][P][I] (fcc_tdoa's d_corr output layout), 16-byte aligned.  Outputs
 * d_dir_idx int32 [T] (candidate index) and d_score float [T].  Asynchronous
 * on `stream`; a non-finite score latches FCC_ERR_NONFINITE in the plan's
 * device error word (read by fcc_plan_sync) and leaves that frame's outputs
 * unspecified.  T = 0 is a no-op.
 * Errors: INVALID_ARG, CUDA.
 */
fcc_status_t fcc_doa_search(fcc_doa_t *doa, const float *d_corr, long long T, int *d_dir_idx, float *d_score,
                            void *stream);

/* Bytes of device workspace fcc_tdoa_doa needs (independent of T beyond a
 * chunk of frames whose correlations stay in L2).  Errors: INVALID_ARG (null,
 * T < 0). */
fcc_status_t fcc_doa_workspace(const fcc_doa_t *doa, long long T, long long *bytes);

/*
 * Spectra in, DoA out: fcc_tdoa (with the correlation output) then
 * fcc_doa_search, chunk by chunk through d_work (at least fcc_doa_workspace
 * bytes, 16-byte aligned).  d_spectra: complex64 [T][M][N/2+1] as fcc_tdoa.
 * d_lag_idx / d_peak: optional per-pair outputs [T][P] as fcc_tdoa (NULL: not
 * kept).  Asynchronous on `stream`; device conditions go to the plan's error
 * word.  Errors: INVALID_ARG, UNSUPPORTED (as fcc_tdoa), CUDA.
 */
fcc_status_t fcc_tdoa_doa(fcc_doa_t *doa, const void *d_spectra, long long T, int *d_dir_idx, float *d_score,
                          int *d_lag_idx, float *d_peak, void *d_work, long long work_bytes, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FCC_DOA_GB300_H */
