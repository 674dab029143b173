/*
 * fcc_smooth.h -- FCC with the recursive cross-spectrum of Sec. 2, Eq. 1:
 *   R(t,f) = (1 - alpha) R(t-1,f) + alpha X_i(t,f) X_j(t,f)^*,   R_hat = R / |R|,
 * for a smoothing factor alpha in (0, 1] (the paper's experiments use 0.1),
 * followed by the same fold, projection, lag-grid reconstruction, argmax and
 * refinement as fcc_tdoa (Secs. 2-3, Eqs. 7-9).  alpha = 1 is fcc_tdoa's input.
 *
 * The recursion runs over the frames of the call in order, from a caller-held
 * state R(0) (the cross-spectrum before the first frame: zero for a fresh
 * stream), and leaves R(T) in the same buffer, so consecutive calls continue one
 * stream.  It is solved exactly (up to FP32 rounding) in three passes over
 * chunks of frames: the recursion from zero inside each chunk, a carry scan
 * over the chunks, and the FCC pass that restarts every chunk from its carry.
 *
 * Supported plans: FP32, an even number of microphones up to 8, 128 <= N <= 512,
 * either form (FCC_FORM_REIM_SPLIT plans project R_hat on their cosine and sine
 * bases instead of folding it, and take no d_coeffs).
 */
#ifndef FCC_SMOOTH_GB300_H
#define FCC_SMOOTH_GB300_H

#include "fcc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Bytes of device workspace fcc_tdoa_smoothed needs for T frames of this plan.
 * Errors: INVALID_ARG, UNSUPPORTED (plan not supported). */
fcc_status_t fcc_smooth_workspace(const fcc_plan_t *plan, long long T, long long *bytes);

/*
 * d_spectra: complex64 [T][M][N/2+1], 16-byte aligned.  d_state: complex64
 * [P][N/2+1] (pairs i < j lexicographic, bins 0..N/2): R(0) on entry, R(T) on
 * return; NULL = a fresh stream whose final state is not kept.  d_work: device
 * workspace of at least fcc_smooth_workspace bytes.  Outputs as fcc_tdoa
 * (d_tau_hat, d_coeffs and d_corr may be NULL; d_corr receives y(tau_i) of
 * every pair-frame, float [T][P][I]).  Asynchronous on `stream`; the device
 * error word (NaN / Inf input, a wait that ran out) is read by fcc_plan_sync.
 * Errors: INVALID_ARG (alpha outside (0, 1], pointers, workspace too small),
 * UNSUPPORTED, CUDA.
 */
fcc_status_t fcc_tdoa_smoothed(fcc_plan_t *plan, const void *d_spectra, long long T, double alpha, void *d_state,
                               void *d_work, long long work_bytes, int *d_lag_idx, float *d_peak, float *d_tau_hat,
                               float *d_coeffs, float *d_corr, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FCC_SMOOTH_GB300_H */
