/*
 * fcc_stft.h -- the STFT front-end: multichannel PCM in, the spectra X_m(t, f)
 * the method starts from (Sec. 2) or directly the per-pair TDoA out.
 *
 * The paper does not print the analysis window or framing; this library uses
 * a periodic Hann window w[n] = 0.5 - 0.5 cos(2 pi n / N) and frames of the
 * plan's N samples every `hop` samples with no padding:
 *
 *   T = 1 + (n_samples - N) / hop   (integer division; 0 if n_samples < N)
 *   X[t][m][k] = sum_{n<N} w[n] x[t hop + n][m] exp(-j 2 pi k n / N),  k = 0..N/2
 *
 * PCM is interleaved [n_samples][M] (M = the plan's microphones): float32 used
 * as is, or int16 scaled by 1/32768.  The transform is FP32 (a radix-4
 * Stockham FFT of the N/2 packed even/odd samples per microphone frame, then
 * the split into the N/2 + 1 bins of the real signal).
 */
#ifndef FCC_STFT_GB300_H
#define FCC_STFT_GB300_H

#include "fcc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { FCC_PCM_F32 = 0, FCC_PCM_S16 = 1 } fcc_pcm_t;

/* Frames of a PCM buffer: T as above (0 if n_samples < N).
 * Errors: INVALID_ARG (null, n_samples < 0, hop < 1). */
fcc_status_t fcc_stft_frames(const fcc_plan_t *plan, long long n_samples, int hop, long long *T);

/*
 * d_pcm: device PCM [n_samples][M] of `type` (4-byte aligned for float32,
 * 2-byte for int16).  d_spectra: complex64 [T][M][N/2+1], 8-byte aligned (the
 * layout fcc_tdoa reads).  Asynchronous on `stream`.
 * Errors: INVALID_ARG, UNSUPPORTED (N outside 64..2048), CUDA.
 */
fcc_status_t fcc_stft(fcc_plan_t *plan, const void *d_pcm, fcc_pcm_t type, long long n_samples, int hop,
                      void *d_spectra, void *stream);

/* Bytes of device workspace recommended for fcc_tdoa_pcm: one chunk of spectra.
 * fcc_tdoa_pcm accepts any workspace of at least one frame of spectra (M (N/2+1)
 * 8 bytes) and processes the frames in chunks of as many as it holds.
 * Errors: INVALID_ARG (null, n_samples < 0, hop < 1). */
fcc_status_t fcc_pcm_workspace(const fcc_plan_t *plan, long long n_samples, int hop, long long *bytes);

/*
 * PCM in, TDoA out: fcc_stft then fcc_tdoa chunk by chunk through d_work
 * (16-byte aligned, at least one frame of spectra; the recommended size is
 * fcc_pcm_workspace), the spectra of a chunk going from one kernel to the next.
 * Outputs as fcc_tdoa ([T][P]; d_tau_hat may be NULL).  Asynchronous on
 * `stream`; device conditions (NaN / Inf samples) go to the plan's error word
 * (fcc_plan_sync).
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA.
 */
fcc_status_t fcc_tdoa_pcm(fcc_plan_t *plan, const void *d_pcm, fcc_pcm_t type, long long n_samples, int hop,
                          int *d_lag_idx, float *d_peak, float *d_tau_hat, void *d_work, long long work_bytes,
                          void *stream);

/*
 * The same from host buffers: PCM chunks are copied to the device (page-locked
 * host memory gives full link speed), transformed and estimated there, and the
 * results copied back, with copies and compute overlapped.  Synchronous: reads
 * the error word at the end like fcc_plan_sync.
 * Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA, NONFINITE, TIMEOUT.
 */
fcc_status_t fcc_tdoa_pcm_host(fcc_plan_t *plan, const void *h_pcm, fcc_pcm_t type, long long n_samples, int hop,
                               int *h_lag_idx, float *h_peak, float *h_tau_hat, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FCC_STFT_GB300_H */
