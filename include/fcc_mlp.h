/*
 * fcc_mlp.h -- C ABI of the learned TDoA head on the FCC projection coefficients.
 *
 * The paper's method stops at the argmax of the reconstructed correlation
 * (Sec. 3, Eq. 10-11).  This head is an extension: a small network that maps a
 * pair-frame's 2K projection coefficients z = (z_e, z_o) (the Sec. 3 outputs of
 * fcc_tdoa's `d_coeffs`, each scaled by its own factor) to a sub-sample TDoA and a
 * confidence logit, trained against the true delay.
 *
 * Network (fixed): x_k = in_scale_k * z_k (n_in = 2K <= 32 inputs),
 *   h1 = GELU(W1 x + b1), h2 = GELU(W2 h1 + b2), (y0, y1) = W3 h2 + b3,
 * hidden width 128, GELU with the exact erf.  Parameters are one FP32 vector
 * packed as W1[128][n_in], b1[128], W2[128][128], b2[128], W3[2][128], b3[2]
 * (row-major, output index first).  The forward and backward use BF16 copies of
 * W1, W2, W3 (round to nearest even from the FP32 masters) with FP32 biases,
 * FP32 arithmetic and FP32 accumulation; Adam updates the FP32 masters and
 * refreshes the BF16 copies.
 *
 * Loss over a batch of n samples with true delay t and plain FCC estimate t_fcc
 * (both in samples, the same unit as y0):
 *   mean_s [ (y0 - t)^2 + conf_weight * BCE(sigmoid(y1), g) ],
 *   g = 1 if |y0 - t| <= |t_fcc - t| else 0,
 * so the confidence learns where the network beats the argmax + parabola.
 * Inference returns y0 where sigmoid(y1) >= threshold and t_fcc elsewhere.
 *
 * All device pointers are caller-owned device memory on the head's device;
 * launches are asynchronous on `stream` (a cudaStream_t, NULL = legacy default).
 */
#ifndef FCC_MLP_GB300_H
#define FCC_MLP_GB300_H

#include "fcc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fcc_mlp fcc_mlp_t;

/* Number of parameters: hidden*n_in + hidden + hidden^2 + hidden + 2*hidden + 2. */
long long fcc_mlp_num_params(int n_in, int hidden);

/*
 * Create a head on `device` (-1 = current) from host FP32 parameters
 * `h_params[fcc_mlp_num_params(n_in, hidden)]` and input scales
 * `h_in_scale[n_in]` (NULL = all 1), both copied.  Adam moments start at
 * zero, step count 0.  hidden must be 128 and 1 <= n_in <= 32
 * (FCC_ERR_UNSUPPORTED otherwise); conf_weight >= 0.  Synchronous.
 * Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA.
 */
fcc_status_t fcc_mlp_create(int n_in, int hidden, const float *h_in_scale, double conf_weight,
                            const float *h_params, int device, fcc_mlp_t **out);

/* Synchronise the device and free the head (NULL is a no-op). */
void fcc_mlp_destroy(fcc_mlp_t *mlp);

/*
 * Copy the FP32 master parameters and the Adam moments (each may be NULL) to
 * host arrays of fcc_mlp_num_params floats, and the step count.  Synchronous
 * (checkpoint).  Errors: INVALID_ARG, CUDA.
 */
fcc_status_t fcc_mlp_get_state(const fcc_mlp_t *mlp, float *params, float *m, float *v, long long *step);

/*
 * Replace the parameters (required), the moments (NULL = zero) and the step
 * count (>= 0) from host arrays, refreshing the BF16 copies.  Synchronous
 * (resume).  Errors: INVALID_ARG, CUDA.
 */
fcc_status_t fcc_mlp_set_state(fcc_mlp_t *mlp, const float *params, const float *m, const float *v,
                               long long step);

/*
 * Gradient of the batch loss with respect to the packed parameters (evaluated
 * with the BF16 weight copies), written to d_grad[num_params]; the mean loss to
 * d_loss[0] if d_loss is not NULL.  d_features[n][n_in] row-major,
 * d_tau_true[n], d_tau_fcc[n].  The per-block partial sums are reduced in a fixed
 * order, so the result is the same bit for bit on every call.  Calls on one head
 * share its workspace: serialise them.  Errors: INVALID_ARG (n <= 0), CUDA.
 */
fcc_status_t fcc_mlp_gradient(fcc_mlp_t *mlp, const float *d_features, const float *d_tau_true,
                              const float *d_tau_fcc, long long n, float *d_grad, float *d_loss,
                              void *stream);

/*
 * One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected, learning
 * rate lr > 0) on the gradient of the batch loss; mean loss before the update to
 * d_loss[0] if not NULL.  Errors: INVALID_ARG, CUDA.
 */
fcc_status_t fcc_mlp_train_step(fcc_mlp_t *mlp, const float *d_features, const float *d_tau_true,
                                const float *d_tau_fcc, long long n, float lr, float *d_loss,
                                void *stream);

/*
 * Forward on the tensor cores (tcgen05, BF16 weights, activations entered as a
 * two-term BF16 split, FP32 accumulation in tensor memory) with the confidence
 * gate: d_tau[s] = y0 if sigmoid(y1) >= threshold,
 * else d_tau_fcc[s] (d_tau_fcc NULL: always y0).  d_conf[s] = sigmoid(y1) and
 * d_raw[s] = y0 are written when not NULL.  n = 0 is a no-op (any pointers).
 * Errors: INVALID_ARG, CUDA.
 */
fcc_status_t fcc_mlp_infer(fcc_mlp_t *mlp, const float *d_features, const float *d_tau_fcc, long long n,
                           float threshold, float *d_tau, float *d_conf, float *d_raw, void *stream);

/*
 * FCC followed by the learned head on every pair-frame: fcc_tdoa(plan, ...)
 * with the refinement and coefficient outputs on, then the gated inference on
 * the [T * P] coefficient rows with the refined FCC estimate as the fallback.
 * Requires n_in == 2K of the plan (and a head trained on the plan's grid).
 * d_coeffs: caller workspace float [T][P][2K]; d_lag_idx, d_peak, d_tau_fcc:
 * the plain FCC outputs [T][P]; d_tau: the gated TDoA [T][P]; d_conf may be
 * NULL.  Two launches on `stream`, asynchronous.
 * Errors: INVALID_ARG (sizes, pointers), UNSUPPORTED, CUDA.
 */
fcc_status_t fcc_tdoa_learned(fcc_plan_t *plan, fcc_mlp_t *mlp, const void *d_spectra, long long T,
                              float threshold, int *d_lag_idx, float *d_peak, float *d_tau_fcc,
                              float *d_coeffs, float *d_tau, float *d_conf, void *stream);

/* Synchronise `stream`, then read and clear the head's device error word
 * (FCC_OK or FCC_ERR_TIMEOUT from a bounded wait of the inference kernel).
 * Errors: INVALID_ARG (NULL), CUDA. */
fcc_status_t fcc_mlp_sync(fcc_mlp_t *mlp, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FCC_MLP_GB300_H */
