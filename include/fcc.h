/*
 * fcc.h -- C ABI of the GB300 (sm_103a) Fast Cross-Correlation TDoA library.
 *
 * Method: Grondin, Maheux, Lauzon, Vincent, Michaud, "Fast Cross-Correlation
 * for TDoA Estimation on Small Aperture Microphone Arrays".  For every STFT
 * frame t and every microphone pair (i, j), i < j, the library computes
 *
 *   R_hat(f) = X_i(f) X_j(f)^* / |X_i(f) X_j(f)^*|          (Sec. 2, eq. 1, alpha = 1)
 *   y(tau)   = 2 Re{ W_K x }                                 (Eq. 4 with rank-K W, Sec. 4)
 *            evaluated through the folded even/odd bases     (Eqs. 6-9)
 *   tau*     = argmax over the lag grid, plus a quadratic refinement (Sec. 2)
 *
 * Conventions used by every entry point:
 *   - Spectra are complex64 (interleaved float re, im), layout [T][M][B] with
 *     B = N/2 + 1 bins, C order, frame-major.  Device pointers must be 16-byte
 *     aligned.
 *   - Pairs p = 0..P-1, P = M(M-1)/2, enumerate (i, j), i < j, in
 *     lexicographic order.
 *   - The lag grid is tau_i = -L + i/den, i = 0..I-1, I = 2 L den + 1 (Sec. 3;
 *     the paper's "I = 4 ceil(tau_max) + 1" is the den = 2 case).
 *   - TDoA sign: tau_ij = t_i - t_j in samples, i.e. positive when mic i hears
 *     the source later than mic j (with R = X_i X_j^* the correlation peaks at
 *     delta_i - delta_j).
 *   - Ties in the argmax go to the lowest lag index.
 *   - The caller owns every input and output buffer.  A plan owns its bases
 *     and its small device workspace; it is used by one stream at a time.
 *   - Asynchronous entry points enqueue on the caller's cudaStream_t (passed as
 *     void*, NULL = legacy default stream) and return without synchronising.
 *     Argument errors are returned at once; conditions found on the device
 *     (non-finite input, a bounded wait that expired) are latched in the plan's
 *     device error word and reported by fcc_plan_sync().
 *   - No C++ exception crosses this ABI.
 */
#ifndef FCC_GB300_H
#define FCC_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FCC_OK = 0,
    FCC_ERR_INVALID_ARG = 1,   /* a null/misaligned pointer or an out-of-range size */
    FCC_ERR_UNSUPPORTED = 2,   /* valid request the library does not handle (e.g. M > 16) */
    FCC_ERR_OOM = 3,           /* a device or pinned-host allocation failed */
    FCC_ERR_CUDA = 4,          /* a CUDA runtime / cuFFT call failed (see fcc_last_error) */
    FCC_ERR_TIMEOUT = 5,       /* a bounded device-side wait expired */
    FCC_ERR_NONFINITE = 6,     /* NaN or Inf in the input spectra (outputs unspecified) */
    FCC_ERR_NOT_CONVERGED = 7  /* the FP64 Jacobi SVD of the plan did not converge */
} fcc_status_t;

typedef enum {
    FCC_PREC_FP32 = 0,  /* FP32 throughout (CUDA-core FFMA path) */
    FCC_PREC_BF16 = 1,  /* projection operands in BF16, FP32 accumulation (tensor cores) */
    FCC_PREC_FP16 = 2   /* projection operands in FP16, FP32 accumulation (tensor cores) */
} fcc_prec_t;

/*
 * Which kernel a plan runs fcc_tdoa on.  AUTO picks the fastest measured one:
 * the CUDA-core kernel for FP32 plans and the shared-memory tensor-core kernel
 * for BF16 / FP16 plans.
 *   CUDA_CORES   the Eq. 9 projection in packed FP32 FMAs (FP32 plans only).
 *   TENSOR_TMEM  the Eq. 9 projection as tcgen05 MMAs whose A operand (the
 *                cross spectra) is written straight into tensor memory; FP32
 *                plans use TF32 with a two-term split of both operands, BF16 /
 *                FP16 plans one rounding of the cross spectra.  Folded plans
 *                with an even number of mics and 128 <= N <= 1024.
 *   TENSOR_SMEM  the 16-bit forms with the A operand staged in shared memory
 *                (BF16 / FP16 plans only).
 */
typedef enum {
    FCC_ENGINE_AUTO = 0,
    FCC_ENGINE_CUDA_CORES = 1,
    FCC_ENGINE_TENSOR_TMEM = 2,
    FCC_ENGINE_TENSOR_SMEM = 3
} fcc_engine_t;

typedef enum {
    FCC_FORM_FOLDED = 0,     /* the paper's even/odd bases on the folded x_s, x_d (Eqs. 6-9) */
    FCC_FORM_REIM_SPLIT = 1  /* cosine bases on Re x and sine bases on Im x: C = Re W and
                                S = Im W (Eq. 3) truncated by their own SVDs; y = 2 (C_K Re x - S_K Im x) */
} fcc_form_t;

/*
 * Plan description (Sec. 3 grid, Sec. 4 rank).  All fields are copied.
 *   n_mics   M, 2 <= M <= 16.
 *   mic_xyz  host [M][3] positions in metres; read only when tau_max <= 0,
 *            to derive L = ceil(max pair distance * fs / c).
 *   fs       sample rate in Hz (> 0).
 *   N        frame size, a power of two, 16 <= N <= 4096.
 *   c        speed of sound in m/s; <= 0 selects 343.
 *   tau_max  lag half-range in samples; L = ceil(tau_max); <= 0: from geometry.
 *   lag_den  grid step 1/lag_den samples, 1 <= lag_den <= 64.
 *   K        rank; 0 selects the energy rule below.
 *   energy   fraction of ||W||_F^2 the kept singular values must hold
 *            (<= 0 selects 0.999); singular values tied with the last kept one
 *            are kept too.
 *   prec     an fcc_prec_t.
 *   device   CUDA device ordinal; < 0 uses the calling thread's current device.
 *   form     an fcc_form_t (0, the default, is the paper's folded form).  The
 *            split form is FP32 only (max(K_c, K_s) <= 16): fcc_tdoa runs it on
 *            the FP32 tile kernel (N <= 1024, with the correlation output but
 *            no coefficient output), fcc_tdoa_smoothed on the per-pair kernel
 *            of fcc_smooth.h (an even number of mics up to 8,
 *            128 <= N <= 512); the autotuner and the batched form take folded
 *            plans only.  Its info reports K_even = K_c (cosine bases) and
 *            K_odd = K_s (sine bases), each chosen by the energy rule on its
 *            own matrix (or both = K when K > 0).
 */
typedef struct {
    int n_mics;
    const double *mic_xyz;
    double fs;
    int N;
    double c;
    double tau_max;
    int lag_den;
    int K;
    double energy;
    int prec;
    int device;
    int form;
} fcc_plan_desc_t;

/* Sizes of a plan; K = K_even + K_odd (even/odd bases of Eq. 6). */
typedef struct {
    int M, P, N, B, Q;      /* Q = N/4: the cropped basis length is Q+1 (Eq. 7) */
    int L, den, I, center;  /* center = L*den, the index of tau = 0 */
    int K, K_even, K_odd;
    int prec;
    double delta;           /* grid step 1/den */
    double fs, c;
    int form;               /* fcc_form_t */
} fcc_plan_info_t;

typedef struct fcc_plan fcc_plan_t;

/*
 * Build the bases for one (geometry, N, grid, K, precision) key (Sec. 4,
 * Eqs. 6-7): the even and odd halves of W are formed in FP64 on the GPU with
 * exact argument reduction, each half gets its own FP64 one-sided Jacobi SVD on
 * the GPU, the singular values are merged and K is chosen, and the cropped
 * bases and the lag dictionary are packed for the kernels.  Synchronous.
 * On success *out owns device memory until fcc_plan_destroy().
 * Errors: INVALID_ARG (bad desc/out), UNSUPPORTED, OOM, CUDA, NOT_CONVERGED.
 */
fcc_status_t fcc_plan_create(const fcc_plan_desc_t *desc, fcc_plan_t **out);

/* Release a plan (NULL is ignored).  Waits for the plan's device work. */
void fcc_plan_destroy(fcc_plan_t *plan);

/* Copy the plan's sizes into *info (host memory).  Errors: INVALID_ARG (NULL). */
fcc_status_t fcc_plan_info(const fcc_plan_t *plan, fcc_plan_info_t *info);

/*
 * Select the kernel fcc_tdoa (and fcc_tdoa_host) runs for this plan (an
 * fcc_engine_t; the same arithmetic of Secs. 2-4 on different hardware units).
 * Not thread-safe against a concurrent launch on the same plan.
 * Errors: INVALID_ARG (null plan, unknown engine), UNSUPPORTED (the engine does
 * not apply to this plan's size or precision; the plan keeps its engine).
 */
fcc_status_t fcc_plan_set_engine(fcc_plan_t *plan, int engine);

/* The engine fcc_tdoa runs for this plan (AUTO resolved).  Errors: INVALID_ARG (NULL). */
fcc_status_t fcc_plan_get_engine(const fcc_plan_t *plan, int *engine);

/* Copy the lag grid tau_0..tau_{I-1} (samples, Sec. 3) into host taus[I].
 * Errors: INVALID_ARG (NULL). */
fcc_status_t fcc_plan_taus(const fcc_plan_t *plan, double *taus);

/*
 * Copy every singular value of the even block (min(I, Q+1) values) and of the
 * odd block (min(I, Q) values), each in descending order, into host arrays
 * s_even / s_odd (either may be NULL); their counts go to *n_even / *n_odd.
 * Together they are the singular values of W (Sec. 4).  Errors: INVALID_ARG
 * (NULL plan).
 */
fcc_status_t fcc_plan_singular_values(const fcc_plan_t *plan, double *s_even, int *n_even,
                                      double *s_odd, int *n_odd);

/*
 * Copy the FP64 bases the kernels use (host arrays, row-major, any may be NULL):
 *   Pe[K_even][Q+1]  cropped even projection bases p_hat_k (Eq. 7), applied to x_s;
 *   Po[K_odd][Q]     cropped odd bases (the real q_hat with p_hat = j q_hat), applied
 *                    to x_d (Eq. 8); entry f = Q is zero for odd bases and omitted;
 *   Ue[I][K_even], Uo[I][K_odd]  dictionary columns (D = U_hat, Sec. 4) with the
 *                    common phase exp(j pi tau / 2) factored out.
 * With z_e = Pe x_s and z_o = Po x_d (complex), the correlation is
 *   y(tau_i) = 2 Re{ exp(j pi tau_i / 2) (Ue z_e + j Uo z_o)[i] }.
 * For FCC_FORM_REIM_SPLIT plans: Pe[K_c][N/2+1] and Po[K_s][N/2+1] are the
 * cosine and sine projections (sigma_k v_k of C and S), Ue[I][K_c] and Uo[I][K_s]
 * their left vectors, and y = 2 (Ue (Pe Re x) - Uo (Po Im x)).
 * Errors: INVALID_ARG (NULL plan).
 */
fcc_status_t fcc_plan_bases(const fcc_plan_t *plan, double *Pe, double *Po, double *Ue, double *Uo);

/*
 * FCC hot path (Sec. 2 PHAT -> Eq. 8 fold -> Eq. 9 projection -> reconstruction
 * on the lag grid -> argmax -> quadratic refinement) over T frames.
 *   d_spectra  device complex64 [T][M][B] (16-byte aligned).
 *   T          number of frames, >= 0 (0 is a no-op).
 *   d_lag_idx  device int32 [T][P]: argmax lag index (required).
 *   d_peak     device float [T][P]: y at the argmax (required).
 *   d_tau_hat  device float [T][P]: refined TDoA in samples, or NULL.
 *   d_coeffs   device float [T][P][2K]: projection coefficients in the order
 *              Re z_e (K_even), Im z_e (K_even), Re z_o (K_odd), Im z_o (K_odd); or NULL
 *              (must be NULL for the split form: UNSUPPORTED).
 *   d_corr     device float [T][P][I]: the correlation y on the grid; or NULL.
 *              FP32 plans with 6-8 bases of a parity and at least 32 lag steps
 *              each way evaluate the grid on the tensor cores (a three-term
 *              FP16 split, FP32 sums) and the argmax lag and its neighbours in
 *              FP32; d_peak equals d_corr at d_lag_idx either way.
 *   stream     cudaStream_t or NULL.
 * Sizes the kernels take: FP32 plans N <= 1024, BF16 / FP16 plans
 * 128 <= N <= 1024, and at most 8 bases of each parity; other plans return
 * UNSUPPORTED here (their bases, fcc_gcc_tdoa and the smoothed path, within its
 * own limits, still work).
 * Asynchronous; allocates nothing.  Errors: INVALID_ARG, UNSUPPORTED, CUDA.
 */
fcc_status_t fcc_tdoa(fcc_plan_t *plan, const void *d_spectra, long long T, int *d_lag_idx,
                      float *d_peak, float *d_tau_hat, float *d_coeffs, float *d_corr,
                      void *stream);

/*
 * fcc_tdoa from and to HOST memory: the frames are streamed to the device in
 * chunks through the plan's double-buffered staging area (allocated on the
 * first call, about 2 x 256 MiB), overlapping host-to-device copies with the
 * kernels; results are copied back.  Host buffers should be page-locked for
 * full copy bandwidth.  Synchronous: returns after the results are in host
 * memory and the device error word has been checked.
 *   h_spectra complex64 [T][M][B]; h_lag_idx int32 [T][P]; h_peak float [T][P];
 *   h_tau_hat float [T][P] or NULL.
 * Errors: INVALID_ARG, UNSUPPORTED, OOM (staging; nothing of it is kept),
 * CUDA, NONFINITE, TIMEOUT.
 */
fcc_status_t fcc_tdoa_host(fcc_plan_t *plan, const void *h_spectra, long long T,
                           int *h_lag_idx, float *h_peak, float *h_tau_hat, void *stream);

/*
 * Same-GPU GCC-PHAT baseline (Sec. 3, eq. 2 through an r-times zero-padded
 * real inverse FFT with r = den; the DC bin, and for r = 1 the Nyquist bin, is
 * doubled so that the values equal eq. 2 exactly): PHAT pair spectra ->
 * batched cuFFT C2R of size rN -> gather on the lag grid -> argmax.
 * Uses the full-rank correlation (no basis truncation).  Runs in chunks of
 * frames through a workspace owned by the plan (created on the first call).
 *   d_corr  device float [T][P][I] or NULL.
 * Asynchronous.  Errors: INVALID_ARG, OOM, CUDA.
 */
fcc_status_t fcc_gcc_tdoa(fcc_plan_t *plan, const void *d_spectra, long long T, int *d_lag_idx,
                          float *d_peak, float *d_corr, void *stream);

/*
 * Basis construction that allocates no device memory.  The paper has no
 * counterpart: it builds its bases once, offline.
 *
 * Who needs it: callers that must not call cudaMalloc / cudaFree while they
 * run -- a real-time audio process whose other streams must never stall (both
 * calls may synchronise the whole device), code embedded in a framework that
 * owns every device byte through its own pool, or an array whose geometry
 * changes on the fly and must get fresh bases without touching the allocator.
 *
 * It computes exactly what fcc_plan_create's basis step computes (the even
 * and odd halves of W in FP64, a Jacobi SVD of each on the GPU, the K rule,
 * canonical signs) for the sizes `desc` describes, but the working matrices
 * live in one static device array of 4 MiB inside the library, which every GPU
 * that loads the library keeps until the process exits.  The grid must satisfy
 * I (N/2 + 1) + 2 I^2 + 32 <= 524288 doubles (I = 2 L lag_den + 1); larger
 * grids return FCC_ERR_UNSUPPORTED with the sizes in fcc_last_error().  No
 * other allocation is made on the device.
 *
 * The first call on a device looks up the array's device address.  Under lazy
 * module loading (the CUDA default) that first call may also be what loads the
 * library's device code on that device, and the 4 MiB array is allocated when
 * the code is loaded: make the first call before any stream capture and before
 * the point from which the caller may no longer allocate.  Every call uses the same array, so
 * calls whose work overlaps on the GPU (from several threads or streams) race
 * and must be serialised by the caller.  Kernels and copies run on `stream`;
 * the call returns after synchronising it.
 *
 * Outputs are host arrays (each may be NULL), laid out as in
 * fcc_plan_singular_values / fcc_plan_bases: s_even[min(I, Q+1)],
 * s_odd[min(I, Q)], Pe[K_even][Q+1], Po[K_odd][Q], Ue[I][K_even],
 * Uo[I][K_odd].  K is known only after the SVD: call once with only `info`
 * to learn K_even / K_odd, then again with arrays of those sizes.
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA, NOT_CONVERGED.
 */
fcc_status_t fcc_plan_bases_noalloc(const fcc_plan_desc_t *desc, fcc_plan_info_t *info,
                                    double *s_even, double *s_odd, double *Pe, double *Po,
                                    double *Ue, double *Uo, void *stream);

/*
 * Synchronise `stream` (NULL = legacy default), then read and clear the plan's
 * device error word: FCC_OK, FCC_ERR_NONFINITE or FCC_ERR_TIMEOUT.
 * Errors: INVALID_ARG (NULL plan), CUDA.
 */
fcc_status_t fcc_plan_sync(fcc_plan_t *plan, void *stream);

/* Static description of a status code. */
const char *fcc_status_string(fcc_status_t status);

/* Detail of the last error raised on the calling thread ("" if none). */
const char *fcc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FCC_GB300_H */
