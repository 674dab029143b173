/*
 * fcc_oracle.c -- plain, slow FP64 reference for Fast Cross-Correlation (FCC)
 * TDoA estimation (Grondin, Maheux, Lauzon, Vincent, Michaud, "Fast
 * Cross-Correlation for TDoA Estimation on Small Aperture Microphone Arrays").
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's CPU
 * baseline call this file; the product library never links, loads or calls it,
 * and it shares no code, header or table with the CUDA path.
 *
 * It follows the paper's definitions literally, in FP64, with no folding,
 * blocking or reordering:
 *   - Sec. 3: the candidate grid tau_i = -L + i*delta, delta = 1/r, which gives
 *     I = 2rL + 1 candidates (the paper prints the r = 2 case, I = 4L + 1).
 *   - Eq. 3: W(i,f) = exp(j 2 pi f tau_i / N), f = 0..N/2 (I x (N/2+1)).
 *   - Sec. 4: W = U S V^H, truncated to the K largest singular values; the
 *     rank-K operator W_K = U_K S_K V_K^H.  The SVD is this file's own complex
 *     one-sided (Hestenes) Jacobi iteration, checked against LAPACK in tests.
 *   - Sec. 2, Eq. 1 with alpha = 1: R = X_i X_j^*, R_hat = R / |R| (R_hat = 0
 *     where |R| = 0); or_tdoa_smoothed runs Eq. 1's recursion for alpha < 1.
 *   - Eq. 2 / Eq. 4: y = 2 Re{ W_K x } with x = R_hat stacked over f.  With
 *     K = rank(W) this is eq. 2 itself (full-rank GCC-PHAT on the grid).
 *   - Sec. 2: tau* = argmax y (lowest index wins an exact tie) and a
 *     three-point quadratic refinement around it.
 *
 * The folded even/odd form of Eqs. 6-9 is deliberately NOT used here: by the
 * paper's argument it must equal 2 Re{W_K x}, which is what the CUDA path is
 * checked against.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846264338327950288

/* Sec. 3: tau_i = -L + i/den, i = 0..2*L*den.  Returns I. */
int or_grid(int L, int den, double *taus)
{
    int I = 2 * L * den + 1;
    if (taus)
        for (int i = 0; i < I; ++i)
            taus[i] = -(double)L + (double)i / (double)den;
    return I;
}

/* Eq. 3: W(i,f) = exp(j 2 pi f tau_i / N), row-major [I][N/2+1]. */
void or_build_W(int N, int I, const double *taus, double *W_re, double *W_im)
{
    int B = N / 2 + 1;
    for (int i = 0; i < I; ++i)
        for (int f = 0; f < B; ++f) {
            double arg = 2.0 * OR_PI * (double)f * taus[i] / (double)N;
            W_re[(size_t)i * B + f] = cos(arg);
            W_im[(size_t)i * B + f] = sin(arg);
        }
}

/*
 * Sec. 4: SVD of a complex m x n matrix A (row-major, re/im planes) by the
 * one-sided Jacobi method of Hestenes (1958).
 *
 * Let a_i (i = 0..m-1) be the rows of A.  The m columns of X = A^H are
 * x_i = conj(a_i) in C^n; these are the vectors being orthogonalised.  Plane rotations J are applied on the right, X <- X J,
 * until all columns are mutually orthogonal; the product of the rotations is
 * the m x m unitary G.  Then A^H G = Y with orthogonal columns y_k, so
 * A = G Y^H = sum_k s_k g_k v_k^H with s_k = |y_k|, v_k = y_k / s_k.
 *
 * Outputs (all row-major): s[r] descending (r = min(m, n)), U[m][r] = G's
 * columns, V[n][r].  Returns the number of sweeps used, or -1 if it did not
 * converge in max_sweeps.
 */
int or_svd(int m, int n, const double *A_re, const double *A_im, double *s,
           double *U_re, double *U_im, double *V_re, double *V_im, int max_sweeps)
{
    /* X: m columns of length n, stored column-contiguous: Xc[k][t]. */
    double *Xr = (double *)malloc(sizeof(double) * (size_t)m * n);
    double *Xi = (double *)malloc(sizeof(double) * (size_t)m * n);
    double *Gr = (double *)calloc((size_t)m * m, sizeof(double));
    double *Gi = (double *)calloc((size_t)m * m, sizeof(double));
    int r = m < n ? m : n;
    for (int k = 0; k < m; ++k) {
        for (int t = 0; t < n; ++t) {
            Xr[(size_t)k * n + t] = A_re[(size_t)k * n + t];
            Xi[(size_t)k * n + t] = -A_im[(size_t)k * n + t];
        }
        Gr[(size_t)k * m + k] = 1.0; /* G stored column-contiguous: Gc[k][row] */
    }
    const double tol = 1e-15;
    int sweep, converged = 0;
    for (sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
        converged = 1;
        for (int p = 0; p < m - 1; ++p)
            for (int q = p + 1; q < m; ++q) {
                double *xpr = Xr + (size_t)p * n, *xpi = Xi + (size_t)p * n;
                double *xqr = Xr + (size_t)q * n, *xqi = Xi + (size_t)q * n;
                double alpha = 0, beta = 0, gr = 0, gi = 0;
                for (int t = 0; t < n; ++t) {
                    alpha += xpr[t] * xpr[t] + xpi[t] * xpi[t];
                    beta += xqr[t] * xqr[t] + xqi[t] * xqi[t];
                    /* gamma = x_p^H x_q */
                    gr += xpr[t] * xqr[t] + xpi[t] * xqi[t];
                    gi += xpr[t] * xqi[t] - xpi[t] * xqr[t];
                }
                double ag = sqrt(gr * gr + gi * gi);
                if (ag <= tol * sqrt(alpha * beta) || ag == 0.0)
                    continue;
                converged = 0;
                /* gamma = |gamma| e^{j theta}; phase-align x_q, then a real
                 * rotation zeroes the off-diagonal of the 2x2 Gram matrix. */
                double er = gr / ag, ei = -gi / ag; /* e^{-j theta} */
                double zeta = (beta - alpha) / (2.0 * ag);
                double t_ = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t_ * t_), sn = c * t_;
                for (int t = 0; t < n; ++t) {
                    double qr = xqr[t] * er - xqi[t] * ei; /* e^{-j theta} x_q */
                    double qi = xqr[t] * ei + xqi[t] * er;
                    double pr = xpr[t], pi = xpi[t];
                    xpr[t] = c * pr - sn * qr;
                    xpi[t] = c * pi - sn * qi;
                    xqr[t] = sn * pr + c * qr;
                    xqi[t] = sn * pi + c * qi;
                }
                double *gpr = Gr + (size_t)p * m, *gpi = Gi + (size_t)p * m;
                double *gqr = Gr + (size_t)q * m, *gqi = Gi + (size_t)q * m;
                for (int t = 0; t < m; ++t) {
                    double qr = gqr[t] * er - gqi[t] * ei;
                    double qi = gqr[t] * ei + gqi[t] * er;
                    double pr = gpr[t], pi = gpi[t];
                    gpr[t] = c * pr - sn * qr;
                    gpi[t] = c * pi - sn * qi;
                    gqr[t] = sn * pr + c * qr;
                    gqi[t] = sn * pi + c * qi;
                }
            }
    }
    /* Column norms and a descending order (selection by index, stable). */
    double *nrm = (double *)malloc(sizeof(double) * m);
    int *ord = (int *)malloc(sizeof(int) * m);
    for (int k = 0; k < m; ++k) {
        double a = 0;
        for (int t = 0; t < n; ++t)
            a += Xr[(size_t)k * n + t] * Xr[(size_t)k * n + t] + Xi[(size_t)k * n + t] * Xi[(size_t)k * n + t];
        nrm[k] = sqrt(a);
        ord[k] = k;
    }
    for (int a = 0; a < m; ++a)
        for (int b = a + 1; b < m; ++b)
            if (nrm[ord[b]] > nrm[ord[a]]) {
                int tmp = ord[a];
                ord[a] = ord[b];
                ord[b] = tmp;
            }
    for (int k = 0; k < r; ++k) {
        int c = ord[k];
        s[k] = nrm[c];
        for (int row = 0; row < m; ++row) {
            U_re[(size_t)row * r + k] = Gr[(size_t)c * m + row];
            U_im[(size_t)row * r + k] = Gi[(size_t)c * m + row];
        }
        double inv = nrm[c] > 0 ? 1.0 / nrm[c] : 0.0;
        for (int t = 0; t < n; ++t) {
            V_re[(size_t)t * r + k] = Xr[(size_t)c * n + t] * inv;
            V_im[(size_t)t * r + k] = Xi[(size_t)c * n + t] * inv;
        }
    }
    free(Xr); free(Xi); free(Gr); free(Gi); free(nrm); free(ord);
    return converged ? sweep : -1;
}

/*
 * Sec. 4 leaves K "to be set experimentally"; the rule used here is the
 * smallest K whose leading singular values hold at least `energy` of the
 * total energy sum(s^2), extended over singular values tied with s_K (relative
 * gap below tie_rel) so that W_K stays uniquely defined.
 */
int or_rank_energy(const double *s, int r, double energy, double tie_rel)
{
    double tot = 0, acc = 0;
    for (int k = 0; k < r; ++k) tot += s[k] * s[k];
    int K = r;
    for (int k = 0; k < r; ++k) {
        acc += s[k] * s[k];
        if (acc >= energy * tot) { K = k + 1; break; }
    }
    while (K < r && s[K - 1] - s[K] <= tie_rel * s[K - 1]) ++K;
    return K;
}

/* Sec. 4: W_K = U_K diag(s_K) V_K^H, row-major [m][n]. */
void or_lowrank(int m, int n, int r, int K, const double *s,
                const double *U_re, const double *U_im,
                const double *V_re, const double *V_im, double *WK_re, double *WK_im)
{
    for (int i = 0; i < m; ++i)
        for (int f = 0; f < n; ++f) {
            double ar = 0, ai = 0;
            for (int k = 0; k < K; ++k) {
                double ur = U_re[(size_t)i * r + k], ui = U_im[(size_t)i * r + k];
                double vr = V_re[(size_t)f * r + k], vi = -V_im[(size_t)f * r + k]; /* conj */
                ar += s[k] * (ur * vr - ui * vi);
                ai += s[k] * (ur * vi + ui * vr);
            }
            WK_re[(size_t)i * n + f] = ar;
            WK_im[(size_t)i * n + f] = ai;
        }
}

/*
 * Sec. 2 (eq. 1 with alpha = 1, then the phase transform): for one frame of
 * spectra X[m][f] (complex64, interleaved re/im), R(f) = X_i(f) X_j(f)^* and
 * R_hat(f) = R(f)/|R(f)|, or 0 where |R(f)| = 0.
 */
void or_phat(const float *X, int B, int i, int j, double *xr, double *xi)
{
    for (int f = 0; f < B; ++f) {
        double ar = X[2 * ((size_t)i * B + f)], ai = X[2 * ((size_t)i * B + f) + 1];
        double br = X[2 * ((size_t)j * B + f)], bi = X[2 * ((size_t)j * B + f) + 1];
        double rr = ar * br + ai * bi; /* X_i X_j^* */
        double ri = ai * br - ar * bi;
        double mag = sqrt(rr * rr + ri * ri);
        if (mag > 0) {
            xr[f] = rr / mag;
            xi[f] = ri / mag;
        } else {
            xr[f] = 0;
            xi[f] = 0;
        }
    }
}

/* Eq. 4: y = 2 Re{ W x } for an I x B complex operator W. */
void or_correlate(int I, int B, const double *W_re, const double *W_im,
                  const double *xr, const double *xi, double *y)
{
    for (int i = 0; i < I; ++i) {
        double acc = 0;
        for (int f = 0; f < B; ++f)
            acc += W_re[(size_t)i * B + f] * xr[f] - W_im[(size_t)i * B + f] * xi[f];
        y[i] = 2.0 * acc;
    }
}

/* Sec. 2: tau* = argmax_i y(tau_i); the lowest index wins an exact tie. */
int or_argmax(const double *y, int I)
{
    int best = 0;
    for (int i = 1; i < I; ++i)
        if (y[i] > y[best]) best = i;
    return best;
}

/*
 * Sec. 2: quadratic interpolation through (tau*-delta, tau*, tau*+delta).  The
 * vertex offset is d = (y- - y+) / (2 (y- - 2 y0 + y+)) grid steps.  No
 * refinement at a grid edge or where the three points are not concave
 * (denominator >= 0); d is clamped to [-1/2, 1/2].
 */
double or_parabola(const double *y, int I, int idx, double tau_idx, double delta)
{
    if (idx <= 0 || idx >= I - 1) return tau_idx;
    double ym = y[idx - 1], y0 = y[idx], yp = y[idx + 1];
    double den = ym - 2.0 * y0 + yp;
    if (!(den < 0)) return tau_idx;
    double d = 0.5 * (ym - yp) / den;
    if (d > 0.5) d = 0.5;
    if (d < -0.5) d = -0.5;
    return tau_idx + delta * d;
}

/*
 * The whole per-pair-frame pipeline over T frames of spectra X[t][m][f]
 * (complex64, f = 0..N/2) and every pair (i, j), i < j, in lexicographic
 * order: R_hat (Sec. 2) -> y = 2 Re{W x} (Eq. 4, W = W_K or the full W) ->
 * argmax -> quadratic refinement.  Outputs are [T][P] (idx, peak, tau_hat)
 * and, if y_out is not NULL, [T][P][I].  Frames are independent (alpha = 1),
 * so they are split across n_threads OpenMP threads.
 */
void or_tdoa(const float *X, long long T, int M, int N, int I,
             const double *W_re, const double *W_im, const double *taus, double delta,
             int *idx_out, double *peak_out, double *tau_out, double *y_out, int n_threads)
{
    int B = N / 2 + 1;
    int P = M * (M - 1) / 2;
#ifdef _OPENMP
    if (n_threads < 1) n_threads = 1;
#pragma omp parallel num_threads(n_threads)
#endif
    {
        double *xr = (double *)malloc(sizeof(double) * B);
        double *xi = (double *)malloc(sizeof(double) * B);
        double *y = (double *)malloc(sizeof(double) * I);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (long long t = 0; t < T; ++t) {
            const float *Xt = X + (size_t)t * M * B * 2;
            int p = 0;
            for (int i = 0; i < M; ++i)
                for (int j = i + 1; j < M; ++j, ++p) {
                    or_phat(Xt, B, i, j, xr, xi);
                    or_correlate(I, B, W_re, W_im, xr, xi, y);
                    int k = or_argmax(y, I);
                    size_t o = (size_t)t * P + p;
                    idx_out[o] = k;
                    peak_out[o] = y[k];
                    tau_out[o] = or_parabola(y, I, k, taus[k], delta);
                    if (y_out)
                        memcpy(y_out + o * I, y, sizeof(double) * I);
                }
        }
        free(xr); free(xi); free(y);
    }
}

/*
 * Sec. 2, Eq. 1 with a smoothing factor alpha in (0, 1]: per pair and bin the
 * cross-spectrum is estimated recursively over the frames,
 *   R(t,f) = (1 - alpha) R(t-1,f) + alpha X_i(t,f) X_j(t,f)^*,
 * starting from R0 (the state before the first frame: zero for a fresh stream),
 * then the phase transform R_hat = R / |R| (0 where |R| = 0), y = 2 Re{ W x },
 * argmax and the three-point refinement, as in or_tdoa.  The recurrence is
 * sequential in t; pairs run in parallel.  R0 (may be NULL: zero) and R_end
 * (may be NULL) are [P][B] complex, re/im interleaved, FP64.
 */
void or_tdoa_smoothed(const float *X, long long T, int M, int N, int I,
                      const double *W_re, const double *W_im, const double *taus, double delta,
                      double alpha, const double *R0, double *R_end,
                      int *idx_out, double *peak_out, double *tau_out, double *y_out, int n_threads)
{
    int B = N / 2 + 1;
    int P = M * (M - 1) / 2;
#ifdef _OPENMP
    if (n_threads < 1) n_threads = 1;
#pragma omp parallel num_threads(n_threads)
#endif
    {
        double *Rr = (double *)malloc(sizeof(double) * B);
        double *Ri = (double *)malloc(sizeof(double) * B);
        double *xr = (double *)malloc(sizeof(double) * B);
        double *xi = (double *)malloc(sizeof(double) * B);
        double *y = (double *)malloc(sizeof(double) * I);
#ifdef _OPENMP
#pragma omp for schedule(dynamic)
#endif
        for (int p = 0; p < P; ++p) {
            /* pair index p -> (i, j), i < j, lexicographic */
            int i = 0, j = 0, q = p;
            for (i = 0; i < M; ++i) {
                if (q < M - 1 - i) { j = i + 1 + q; break; }
                q -= M - 1 - i;
            }
            for (int f = 0; f < B; ++f) {
                Rr[f] = R0 ? R0[2 * ((size_t)p * B + f)] : 0.0;
                Ri[f] = R0 ? R0[2 * ((size_t)p * B + f) + 1] : 0.0;
            }
            for (long long t = 0; t < T; ++t) {
                const float *Xt = X + (size_t)t * M * B * 2;
                for (int f = 0; f < B; ++f) {
                    double ar = Xt[2 * ((size_t)i * B + f)], ai = Xt[2 * ((size_t)i * B + f) + 1];
                    double br = Xt[2 * ((size_t)j * B + f)], bi = Xt[2 * ((size_t)j * B + f) + 1];
                    double cr = ar * br + ai * bi; /* X_i X_j^* */
                    double ci = ai * br - ar * bi;
                    Rr[f] = (1.0 - alpha) * Rr[f] + alpha * cr;
                    Ri[f] = (1.0 - alpha) * Ri[f] + alpha * ci;
                    double mag = sqrt(Rr[f] * Rr[f] + Ri[f] * Ri[f]);
                    xr[f] = mag > 0 ? Rr[f] / mag : 0.0;
                    xi[f] = mag > 0 ? Ri[f] / mag : 0.0;
                }
                or_correlate(I, B, W_re, W_im, xr, xi, y);
                int k = or_argmax(y, I);
                size_t o = (size_t)t * P + p;
                idx_out[o] = k;
                peak_out[o] = y[k];
                tau_out[o] = or_parabola(y, I, k, taus[k], delta);
                if (y_out)
                    memcpy(y_out + o * I, y, sizeof(double) * I);
            }
            if (R_end)
                for (int f = 0; f < B; ++f) {
                    R_end[2 * ((size_t)p * B + f)] = Rr[f];
                    R_end[2 * ((size_t)p * B + f) + 1] = Ri[f];
                }
        }
        free(Rr); free(Ri); free(xr); free(xi); free(y);
    }
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Learned TDoA head (not part of the paper's method; an extension that maps a
 * pair-frame's 2K projection coefficients to a sub-sample TDoA and a
 * confidence).  Plain FP64 definitions, one sample at a time:
 *   a1 = W1 x + b1,  h1 = gelu(a1)           (H x nin, exact erf GELU)
 *   a2 = W2 h1 + b2, h2 = gelu(a2)           (H x H)
 *   y  = W3 h2 + b3                          (2 x H): y0 = TDoA, y1 = confidence logit
 * Loss (mean over n): (y0 - t)^2 + lambda * BCE(sigmoid(y1), g) with the
 * target g = [|y0 - t| <= |t_fcc - t|] (held constant).  Parameters are packed
 * as W1, b1, W2, b2, W3, b3 (row-major).
 * ------------------------------------------------------------------------ */
static double or_gelu(double a) { return 0.5 * a * (1.0 + erf(a / sqrt(2.0))); }
static double or_gelu_d(double a)
{
    return 0.5 * (1.0 + erf(a / sqrt(2.0))) + a * exp(-0.5 * a * a) / sqrt(2.0 * OR_PI);
}

long long or_mlp_nparams(int nin, int H) { return (long long)H * nin + H + (long long)H * H + H + 2 * H + 2; }

static void or_mlp_unpack(const double *p, int nin, int H, const double **W1, const double **b1,
                          const double **W2, const double **b2, const double **W3, const double **b3)
{
    *W1 = p;
    *b1 = *W1 + (size_t)H * nin;
    *W2 = *b1 + H;
    *b2 = *W2 + (size_t)H * H;
    *W3 = *b2 + H;
    *b3 = *W3 + 2 * (size_t)H;
}

static void or_mlp_one(const double *x, int nin, int H, const double *params, double *a1, double *a2, double *y)
{
    const double *W1, *b1, *W2, *b2, *W3, *b3;
    or_mlp_unpack(params, nin, H, &W1, &b1, &W2, &b2, &W3, &b3);
    for (int j = 0; j < H; ++j) {
        double s = b1[j];
        for (int i = 0; i < nin; ++i) s += W1[(size_t)j * nin + i] * x[i];
        a1[j] = s;
    }
    for (int j = 0; j < H; ++j) {
        double s = b2[j];
        for (int i = 0; i < H; ++i) s += W2[(size_t)j * H + i] * or_gelu(a1[i]);
        a2[j] = s;
    }
    for (int o = 0; o < 2; ++o) {
        double s = b3[o];
        for (int j = 0; j < H; ++j) s += W3[(size_t)o * H + j] * or_gelu(a2[j]);
        y[o] = s;
    }
}

void or_mlp_forward(const double *x, long long n, int nin, int H, const double *params, double *y)
{
    double *a1 = (double *)malloc(sizeof(double) * H), *a2 = (double *)malloc(sizeof(double) * H);
    for (long long s = 0; s < n; ++s) or_mlp_one(x + (size_t)s * nin, nin, H, params, a1, a2, y + 2 * s);
    free(a1);
    free(a2);
}

/* Mean loss; grad (same packing as params) is overwritten with dLoss/dparams. */
double or_mlp_loss_grad(const double *x, long long n, int nin, int H, const double *params, const double *t,
                        const double *tfcc, double lambda, double *grad)
{
    const double *W1, *b1, *W2, *b2, *W3, *b3;
    or_mlp_unpack(params, nin, H, &W1, &b1, &W2, &b2, &W3, &b3);
    const long long np_ = or_mlp_nparams(nin, H);
    for (long long k = 0; k < np_; ++k) grad[k] = 0.0;
    double *gW1 = grad, *gb1 = gW1 + (size_t)H * nin, *gW2 = gb1 + H, *gb2 = gW2 + (size_t)H * H, *gW3 = gb2 + H,
           *gb3 = gW3 + 2 * (size_t)H;
    double *a1 = (double *)malloc(sizeof(double) * H), *a2 = (double *)malloc(sizeof(double) * H);
    double *d2 = (double *)malloc(sizeof(double) * H), *d1 = (double *)malloc(sizeof(double) * H);
    double loss = 0.0;
    for (long long s = 0; s < n; ++s) {
        const double *xs = x + (size_t)s * nin;
        double y[2];
        or_mlp_one(xs, nin, H, params, a1, a2, y);
        const double e = y[0] - t[s];
        const double g = fabs(e) <= fabs(tfcc[s] - t[s]) ? 1.0 : 0.0;
        const double c = 1.0 / (1.0 + exp(-y[1]));
        /* BCE(sigmoid(y1), g) = softplus(y1) - g y1, written stably */
        const double bce = (y[1] > 0 ? y[1] + log1p(exp(-y[1])) : log1p(exp(y[1]))) - g * y[1];
        loss += e * e + lambda * bce;
        const double dy0 = 2.0 * e / (double)n, dy1 = lambda * (c - g) / (double)n;
        for (int j = 0; j < H; ++j) {
            const double h2 = or_gelu(a2[j]);
            gW3[j] += dy0 * h2;
            gW3[H + j] += dy1 * h2;
            d2[j] = (W3[j] * dy0 + W3[H + j] * dy1) * or_gelu_d(a2[j]);
            gb2[j] += d2[j];
        }
        gb3[0] += dy0;
        gb3[1] += dy1;
        for (int i = 0; i < H; ++i) {
            const double h1 = or_gelu(a1[i]);
            double s2 = 0.0;
            for (int j = 0; j < H; ++j) {
                gW2[(size_t)j * H + i] += d2[j] * h1;
                s2 += W2[(size_t)j * H + i] * d2[j];
            }
            d1[i] = s2 * or_gelu_d(a1[i]);
            gb1[i] += d1[i];
            for (int k = 0; k < nin; ++k) gW1[(size_t)i * nin + k] += d1[i] * xs[k];
        }
    }
    free(a1);
    free(a2);
    free(d1);
    free(d2);
    return loss / (double)n;
}

/* Adam (Kingma & Ba 2015) with bias correction; step counts from 1. */
void or_adam(double *p, const double *g, double *m, double *v, long long n, int step, double lr, double beta1,
             double beta2, double eps)
{
    const double c1 = 1.0 - pow(beta1, step), c2 = 1.0 - pow(beta2, step);
    for (long long k = 0; k < n; ++k) {
        m[k] = beta1 * m[k] + (1.0 - beta1) * g[k];
        v[k] = beta2 * v[k] + (1.0 - beta2) * g[k] * g[k];
        p[k] -= lr * (m[k] / c1) / (sqrt(v[k] / c2) + eps);
    }
}

/*
 * Multi-pair DoA search over direction candidates (the step the paper's
 * conclusion names after per-pair TDoA; the paper prints no formula, so this
 * is the steered-response power it refers to): for a candidate unit vector u,
 * a far-field plane wave from u reaches mic m at t_m = -(fs / c) (r_m . u)
 * samples, so pair (i, j) sees tau_ij(u) = t_i - t_j.  The pair's correlation
 * on the lag grid y_ij(tau_k), tau_k = -L + k / den, is read at tau_ij(u) by
 * linear interpolation (grid position (tau + L) den, clamped to [0, I - 1]);
 * score(u) = sum over pairs.  Per frame: the best candidate (lowest index on
 * an exact tie) and its score; scores_out (may be NULL) gets every score.
 *
 * y: [T][P][I] (pairs i < j lexicographic); mic_xyz: [M][3] metres;
 * dirs: [D][3] unit vectors.  Frames in parallel.
 */
void or_doa_srp(const double *y, long long T, int M, int I, int L, int den, const double *mic_xyz,
                double fs, double c, const double *dirs, int D, int *idx_out, double *score_out,
                double *scores_out, int n_threads)
{
    int P = M * (M - 1) / 2;
    /* grid positions and weights per (direction, pair), FP64 */
    int *k0 = (int *)malloc(sizeof(int) * (size_t)D * P);
    double *wt = (double *)malloc(sizeof(double) * (size_t)D * P);
    for (int d = 0; d < D; ++d) {
        int p = 0;
        for (int i = 0; i < M; ++i)
            for (int j = i + 1; j < M; ++j, ++p) {
                double ti = -(fs / c) * (mic_xyz[3 * i] * dirs[3 * d] + mic_xyz[3 * i + 1] * dirs[3 * d + 1] +
                                         mic_xyz[3 * i + 2] * dirs[3 * d + 2]);
                double tj = -(fs / c) * (mic_xyz[3 * j] * dirs[3 * d] + mic_xyz[3 * j + 1] * dirs[3 * d + 1] +
                                         mic_xyz[3 * j + 2] * dirs[3 * d + 2]);
                double pos = (ti - tj + (double)L) * (double)den;
                if (pos < 0.0) pos = 0.0;
                if (pos > (double)(I - 1)) pos = (double)(I - 1);
                int k = (int)floor(pos);
                if (k > I - 2) k = I - 2;
                k0[(size_t)d * P + p] = k;
                wt[(size_t)d * P + p] = pos - (double)k;
            }
    }
#ifdef _OPENMP
    if (n_threads < 1) n_threads = 1;
#pragma omp parallel for num_threads(n_threads) schedule(static)
#endif
    for (long long t = 0; t < T; ++t) {
        const double *yt = y + (size_t)t * P * I;
        int best = 0;
        double best_s = 0.0;
        for (int d = 0; d < D; ++d) {
            double s = 0.0;
            for (int p = 0; p < P; ++p) {
                int k = k0[(size_t)d * P + p];
                double w = wt[(size_t)d * P + p];
                s += (1.0 - w) * yt[(size_t)p * I + k] + w * yt[(size_t)p * I + k + 1];
            }
            if (scores_out) scores_out[(size_t)t * D + d] = s;
            if (d == 0 || s > best_s) {
                best = d;
                best_s = s;
            }
        }
        idx_out[t] = best;
        score_out[t] = best_s;
    }
    free(k0);
    free(wt);
}
