// fcc_plan.cu -- basis construction for one plan key (Sec. 4, Eqs. 6-7).
//
// W(i,f) = exp(j 2 pi f tau_i / N) (Eq. 3).  With g = f - N/4 and phi_i =
// exp(j pi tau_i / 2), W = diag(phi) (C + j S) where C(i,g) = cos(2 pi g tau_i/N)
// is even in g and S(i,g) = sin(2 pi g tau_i / N) is odd in g.  For a grid that
// is symmetric about 0, W^H W = C^T C + S^T S, so the right singular vectors of
// W split into functions even about f = N/4 (those of C) and odd ones (those
// of S) -- the parity property of Eq. 6.  Folding x with the orthonormal maps
//   F_e: x -> [(x(f) + x(N/2-f))/sqrt2 for f < N/4,  x(N/4)]   (Eq. 8, x_s)
//   F_o: x -> [(x(f) - x(N/2-f))/sqrt2 for f < N/4]            (Eq. 8, x_d)
// gives two small real matrices, one per parity,
//   A_e(i,f) = w_f cos(2 pi (f - N/4) tau_i / N),  w_f = sqrt2 (f < N/4), 1 (f = N/4)
//   A_o(i,f) = sqrt2 sin(2 pi (f - N/4) tau_i / N),  f < N/4,
// whose singular values together are those of W.  Each is decomposed here by
// an FP64 one-sided Jacobi SVD (Hestenes 1958; parallel round-robin ordering as
// in Brent & Luk 1985) on the GPU, one CTA per block.  The host then merges the
// two spectra, picks K, and packs the cropped bases p_hat (Eq. 7) and the lag
// dictionary for the kernels.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <numeric>

#include "fcc_internal.h"

namespace fcc {
namespace {

constexpr int kJacobiThreads = 1024;
constexpr int kMaxSweeps = 60;

// cos/sin of pi * n / d for integers n, d > 0, with n reduced exactly mod 2d
// so that the FP64 sincospi call sees an argument in [0, 2).
__device__ __forceinline__ void sincospi_ratio(long long n, long long d, double *s, double *c)
{
    long long p = 2 * d;
    long long r = n % p;
    if (r < 0) r += p;
    sincospi((double)r / (double)d, s, c);
}

// A_e [I][Q+1] and A_o [I][Q]; tau_i = (i - L den)/den, so
// 2 pi (f - Q) tau_i / N = pi * 2 (f - Q) (i - L den) / (den N).
__global__ void build_halves_kernel(int I, int Ld, int den, int N, int Q, double *Ae, double *Ao)
{
    int i = blockIdx.y;
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= I || f > Q) return;
    long long m = (long long)i - Ld;
    long long num = 2LL * (f - Q) * m;
    double s, c;
    sincospi_ratio(num, (long long)den * N, &s, &c);
    const double r2 = 1.4142135623730950488;
    Ae[(size_t)i * (Q + 1) + f] = (f < Q ? r2 : 1.0) * c;
    if (f < Q) Ao[(size_t)i * Q + f] = r2 * s;
}

// The split form's matrices C = Re W and S = Im W (Eq. 3), [I][N/2 + 1]:
// 2 pi f tau_i / N = pi * 2 f (i - L den) / (den N).
__global__ void build_reim_kernel(int I, int Ld, int den, int N, int B, double *Ac, double *As)
{
    int i = blockIdx.y;
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= I || f >= B) return;
    double s, c;
    sincospi_ratio(2LL * f * ((long long)i - Ld), (long long)den * N, &s, &c);
    Ac[(size_t)i * B + f] = c;
    As[(size_t)i * B + f] = s;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One-sided Jacobi on the n row vectors x_k (length len) of X [n][len]:
// rotations x_p <- c x_p - s x_q, x_q <- s x_p + c x_q make the rows mutually
// orthogonal.  The same rotations are applied to the rows of J (identity at
// the start), so at convergence X = J A with J orthogonal and rows y_k of X
// orthogonal; hence A = J^T X = sum_k J[k][:]^T y_k, i.e. u_k = J[k][:],
// sigma_k = |y_k| and v_k = y_k / sigma_k.  Block b of the grid works on job b.
struct JacobiJob {
    double *X;
    double *J;
    int n, len;
    int *sweeps;  // out: sweeps used, or -1 if not converged
};

__global__ void __launch_bounds__(kJacobiThreads) jacobi_svd_kernel(JacobiJob j0, JacobiJob j1,
                                                                    double tiny2)
{
    JacobiJob job = blockIdx.x == 0 ? j0 : j1;
    const int n = job.n, len = job.len;
    double *X = job.X, *J = job.J;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) J[e] = (e / n == e % n) ? 1.0 : 0.0;
    __shared__ int rotated;
    const int np = n + (n & 1);  // players in the round-robin, one phantom if n is odd
    int sweep = 0;
    bool done = false;
    __syncthreads();
    for (; sweep < kMaxSweeps && !done; ++sweep) {
        if (threadIdx.x == 0) rotated = 0;
        __syncthreads();
        for (int r = 0; r < np - 1; ++r) {
            for (int k = warp; k < np / 2; k += nwarps) {
                int p, q;
                if (k == 0) {
                    p = 0;
                    q = r % (np - 1) + 1;
                } else {
                    p = (r + k) % (np - 1) + 1;
                    q = ((r - k) % (np - 1) + (np - 1)) % (np - 1) + 1;
                }
                if (p >= n || q >= n) continue;
                double *xp = X + (size_t)p * len, *xq = X + (size_t)q * len;
                double a = 0, b = 0, g = 0;
                for (int t = lane; t < len; t += 32) {
                    double u = xp[t], v = xq[t];
                    a = fma(u, u, a);
                    b = fma(v, v, b);
                    g = fma(u, v, g);
                }
                a = warp_sum(a);
                b = warp_sum(b);
                g = warp_sum(g);
                // skip pairs already orthogonal to working precision and pairs
                // holding a vector that is negligible against ||A||_F
                if (a <= tiny2 || b <= tiny2 || fabs(g) <= 1e-15 * sqrt(a * b)) continue;
                double zeta = (b - a) / (2.0 * g);
                double t_ = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + hypot(1.0, zeta));
                double c = 1.0 / sqrt(1.0 + t_ * t_), s = c * t_;
                for (int t = lane; t < len; t += 32) {
                    double u = xp[t], v = xq[t];
                    xp[t] = c * u - s * v;
                    xq[t] = s * u + c * v;
                }
                double *jp = J + (size_t)p * n, *jq = J + (size_t)q * n;
                for (int t = lane; t < n; t += 32) {
                    double u = jp[t], v = jq[t];
                    jp[t] = c * u - s * v;
                    jq[t] = s * u + c * v;
                }
                if (lane == 0) rotated = 1;
            }
            __syncthreads();
        }
        done = (rotated == 0);
        __syncthreads();
    }
    if (threadIdx.x == 0) *job.sweeps = done ? sweep : -1;
}

struct Vec {
    double sigma;
    int parity;  // 0 even, 1 odd
    int idx;     // row within its block
};

// Build the two halves of W and run the Jacobi SVD of each (one CTA per half).
void launch_basis_kernels(const fcc_plan_info_t &in, double *d_Ae, double *d_Ao, double *d_Je, double *d_Jo,
                          int *d_sw, cudaStream_t st)
{
    const int I = in.I, Q = in.Q;
    dim3 gb((Q + 1 + 127) / 128, I);
    build_halves_kernel<<<gb, 128, 0, st>>>(I, in.L * in.den, in.den, in.N, Q, d_Ae, d_Ao);
    // ||A||_F^2 = I (N/2 + 1) per block at most; vectors below 1e-30 of it are noise
    double tiny2 = 1e-30 * (double)I * (double)(in.N / 2 + 1);
    JacobiJob je{d_Ae, d_Je, I, Q + 1, d_sw};
    JacobiJob jo{d_Ao, d_Jo, I, Q, d_sw + 1};
    jacobi_svd_kernel<<<2, kJacobiThreads, 0, st>>>(je, jo, tiny2);
}

}  // namespace

// Process-wide cache of finished bases: the bases depend only on N, the lag
// grid and the K rule (not on the array geometry or fs), so plans that share a
// key -- e.g. the arrays of a batch -- share one construction.
struct BasisKey {
    int dev, N, I, den, K_req;
    double energy;
    int form;
    bool operator<(const BasisKey &o) const
    {
        if (form != o.form) return form < o.form;
        if (dev != o.dev) return dev < o.dev;
        if (N != o.N) return N < o.N;
        if (I != o.I) return I < o.I;
        if (den != o.den) return den < o.den;
        if (K_req != o.K_req) return K_req < o.K_req;
        return energy < o.energy;
    }
};
struct BasisEntry {
    int K, KE, KO;
    std::vector<double> s_even, s_odd, Pe, Po, Ue, Uo;
};
static std::mutex g_basis_mu;
static std::map<BasisKey, BasisEntry> g_basis_cache;

static fcc_status_t build_plan_bases_uncached(fcc_plan *plan, int K_req, double energy);

fcc_status_t build_plan_bases(fcc_plan *plan, int K_req, double energy)
{
    fcc_plan_info_t &in = plan->info;
    const BasisKey key{plan->device, in.N, in.I, in.den, K_req > 0 ? K_req : 0, K_req > 0 ? 0.0 : energy, in.form};
    {
        std::lock_guard<std::mutex> lk(g_basis_mu);
        auto it = g_basis_cache.find(key);
        if (it != g_basis_cache.end()) {
            const BasisEntry &b = it->second;
            in.K = b.K;
            in.K_even = b.KE;
            in.K_odd = b.KO;
            plan->s_even = b.s_even;
            plan->s_odd = b.s_odd;
            plan->Pe = b.Pe;
            plan->Po = b.Po;
            plan->Ue = b.Ue;
            plan->Uo = b.Uo;
            return FCC_OK;
        }
    }
    fcc_status_t st = build_plan_bases_uncached(plan, K_req, energy);
    if (st != FCC_OK) return st;
    std::lock_guard<std::mutex> lk(g_basis_mu);
    g_basis_cache[key] = BasisEntry{in.K, in.K_even, in.K_odd, plan->s_even, plan->s_odd,
                                    plan->Pe, plan->Po, plan->Ue, plan->Uo};
    return FCC_OK;
}

static fcc_status_t build_reim_bases(fcc_plan *plan, int K_req, double energy);

static fcc_status_t build_plan_bases_uncached(fcc_plan *plan, int K_req, double energy)
{
    fcc_plan_info_t &in = plan->info;
    if (in.form == FCC_FORM_REIM_SPLIT) return build_reim_bases(plan, K_req, energy);
    const int I = in.I, Q = in.Q, nE = Q + 1, nO = Q;
    double *d_Ae = nullptr, *d_Ao = nullptr, *d_Je = nullptr, *d_Jo = nullptr;
    int *d_sw = nullptr;
    auto cleanup = [&]() {
        cudaFree(d_Ae);
        cudaFree(d_Ao);
        cudaFree(d_Je);
        cudaFree(d_Jo);
        cudaFree(d_sw);
    };
    size_t bytes = sizeof(double) * ((size_t)I * nE + (size_t)I * nO + 2 * (size_t)I * I);
    if (cudaMalloc(&d_Ae, sizeof(double) * (size_t)I * nE) != cudaSuccess ||
        cudaMalloc(&d_Ao, sizeof(double) * (size_t)I * nO) != cudaSuccess ||
        cudaMalloc(&d_Je, sizeof(double) * (size_t)I * I) != cudaSuccess ||
        cudaMalloc(&d_Jo, sizeof(double) * (size_t)I * I) != cudaSuccess ||
        cudaMalloc(&d_sw, 2 * sizeof(int)) != cudaSuccess) {
        cleanup();
        (void)cudaGetLastError();
        return fail(FCC_ERR_OOM, "plan workspace (" + std::to_string(bytes) + " bytes)");
    }
    launch_basis_kernels(in, d_Ae, d_Ao, d_Je, d_Jo, d_sw, 0);
    std::vector<double> Xe((size_t)I * nE), Xo((size_t)I * nO), Je((size_t)I * I), Jo((size_t)I * I);
    int sw[2] = {0, 0};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(Xe.data(), d_Ae, sizeof(double) * Xe.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(Xo.data(), d_Ao, sizeof(double) * Xo.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(Je.data(), d_Je, sizeof(double) * Je.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(Jo.data(), d_Jo, sizeof(double) * Jo.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(sw, d_sw, sizeof(sw), cudaMemcpyDeviceToHost);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "plan basis construction");
    if (sw[0] < 0 || sw[1] < 0) return fail(FCC_ERR_NOT_CONVERGED, "Jacobi SVD did not converge");
    return finish_plan_bases(plan, Xe, Xo, Je, Jo, K_req, energy);
}

// Host part of the basis construction, from the rotated rows (sigma v) and the
// accumulated rotations (u) of both halves: merge the singular values, pick K,
// fix signs and write the cropped bases and the dictionary into the plan.
fcc_status_t finish_plan_bases(fcc_plan *plan, const std::vector<double> &Xe, const std::vector<double> &Xo,
                               const std::vector<double> &Je, const std::vector<double> &Jo, int K_req,
                               double energy)
{
    fcc_plan_info_t &in = plan->info;
    const int I = in.I, Q = in.Q, nE = Q + 1, nO = Q;

    // singular values = row norms of the rotated matrices
    auto norms = [](const std::vector<double> &X, int n, int len) {
        std::vector<double> s(n);
        for (int k = 0; k < n; ++k) {
            double a = 0;
            for (int t = 0; t < len; ++t) a += X[(size_t)k * len + t] * X[(size_t)k * len + t];
            s[k] = std::sqrt(a);
        }
        return s;
    };
    std::vector<double> se = norms(Xe, I, nE), so = norms(Xo, I, nO);
    std::vector<Vec> all;
    for (int k = 0; k < I; ++k) all.push_back({se[k], 0, k});
    for (int k = 0; k < I; ++k) all.push_back({so[k], 1, k});
    std::stable_sort(all.begin(), all.end(), [](const Vec &a, const Vec &b) { return a.sigma > b.sigma; });
    auto sorted_block = [](std::vector<double> s, int keep) {
        std::sort(s.begin(), s.end(), std::greater<double>());
        s.resize(std::min<size_t>(s.size(), keep));
        return s;
    };
    plan->s_even = sorted_block(se, std::min(I, nE));
    plan->s_odd = sorted_block(so, std::min(I, nO));

    // K: requested, or the smallest K holding `energy` of sum(s^2) (Sec. 4 leaves
    // K to the user), extended over singular values tied with the K-th.
    double tot = 0;
    for (auto &v : all) tot += v.sigma * v.sigma;
    int n_all = (int)all.size();
    int K = K_req;
    if (K <= 0) {
        double acc = 0;
        K = n_all;
        for (int k = 0; k < n_all; ++k) {
            acc += all[k].sigma * all[k].sigma;
            if (acc >= energy * tot) {
                K = k + 1;
                break;
            }
        }
        while (K < n_all && all[K - 1].sigma - all[K].sigma <= 1e-12 * all[K - 1].sigma) ++K;
    }
    if (K > n_all) return fail(FCC_ERR_INVALID_ARG, "K exceeds the number of singular values");
    if (all[K - 1].sigma <= 1e-12 * all[0].sigma)
        return fail(FCC_ERR_INVALID_ARG, "K exceeds the numerical rank of W");

    std::vector<const Vec *> ev, ov;
    for (int k = 0; k < K; ++k) (all[k].parity == 0 ? ev : ov).push_back(&all[k]);
    const int KE = (int)ev.size(), KO = (int)ov.size();
    in.K = K;
    in.K_even = KE;
    in.K_odd = KO;
    plan->Pe.assign((size_t)KE * nE, 0.0);
    plan->Po.assign((size_t)KO * nO, 0.0);
    plan->Ue.assign((size_t)I * KE, 0.0);
    plan->Uo.assign((size_t)I * KO, 0.0);
    const double r2 = std::sqrt(2.0);
    // For each kept vector: sigma v = y (the rotated row), u = J row.  Canonical
    // sign: the largest-magnitude entry of v (lowest index on ties) is positive.
    auto emit = [&](const Vec *v, const std::vector<double> &X, const std::vector<double> &Jm,
                    int len, int col, int K_par, std::vector<double> &Pm, std::vector<double> &Um,
                    bool even) {
        const double *y = &X[(size_t)v->idx * len];
        const double *u = &Jm[(size_t)v->idx * I];
        int am = 0;
        for (int t = 1; t < len; ++t)
            if (std::fabs(y[t]) > std::fabs(y[am])) am = t;
        double sg = y[am] < 0 ? -1.0 : 1.0;
        for (int t = 0; t < len; ++t) {
            double w = even ? (t < Q ? r2 : 1.0) : r2;
            Pm[(size_t)col * len + t] = sg * y[t] / w;
        }
        for (int i = 0; i < I; ++i) Um[(size_t)i * K_par + col] = sg * u[i];
    };
    for (int k = 0; k < KE; ++k) emit(ev[k], Xe, Je, nE, k, KE, plan->Pe, plan->Ue, true);
    for (int k = 0; k < KO; ++k) emit(ov[k], Xo, Jo, nO, k, KO, plan->Po, plan->Uo, false);
    return FCC_OK;
}

// The split form: C = Re W and S = Im W each get their own FP64 Jacobi SVD on
// the GPU and their own rank (the energy rule on that matrix's singular values,
// extended over ties, or K_req for both).  Kept vectors: projection rows
// sigma_k v_k into Pe (C) / Po (S) over all N/2 + 1 bins, left vectors u_k into
// Ue / Uo, with the canonical sign of the folded form.
static fcc_status_t build_reim_bases(fcc_plan *plan, int K_req, double energy)
{
    fcc_plan_info_t &in = plan->info;
    const int I = in.I, B = in.B;
    double *d_A[2] = {nullptr, nullptr}, *d_J[2] = {nullptr, nullptr};
    int *d_sw = nullptr;
    auto cleanup = [&]() {
        for (int b = 0; b < 2; ++b) {
            cudaFree(d_A[b]);
            cudaFree(d_J[b]);
        }
        cudaFree(d_sw);
    };
    bool ok = cudaMalloc(&d_sw, 2 * sizeof(int)) == cudaSuccess;
    for (int b = 0; b < 2 && ok; ++b)
        ok = cudaMalloc(&d_A[b], sizeof(double) * (size_t)I * B) == cudaSuccess &&
             cudaMalloc(&d_J[b], sizeof(double) * (size_t)I * I) == cudaSuccess;
    if (!ok) {
        cleanup();
        (void)cudaGetLastError();
        return fail(FCC_ERR_OOM, "split-form plan workspace");
    }
    dim3 gb((B + 127) / 128, I);
    build_reim_kernel<<<gb, 128>>>(I, in.L * in.den, in.den, in.N, B, d_A[0], d_A[1]);
    const double tiny2 = 1e-30 * (double)I * (double)B;
    jacobi_svd_kernel<<<2, kJacobiThreads>>>(JacobiJob{d_A[0], d_J[0], I, B, d_sw},
                                            JacobiJob{d_A[1], d_J[1], I, B, d_sw + 1}, tiny2);
    std::vector<double> X[2], J[2];
    int sw[2] = {0, 0};
    cudaError_t e = cudaGetLastError();
    for (int b = 0; b < 2; ++b) {
        X[b].resize((size_t)I * B);
        J[b].resize((size_t)I * I);
        if (e == cudaSuccess) e = cudaMemcpy(X[b].data(), d_A[b], sizeof(double) * X[b].size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(J[b].data(), d_J[b], sizeof(double) * J[b].size(), cudaMemcpyDeviceToHost);
    }
    if (e == cudaSuccess) e = cudaMemcpy(sw, d_sw, sizeof(sw), cudaMemcpyDeviceToHost);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "split-form basis construction");
    if (sw[0] < 0 || sw[1] < 0) return fail(FCC_ERR_NOT_CONVERGED, "Jacobi SVD did not converge");
    int K[2];
    std::vector<double> P[2], U[2];
    for (int b = 0; b < 2; ++b) {
        std::vector<double> sig(I);
        std::vector<int> order(I);
        for (int k = 0; k < I; ++k) {
            double a = 0;
            for (int t = 0; t < B; ++t) a += X[b][(size_t)k * B + t] * X[b][(size_t)k * B + t];
            sig[k] = std::sqrt(a);
            order[k] = k;
        }
        std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return sig[a] > sig[c]; });
        std::vector<double> sorted(I);
        double tot = 0;
        for (int k = 0; k < I; ++k) {
            sorted[k] = sig[order[k]];
            tot += sorted[k] * sorted[k];
        }
        int Kb = K_req;
        if (Kb <= 0) {
            double acc = 0;
            Kb = I;
            for (int k = 0; k < I; ++k) {
                acc += sorted[k] * sorted[k];
                if (acc >= energy * tot) {
                    Kb = k + 1;
                    break;
                }
            }
            while (Kb < I && sorted[Kb - 1] - sorted[Kb] <= 1e-12 * sorted[Kb - 1]) ++Kb;
        }
        if (Kb > I || sorted[Kb - 1] <= 1e-12 * sorted[0])
            return fail(FCC_ERR_INVALID_ARG, "K exceeds the numerical rank of the cosine or sine matrix");
        K[b] = Kb;
        sorted.resize(std::min(I, B));
        (b == 0 ? plan->s_even : plan->s_odd) = sorted;
        P[b].assign((size_t)Kb * B, 0.0);
        U[b].assign((size_t)I * Kb, 0.0);
        for (int k = 0; k < Kb; ++k) {
            const double *y = &X[b][(size_t)order[k] * B];
            const double *u = &J[b][(size_t)order[k] * I];
            int am = 0;
            for (int t = 1; t < B; ++t)
                if (std::fabs(y[t]) > std::fabs(y[am])) am = t;
            const double sg = y[am] < 0 ? -1.0 : 1.0;
            for (int t = 0; t < B; ++t) P[b][(size_t)k * B + t] = sg * y[t];
            for (int i = 0; i < I; ++i) U[b][(size_t)i * Kb + k] = sg * u[i];
        }
    }
    in.K_even = K[0];
    in.K_odd = K[1];
    in.K = K[0] + K[1];
    plan->Pe = P[0];
    plan->Po = P[1];
    plan->Ue = U[0];
    plan->Uo = U[1];
    return FCC_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free basis construction (fcc_plan_bases_noalloc).  The working
// matrices of the two Jacobi SVDs live in one static device array instead of
// cudaMalloc'd memory.  Layout (doubles): [0, 32) two int sweep counters,
// then A_e [I][Q+1], A_o [I][Q], J_e [I][I], J_o [I][I].
}  // namespace fcc

// 4 MiB, held by every GPU that loads this library until the process exits.
static constexpr size_t kNoAllocDoubles = size_t(1) << 19;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

namespace fcc {
namespace {

constexpr size_t kNoAllocHeader = 32;  // 256 bytes
std::mutex g_noalloc_mu;
double *g_noalloc_addr[256] = {};

// Device address of the static array on the current device (looked up once
// per device; the host-side symbol is not a device address).
fcc_status_t noalloc_scratch(int dev, double **out)
{
    if (dev < 0 || dev >= 256) return fail(FCC_ERR_UNSUPPORTED, "device ordinal above 255");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_addr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_addr[dev];
    return FCC_OK;
}

}  // namespace
}  // namespace fcc

extern "C" fcc_status_t fcc_plan_bases_noalloc(const fcc_plan_desc_t *desc, fcc_plan_info_t *info,
                                               double *s_even, double *s_odd, double *Pe, double *Po,
                                               double *Ue, double *Uo, void *stream)
{
    using namespace fcc;
    fcc_plan tmp;  // host-side fields only; nothing on the device is created
    int dev = 0;
    fcc_status_t st = plan_info_from_desc(desc, tmp.info, dev);
    if (st != FCC_OK) return st;
    if (tmp.info.form != FCC_FORM_FOLDED) return fail(FCC_ERR_UNSUPPORTED, "the allocation-free build is for the folded form");
    const fcc_plan_info_t &in = tmp.info;
    const size_t I = in.I, Q = in.Q;
    const size_t need = kNoAllocHeader + I * (2 * Q + 1) + 2 * I * I;
    if (need > kNoAllocDoubles)
        return fail(FCC_ERR_UNSUPPORTED,
                    "grid needs " + std::to_string(need * 8) + " bytes of scratch; the static array holds " +
                        std::to_string(kNoAllocDoubles * 8) + " (I (N/2 + 1) + 2 I^2 + 32 <= 524288 doubles)");
    DeviceScope scope(dev);
    if (!scope.ok) return fail(FCC_ERR_CUDA, "cudaSetDevice failed");
    double *base = nullptr;
    st = noalloc_scratch(dev, &base);
    if (st != FCC_OK) return st;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    int *d_sw = reinterpret_cast<int *>(base);
    double *d_Ae = base + kNoAllocHeader;
    double *d_Ao = d_Ae + I * (Q + 1);
    double *d_Je = d_Ao + I * Q;
    double *d_Jo = d_Je + I * I;
    // the sweep counters start at -1 ("not converged"), so stale contents of a
    // previous call can never pass for this call's result
    FCC_CUDA_TRY(cudaMemsetAsync(d_sw, 0xff, 2 * sizeof(int), cs));
    launch_basis_kernels(in, d_Ae, d_Ao, d_Je, d_Jo, d_sw, cs);
    FCC_CUDA_TRY(cudaGetLastError());
    std::vector<double> Xe(I * (Q + 1)), Xo(I * Q), Je(I * I), Jo(I * I);
    int sw[2] = {-1, -1};
    FCC_CUDA_TRY(cudaMemcpyAsync(Xe.data(), d_Ae, sizeof(double) * Xe.size(), cudaMemcpyDeviceToHost, cs));
    FCC_CUDA_TRY(cudaMemcpyAsync(Xo.data(), d_Ao, sizeof(double) * Xo.size(), cudaMemcpyDeviceToHost, cs));
    FCC_CUDA_TRY(cudaMemcpyAsync(Je.data(), d_Je, sizeof(double) * Je.size(), cudaMemcpyDeviceToHost, cs));
    FCC_CUDA_TRY(cudaMemcpyAsync(Jo.data(), d_Jo, sizeof(double) * Jo.size(), cudaMemcpyDeviceToHost, cs));
    FCC_CUDA_TRY(cudaMemcpyAsync(sw, d_sw, sizeof(sw), cudaMemcpyDeviceToHost, cs));
    FCC_CUDA_TRY(cudaStreamSynchronize(cs));
    if (sw[0] < 0 || sw[1] < 0) return fail(FCC_ERR_NOT_CONVERGED, "Jacobi SVD did not converge");
    st = finish_plan_bases(&tmp, Xe, Xo, Je, Jo, desc->K, desc->energy > 0 ? desc->energy : 0.999);
    if (st != FCC_OK) return st;
    if (info) *info = tmp.info;
    if (s_even) std::copy(tmp.s_even.begin(), tmp.s_even.end(), s_even);
    if (s_odd) std::copy(tmp.s_odd.begin(), tmp.s_odd.end(), s_odd);
    if (Pe) std::copy(tmp.Pe.begin(), tmp.Pe.end(), Pe);
    if (Po) std::copy(tmp.Po.begin(), tmp.Po.end(), Po);
    if (Ue) std::copy(tmp.Ue.begin(), tmp.Ue.end(), Ue);
    if (Uo) std::copy(tmp.Uo.begin(), tmp.Uo.end(), Uo);
    return FCC_OK;
}
