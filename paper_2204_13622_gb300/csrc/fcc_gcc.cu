// fcc_gcc.cu -- same-GPU GCC-PHAT baseline (Sec. 3).
//
// y(tau) of eq. 2 on the 1/r grid through an r-times zero-padded real inverse
// FFT: for the half spectrum R'' of length rN/2+1 with R''(f) = R_hat(f) for
// f <= N/2 and 0 above, the unnormalised C2R output at sample n is
//   R''(0) + 2 Re sum_{f=1}^{N/2} R_hat(f) e^{j 2 pi f n/(rN)}      (r > 1),
// so doubling the (real) DC bin -- and for r = 1 also the Nyquist bin -- makes
// it exactly y(n/r) of eq. 2.  Pipeline per chunk of frames:
//   PHAT kernel (pair spectra, padded, to HBM) -> cufftExecC2R (batched) ->
//   gather of the I grid lags + argmax (lowest index on ties).
#include <cfloat>
#include <cufft.h>

#include "fcc_internal.h"

namespace fcc {
namespace {

struct GccState {
    int device = -1;
    long long chunk = 0;  // frames per chunk
    int r = 0;
    cufftHandle fft = 0;
    bool fft_ok = false;
    cufftComplex *pad = nullptr;  // [chunk*P][rN/2+1]
    float *out = nullptr;         // [chunk*P][rN]
    int2 *pairs = nullptr;        // [P]
};

__device__ __forceinline__ float2 unit(float2 x)
{
    float s = fmaf(x.x, x.x, x.y * x.y);
    if (s >= FLT_MIN && s <= FLT_MAX) {
        float r = rsqrtf(s);
        return make_float2(x.x * r, x.y * r);
    }
    if (!(fabsf(x.x) <= FLT_MAX) || !(fabsf(x.y) <= FLT_MAX)) return make_float2(0.f, 0.f);
    float m = fmaxf(fabsf(x.x), fabsf(x.y));
    if (m == 0.f) return make_float2(0.f, 0.f);
    float a = x.x / m, b = x.y / m;
    float r = rsqrtf(fmaf(a, a, b * b));
    return make_float2(a * r, b * r);
}

// One thread per (pair-frame, padded bin).
__global__ void gcc_phat_pad_kernel(const float2 *__restrict__ X, long long t0, long long nframes, int M, int B,
                                    int P, int RB, int r, const int2 *__restrict__ pairs,
                                    cufftComplex *__restrict__ pad, unsigned *err)
{
    const long long total = nframes * P * (long long)RB;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(e % RB);
        const long long pf = e / RB;
        const long long t = pf / P;
        const int p = (int)(pf - t * P);
        cufftComplex v = make_float2(0.f, 0.f);
        if (f < B) {
            const int2 ij = pairs[p];
            const float2 *Xt = X + (size_t)(t0 + t) * M * B;
            const float2 xi = Xt[(size_t)ij.x * B + f], xj = Xt[(size_t)ij.y * B + f];
            if (!(fabsf(xi.x) <= FLT_MAX && fabsf(xi.y) <= FLT_MAX && fabsf(xj.x) <= FLT_MAX &&
                  fabsf(xj.y) <= FLT_MAX))
                atomicOr(err, kErrNonFinite);
            const float2 ui = unit(xi), uj = unit(xj);
            v.x = fmaf(ui.x, uj.x, ui.y * uj.y);
            v.y = fmaf(ui.y, uj.x, -(ui.x * uj.y));
            if (f == 0 || (r == 1 && f == B - 1)) {
                v.x *= 2.f;  // counted twice by eq. 2; C2R takes these bins real
                v.y = 0.f;
            }
        }
        pad[e] = v;
    }
}

// One thread per pair-frame: gather the grid lags n = (i - center) mod rN.
__global__ void gcc_gather_kernel(const float *__restrict__ out, long long t0, long long nframes, int P, int RN,
                                  int I, int center, int *idx, float *peak, float *corr)
{
    const long long npf = nframes * P;
    for (long long pf = blockIdx.x * (long long)blockDim.x + threadIdx.x; pf < npf;
         pf += (long long)gridDim.x * blockDim.x) {
        const float *y = out + (size_t)pf * RN;
        float best = -FLT_MAX;
        int bi = 0;
        const size_t o = (size_t)t0 * P + pf;
        for (int i = 0; i < I; ++i) {
            int n = i - center;
            if (n < 0) n += RN;
            const float v = y[n];
            if (i == 0 || v > best) {
                best = v;
                bi = i;
            }
            if (corr) corr[o * I + i] = v;
        }
        idx[o] = bi;
        peak[o] = best;
    }
}

fcc_status_t build_state(fcc_plan *plan, GccState *&gs)
{
    const fcc_plan_info_t &in = plan->info;
    gs = new GccState();
    plan->gcc_state = gs;
    gs->device = plan->device;
    gs->r = in.den;
    const long long RB = (long long)in.den * in.N / 2 + 1;
    const long long RN = (long long)in.den * in.N;
    // keep each workspace near 1 GiB
    gs->chunk = std::max<long long>(1, (1LL << 27) / ((long long)in.P * RB));
    std::vector<int2> pr;
    for (int i = 0; i < in.M; ++i)
        for (int j = i + 1; j < in.M; ++j) pr.push_back(make_int2(i, j));
    FCC_CUDA_TRY(cudaMalloc(&gs->pairs, pr.size() * sizeof(int2)));
    FCC_CUDA_TRY(cudaMemcpy(gs->pairs, pr.data(), pr.size() * sizeof(int2), cudaMemcpyHostToDevice));
    FCC_CUDA_TRY(cudaMalloc(&gs->pad, (size_t)gs->chunk * in.P * RB * sizeof(cufftComplex)));
    FCC_CUDA_TRY(cudaMemset(gs->pad, 0, (size_t)gs->chunk * in.P * RB * sizeof(cufftComplex)));
    FCC_CUDA_TRY(cudaMalloc(&gs->out, (size_t)gs->chunk * in.P * RN * sizeof(float)));
    int n[1] = {(int)RN};
    int inembed[1] = {(int)RB}, onembed[1] = {(int)RN};
    cufftResult cr = cufftPlanMany(&gs->fft, 1, n, inembed, 1, (int)RB, onembed, 1, (int)RN, CUFFT_C2R,
                                   (int)(gs->chunk * in.P));
    if (cr != CUFFT_SUCCESS) return fail(FCC_ERR_CUDA, "cufftPlanMany failed (" + std::to_string((int)cr) + ")");
    gs->fft_ok = true;
    return FCC_OK;
}

// The plan's GCC workspace, created on first use; a failed creation frees what
// it had allocated, so a later call starts again from nothing.
fcc_status_t ensure_state(fcc_plan *plan, GccState *&gs)
{
    gs = static_cast<GccState *>(plan->gcc_state);
    if (gs) return FCC_OK;
    const fcc_status_t st = build_state(plan, gs);
    if (st != FCC_OK) {
        gcc_destroy(plan);
        gs = nullptr;
    }
    return st;
}

}  // namespace

fcc_status_t gcc_run(fcc_plan *plan, const float2 *spectra, long long T, int *idx, float *peak, float *corr,
                     cudaStream_t st)
{
    GccState *gs = nullptr;
    fcc_status_t s = ensure_state(plan, gs);
    if (s != FCC_OK) return s;
    const fcc_plan_info_t &in = plan->info;
    const int RB = in.den * in.N / 2 + 1, RN = in.den * in.N;
    if (cufftSetStream(gs->fft, st) != CUFFT_SUCCESS) return fail(FCC_ERR_CUDA, "cufftSetStream failed");
    for (long long t0 = 0; t0 < T; t0 += gs->chunk) {
        const long long n = std::min(gs->chunk, T - t0);
        const long long work = n * in.P * (long long)RB;
        const int blocks = (int)std::min<long long>((work + 255) / 256, (long long)plan->num_sms * 16);
        gcc_phat_pad_kernel<<<blocks, 256, 0, st>>>(spectra, t0, n, in.M, in.B, in.P, RB, gs->r, gs->pairs, gs->pad,
                                                    plan->d_err);
        // the plan was made for a full chunk; the rows past n of a short last
        // chunk hold stale finite data and are never gathered
        if (cufftExecC2R(gs->fft, gs->pad, gs->out) != CUFFT_SUCCESS) return fail(FCC_ERR_CUDA, "cufftExecC2R failed");
        const long long npf = n * in.P;
        const int gblocks = (int)std::min<long long>((npf + 255) / 256, (long long)plan->num_sms * 16);
        gcc_gather_kernel<<<gblocks, 256, 0, st>>>(gs->out, t0, n, in.P, RN, in.I, in.center, idx, peak, corr);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "gcc kernels");
    }
    return FCC_OK;
}

void gcc_destroy(fcc_plan *plan)
{
    GccState *gs = static_cast<GccState *>(plan->gcc_state);
    if (!gs) return;
    if (gs->fft_ok) cufftDestroy(gs->fft);
    cudaFree(gs->pad);
    cudaFree(gs->out);
    cudaFree(gs->pairs);
    delete gs;
    plan->gcc_state = nullptr;
}

}  // namespace fcc
