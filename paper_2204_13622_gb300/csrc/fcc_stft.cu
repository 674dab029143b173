// fcc_stft.cu -- the STFT front-end (Sec. 2 starts from the microphones' STFT
// X_m(t, f)): periodic Hann window, frames of N samples every hop samples, and
// per (frame, microphone) a real FFT of N points, done as an N/2-point complex
// FFT of the packed samples z[j] = x[2j] + i x[2j + 1] followed by the split
//   X[k] = E[k] + e^{-2 pi i k / N} O[k],  E = (Z[k] + Z*[H-k]) / 2,
//   O = (Z[k] - Z*[H-k]) / 2i,  H = N/2, k = 0..H (Z periodic in H).
// The complex FFT of H = 32 R1 points is the four-step form with n = 32 n1 + n2
// and k = k1 + R1 k2: lane n2 holds z[32 n1 + n2] for n1 < R1 in registers,
//   1. an R1-point DFT over n1 in registers (radix-2, decimation in frequency:
//      register r ends with k1 = bitrev(r));
//   2. the twiddle W_H^{n2 k1};
//   3. a 32-point DFT over n2 across the warp's lanes (five radix-2 stages with
//      butterfly partners from __shfl_xor_sync; lane p ends with k2 = bitrev(p));
//   4. one store into shared memory at index i + i / R1 (bank-conflict free for a
//      fixed register), then the split above reads Z[k] and Z[H - k].
//
// For N = 512 (R1 = 8) step 3 is instead 8 x 4: one shared-memory transpose, an
// 8-point DFT in registers, the twiddles W_32^{b c}, and a 4-point DFT over two
// shuffle stages (fewer shuffles and twiddle products than five lane stages).
//
// stft_kernel<N, S>: one warp per (frame, microphone); twiddles and the window
// are tables computed in FP64 on the host.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fcc_internal.h"
#include "fcc_stft.h"

namespace fcc {
namespace {

constexpr int kStftWarps = 8;
// spectra per device chunk (recommended workspace): measured on the 8-mic circle,
// 2^20 frames, per step: 64 MB 22.4 ms, 256 MB 19.2 ms, 1 GB 18.0 ms, 4 GB 17.6 ms
// (fewer launches count for more than keeping a chunk in L2)
constexpr long long kPcmChunkBytes = 1LL << 30;
constexpr long long kHostChunkFrames = 1LL << 16;  // frames per host chunk of fcc_tdoa_pcm_host

struct StftParams {
    const void *pcm;
    int type;           // FCC_PCM_F32 or FCC_PCM_S16
    long long T;
    int M, hop;
    const float *tab;   // [2H] FFT twiddles e^{-2 pi i m / H}, [2(H+1)] split twiddles e^{-2 pi i k / N}, [N] window
    float2 *out;        // [T][M][H + 1]
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }
__host__ __device__ constexpr int bitrev(int x, int bits) { return bits == 0 ? 0 : ((x & 1) << (bits - 1)) | bitrev(x >> 1, bits - 1); }

template <int N, typename S>
__global__ void __launch_bounds__(32 * kStftWarps) stft_kernel(const __grid_constant__ StftParams p)
{
    constexpr int H = N / 2, B = H + 1, R1 = H / 32, LB = ilog2(R1);
    extern __shared__ __align__(16) unsigned char sm[];
    float2 *tw = reinterpret_cast<float2 *>(sm);  // [H]: W_H^m
    float2 *sp = tw + H;                          // [H + 1]: W_N^k, padded to H + 2
    float *win = reinterpret_cast<float *>(sp + H + 2);
    float2 *bufs = reinterpret_cast<float2 *>(win + N);  // [warps][H + 32]
    const float2 *tab2 = reinterpret_cast<const float2 *>(p.tab);
    for (int e = threadIdx.x; e < H; e += blockDim.x) tw[e] = tab2[e];
    for (int e = threadIdx.x; e <= H; e += blockDim.x) sp[e] = tab2[H + e];
    for (int e = threadIdx.x; e < N; e += blockDim.x) win[e] = p.tab[2 * H + 2 * (H + 1) + e];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned FULLM = 0xffffffffu;
    float2 *buf = bufs + (size_t)warp * (H + 32);
    const float2 *win2 = reinterpret_cast<const float2 *>(win);
    // per-lane twiddles of the cross-lane stages h = 16, 8, 4, 2 (lower lanes W_{2h}^{p mod h}, upper 1)
    float2 ct[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int h = 16 >> s;
        ct[s] = (lane & h) ? tw[(lane % h) * (16 / h) * (H / 32)] : make_float2(1.f, 0.f);
    }
    const int k2 = (int)(__brev((unsigned)lane) >> 27);
    // N = 512 (R1 = 8): the 32-point DFT is 8 x 4 through a shared-memory transpose;
    // lane (k1, b) = (lane / 4, lane % 4) keeps the twiddles W_32^{b c} for c = bitrev3(q)
    float2 t32[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) t32[q] = tw[((lane & 3) * bitrev(q, 3) * (H / 32)) & (H - 1)];
    const float scale = sizeof(S) == 2 ? 1.f / 32768.f : 1.f;
    const long long items = p.T * p.M;
    const S *pcm = static_cast<const S *>(p.pcm);
    for (long long it = (long long)blockIdx.x * kStftWarps + warp; it < items; it += (long long)gridDim.x * kStftWarps) {
        const long long t = it / p.M;
        const int m = (int)(it - t * p.M);
        const S *x = pcm + (size_t)(t * p.hop) * p.M + m;
        float2 v[R1];
#pragma unroll
        for (int r = 0; r < R1; ++r) {
            const int j = 32 * r + lane;  // z[j] = (w x)[2j] + i (w x)[2j + 1]
            const float2 w = win2[j];
            v[r] = make_float2(w.x * scale * (float)x[(size_t)(2 * j) * p.M], w.y * scale * (float)x[(size_t)(2 * j + 1) * p.M]);
        }
        // 1. R1-point DFT over n1 (decimation in frequency)
#pragma unroll
        for (int h = R1 / 2; h >= 1; h /= 2) {
#pragma unroll
            for (int r = 0; r < R1; ++r) {
                if (r & h) continue;
                const float2 a = v[r], b = v[r + h];
                const int i = r % h;
                v[r] = make_float2(a.x + b.x, a.y + b.y);
                const float2 d = make_float2(a.x - b.x, a.y - b.y);
                v[r + h] = i == 0 ? d : cmul(d, tw[i * (H / (2 * h))]);
            }
        }
        // 2. twiddle W_H^{n2 k1}
#pragma unroll
        for (int r = 1; r < R1; ++r) v[r] = cmul(v[r], tw[lane * bitrev(r, LB)]);
        if constexpr (R1 == 8) {
            // 3. 32-point DFT over n2 = 4 a + b (k2 = c + 8 d): row k1 of the transpose
            //    at stride 36 (conflict-free both ways), an 8-point DFT over a in
            //    registers, W_32^{b c}, then a 4-point DFT over b across lanes
#pragma unroll
            for (int r = 0; r < 8; ++r) buf[bitrev(r, 3) * 36 + lane] = v[r];
            __syncwarp();
            const int k1 = lane >> 2, b = lane & 3;
#pragma unroll
            for (int a = 0; a < 8; ++a) v[a] = buf[k1 * 36 + 4 * a + b];
            __syncwarp();
#pragma unroll
            for (int h = 4; h >= 1; h /= 2) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (q & h) continue;
                    const float2 a = v[q], c = v[q + h];
                    const int i = q % h;
                    v[q] = make_float2(a.x + c.x, a.y + c.y);
                    const float2 d = make_float2(a.x - c.x, a.y - c.y);
                    v[q + h] = i == 0 ? d : cmul(d, tw[i * (8 / (2 * h)) * (H / 8)]);
                }
            }
#pragma unroll
            for (int q = 1; q < 8; ++q) v[q] = cmul(v[q], t32[q]);
#pragma unroll
            for (int h = 2; h >= 1; h /= 2) {
                const float sg = (lane & h) ? -1.f : 1.f;
                const bool rot = h == 2 && (lane & 2) && (lane & 1);  // W_4^1 = -i on the lower half
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float ox = __shfl_xor_sync(FULLM, v[q].x, h), oy = __shfl_xor_sync(FULLM, v[q].y, h);
                    const float2 tv = make_float2(fmaf(sg, v[q].x, ox), fmaf(sg, v[q].y, oy));
                    v[q] = rot ? make_float2(tv.y, -tv.x) : tv;
                }
            }
            // 4. Z[k1 + 8 c + 64 d] (d = bitrev2(b)) at index i + 4 (i >> 6)
            const int d = ((b & 1) << 1) | (b >> 1);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int i = k1 + 8 * bitrev(q, 3) + 64 * d;
                buf[i + 4 * (i >> 6)] = v[q];
            }
        } else {
            // 3. 32-point DFT across the lanes
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                const int h = 16 >> s;
                const float sg = (lane & h) ? -1.f : 1.f;
#pragma unroll
                for (int r = 0; r < R1; ++r) {
                    const float ox = __shfl_xor_sync(FULLM, v[r].x, h), oy = __shfl_xor_sync(FULLM, v[r].y, h);
                    float2 tv = make_float2(fmaf(sg, v[r].x, ox), fmaf(sg, v[r].y, oy));
                    if (s < 4) tv = cmul(tv, ct[s]);
                    v[r] = tv;
                }
            }
            // 4. Z[k1 + R1 k2] into the buffer at index i + i / R1
#pragma unroll
            for (int r = 0; r < R1; ++r) {
                const int i = bitrev(r, LB) + R1 * k2;
                buf[i + (i >> LB)] = v[r];
            }
        }
        __syncwarp();
        // split into the H + 1 bins of the real frame
        float2 *out = p.out + (size_t)it * B;
        for (int k = lane; k <= H; k += 32) {
            const int i0 = k & (H - 1), i1 = (H - k) & (H - 1);
            const float2 zk = R1 == 8 ? buf[i0 + 4 * (i0 >> 6)] : buf[i0 + (i0 >> LB)];
            const float2 zm = R1 == 8 ? buf[i1 + 4 * (i1 >> 6)] : buf[i1 + (i1 >> LB)];
            const float2 E = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
            const float2 O = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));  // (Z[k] - Z*[H-k]) / 2i
            const float2 w = cmul(sp[k], O);
            out[k] = make_float2(E.x + w.x, E.y + w.y);
        }
        __syncwarp();  // the buffer is reused by the next item
    }
}

size_t stft_smem(int N)
{
    const int H = N / 2;
    return (size_t)(H + H + 2) * sizeof(float2) + (size_t)N * sizeof(float) + (size_t)kStftWarps * (H + 32) * sizeof(float2);
}

}  // namespace

// Twiddles and window of the STFT front-end, built when the plan is created (64 <= N <= 2048).
fcc_status_t prepare_stft(fcc_plan *plan)
{
    if (plan->d_stft_tab || plan->info.N < 64 || plan->info.N > 2048) return FCC_OK;
    const int N = plan->info.N, H = N / 2;
    std::vector<float> tab((size_t)2 * H + 2 * (H + 1) + N);
    const double two_pi = 6.283185307179586476925286766559;
    for (int m = 0; m < H; ++m) {
        tab[2 * m] = (float)std::cos(two_pi * m / H);
        tab[2 * m + 1] = (float)-std::sin(two_pi * m / H);
    }
    for (int k = 0; k <= H; ++k) {
        tab[2 * H + 2 * k] = (float)std::cos(two_pi * k / N);
        tab[2 * H + 2 * k + 1] = (float)-std::sin(two_pi * k / N);
    }
    for (int n = 0; n < N; ++n) tab[2 * H + 2 * (H + 1) + n] = (float)(0.5 - 0.5 * std::cos(two_pi * n / N));
    float *d = nullptr;
    FCC_CUDA_TRY(dev_alloc((void **)&d, tab.size() * sizeof(float)));
    cudaError_t e = cudaMemcpy(d, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "cudaMemcpy(stft tables)");
    }
    plan->d_stft_tab = d;
    return FCC_OK;
}

namespace {

template <int N, typename S>
fcc_status_t launch_stft_n(const StftParams &prm, int num_sms, cudaStream_t st)
{
    const size_t smem = stft_smem(N);
    cudaError_t e = cudaFuncSetAttribute(stft_kernel<N, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(stft_kernel)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stft_kernel<N, S>, 32 * kStftWarps, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    const long long need = (prm.T * prm.M + kStftWarps - 1) / kStftWarps;
    const int grid = (int)std::max<long long>(1, std::min<long long>(need, (long long)num_sms * std::max(per_sm, 1)));
    stft_kernel<N, S><<<grid, 32 * kStftWarps, smem, st>>>(prm);
    e = cudaGetLastError();
    return e == cudaSuccess ? FCC_OK : cuda_fail(e, "stft_kernel launch");
}

template <int N>
fcc_status_t launch_stft_t(const StftParams &prm, int num_sms, cudaStream_t st)
{
    return prm.type == FCC_PCM_S16 ? launch_stft_n<N, short>(prm, num_sms, st) : launch_stft_n<N, float>(prm, num_sms, st);
}

fcc_status_t launch_stft(fcc_plan *plan, const void *pcm, int type, long long T, int hop, float2 *out, cudaStream_t st)
{
    if (!plan->d_stft_tab) return fail(FCC_ERR_UNSUPPORTED, "the STFT front-end needs 64 <= N <= 2048");
    StftParams prm{};
    prm.pcm = pcm;
    prm.type = type;
    prm.T = T;
    prm.M = plan->info.M;
    prm.hop = hop;
    prm.tab = plan->d_stft_tab;
    prm.out = out;
    switch (plan->info.N) {
    case 64: return launch_stft_t<64>(prm, plan->num_sms, st);
    case 128: return launch_stft_t<128>(prm, plan->num_sms, st);
    case 256: return launch_stft_t<256>(prm, plan->num_sms, st);
    case 512: return launch_stft_t<512>(prm, plan->num_sms, st);
    case 1024: return launch_stft_t<1024>(prm, plan->num_sms, st);
    case 2048: return launch_stft_t<2048>(prm, plan->num_sms, st);
    default: return fail(FCC_ERR_UNSUPPORTED, "the STFT front-end needs 64 <= N <= 2048");
    }
}

long long frames_of(long long n_samples, int N, int hop) { return n_samples < N ? 0 : 1 + (n_samples - N) / hop; }

size_t sample_bytes(int type) { return type == FCC_PCM_S16 ? 2 : 4; }

long long device_chunk(const fcc_plan *plan)
{
    const long long fb = (long long)plan->info.M * plan->info.B * 8;
    return std::max<long long>(1, kPcmChunkBytes / fb);
}

fcc_status_t check_pcm(const fcc_plan *plan, int type, long long n_samples, int hop)
{
    if (type != FCC_PCM_F32 && type != FCC_PCM_S16) return fail(FCC_ERR_INVALID_ARG, "unknown PCM type");
    if (n_samples < 0) return fail(FCC_ERR_INVALID_ARG, "n_samples < 0");
    if (hop < 1) return fail(FCC_ERR_INVALID_ARG, "hop < 1");
    if (plan->info.N < 64 || plan->info.N > 2048) return fail(FCC_ERR_UNSUPPORTED, "the STFT front-end needs 64 <= N <= 2048");
    return FCC_OK;
}

// frames [t0, t0 + n) of the PCM, ch at a time: STFT into `spec`, then FCC into the outputs at t0
fcc_status_t pcm_chunks(fcc_plan *plan, const unsigned char *pcm, int type, long long T, int hop, int *idx,
                        float *peak, float *tau, float2 *spec, long long ch, cudaStream_t st)
{
    const fcc_plan_info_t &in = plan->info;
    const size_t sb = sample_bytes(type) * (size_t)in.M;
    for (long long t0 = 0; t0 < T; t0 += ch) {
        const long long n = std::min(ch, T - t0);
        fcc_status_t s = launch_stft(plan, pcm + (size_t)t0 * hop * sb, type, n, hop, spec, st);
        if (s != FCC_OK) return s;
        const size_t o = (size_t)t0 * in.P;
        s = launch_tdoa(plan, spec, n, idx + o, peak + o, tau ? tau + o : nullptr, nullptr, nullptr, st);
        if (s != FCC_OK) return s;
    }
    return FCC_OK;
}

}  // namespace

// Host-streaming state of fcc_tdoa_pcm_host, owned by the plan.
struct PcmState {
    void *d_pcm[2] = {nullptr, nullptr};
    int *d_idx[2] = {nullptr, nullptr};
    float *d_peak[2] = {nullptr, nullptr}, *d_tau[2] = {nullptr, nullptr};
    float2 *d_spec = nullptr;
    size_t pcm_cap = 0;
    cudaStream_t copy = nullptr;
    cudaEvent_t ev[5] = {};
};

void pcm_destroy(fcc_plan *plan)
{
    PcmState *s = static_cast<PcmState *>(plan->pcm_state);
    if (!s) return;
    for (int b = 0; b < 2; ++b) {
        cudaFree(s->d_pcm[b]);
        cudaFree(s->d_idx[b]);
        cudaFree(s->d_peak[b]);
        cudaFree(s->d_tau[b]);
    }
    cudaFree(s->d_spec);
    if (s->copy) cudaStreamDestroy(s->copy);
    for (auto &e : s->ev)
        if (e) cudaEventDestroy(e);
    delete s;
    plan->pcm_state = nullptr;
}

}  // namespace fcc

using namespace fcc;

extern "C" {

fcc_status_t fcc_stft_frames(const fcc_plan_t *plan, long long n_samples, int hop, long long *T)
{
    if (!plan || !T) return fail(FCC_ERR_INVALID_ARG, "null argument");
    if (n_samples < 0) return fail(FCC_ERR_INVALID_ARG, "n_samples < 0");
    if (hop < 1) return fail(FCC_ERR_INVALID_ARG, "hop < 1");
    *T = frames_of(n_samples, plan->info.N, hop);
    return FCC_OK;
}

fcc_status_t fcc_stft(fcc_plan_t *plan, const void *d_pcm, fcc_pcm_t type, long long n_samples, int hop,
                      void *d_spectra, void *stream)
{
    if (!plan) return fail(FCC_ERR_INVALID_ARG, "null plan");
    fcc_status_t s = check_pcm(plan, type, n_samples, hop);
    if (s != FCC_OK) return s;
    const long long T = frames_of(n_samples, plan->info.N, hop);
    if (T == 0) return FCC_OK;
    if (!d_pcm || !d_spectra) return fail(FCC_ERR_INVALID_ARG, "null pcm/spectra");
    if ((reinterpret_cast<uintptr_t>(d_pcm) & (sample_bytes(type) - 1)) || (reinterpret_cast<uintptr_t>(d_spectra) & 7))
        return fail(FCC_ERR_INVALID_ARG, "misaligned buffer");
    DeviceScope scope(plan->device);
    if (!scope.ok) return fail(FCC_ERR_CUDA, "cudaSetDevice failed");
    return launch_stft(plan, d_pcm, type, T, hop, static_cast<float2 *>(d_spectra), static_cast<cudaStream_t>(stream));
}

fcc_status_t fcc_pcm_workspace(const fcc_plan_t *plan, long long n_samples, int hop, long long *bytes)
{
    if (!plan || !bytes) return fail(FCC_ERR_INVALID_ARG, "null argument");
    if (n_samples < 0 || hop < 1) return fail(FCC_ERR_INVALID_ARG, "n_samples < 0 or hop < 1");
    const long long T = frames_of(n_samples, plan->info.N, hop);
    *bytes = std::min(T, device_chunk(plan)) * plan->info.M * plan->info.B * 8;
    return FCC_OK;
}

fcc_status_t fcc_tdoa_pcm(fcc_plan_t *plan, const void *d_pcm, fcc_pcm_t type, long long n_samples, int hop,
                          int *d_lag_idx, float *d_peak, float *d_tau_hat, void *d_work, long long work_bytes,
                          void *stream)
{
    if (!plan) return fail(FCC_ERR_INVALID_ARG, "null plan");
    fcc_status_t s = check_pcm(plan, type, n_samples, hop);
    if (s != FCC_OK) return s;
    const long long T = frames_of(n_samples, plan->info.N, hop);
    if (T == 0) return FCC_OK;
    if (!d_pcm || !d_lag_idx || !d_peak || !d_work) return fail(FCC_ERR_INVALID_ARG, "null pcm/outputs/workspace");
    if ((reinterpret_cast<uintptr_t>(d_pcm) & (sample_bytes(type) - 1)) || (reinterpret_cast<uintptr_t>(d_work) & 15) ||
        ((reinterpret_cast<uintptr_t>(d_lag_idx) | reinterpret_cast<uintptr_t>(d_peak) |
          reinterpret_cast<uintptr_t>(d_tau_hat)) & 3))
        return fail(FCC_ERR_INVALID_ARG, "misaligned buffer");
    // the workspace holds one chunk of spectra: a larger one means fewer, larger chunks
    const long long frame_bytes = (long long)plan->info.M * plan->info.B * 8;
    if (work_bytes < frame_bytes) return fail(FCC_ERR_INVALID_ARG, "workspace smaller than one frame of spectra");
    if (!plan->kh) return fail(FCC_ERR_UNSUPPORTED, "more than 8 bases of one parity");
    DeviceScope scope(plan->device);
    if (!scope.ok) return fail(FCC_ERR_CUDA, "cudaSetDevice failed");
    return pcm_chunks(plan, static_cast<const unsigned char *>(d_pcm), type, T, hop, d_lag_idx, d_peak, d_tau_hat,
                      static_cast<float2 *>(d_work), std::min(T, work_bytes / frame_bytes),
                      static_cast<cudaStream_t>(stream));
}

fcc_status_t fcc_tdoa_pcm_host(fcc_plan_t *plan, const void *h_pcm, fcc_pcm_t type, long long n_samples, int hop,
                               int *h_lag_idx, float *h_peak, float *h_tau_hat, void *stream)
{
    if (!plan) return fail(FCC_ERR_INVALID_ARG, "null plan");
    fcc_status_t s = check_pcm(plan, type, n_samples, hop);
    if (s != FCC_OK) return s;
    const fcc_plan_info_t &in = plan->info;
    const long long T = frames_of(n_samples, in.N, hop);
    if (T == 0) return FCC_OK;
    if (!h_pcm || !h_lag_idx || !h_peak) return fail(FCC_ERR_INVALID_ARG, "null host buffer");
    if (!plan->kh) return fail(FCC_ERR_UNSUPPORTED, "more than 8 bases of one parity");
    DeviceScope scope(plan->device);
    if (!scope.ok) return fail(FCC_ERR_CUDA, "cudaSetDevice failed");
    const size_t sb = sample_bytes(type) * (size_t)in.M;
    const long long hc = kHostChunkFrames;
    const size_t pcm_bytes = ((size_t)(hc - 1) * hop + in.N) * sb;
    PcmState *ps = static_cast<PcmState *>(plan->pcm_state);
    if (!ps) {
        ps = new (std::nothrow) PcmState;
        if (!ps) return fail(FCC_ERR_OOM, "host allocation");
        plan->pcm_state = ps;
        // a failed creation frees what it made, so a later call starts again
        cudaError_t e = cudaSuccess;
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = dev_alloc((void **)&ps->d_idx[b], (size_t)hc * in.P * sizeof(int));
            if (e == cudaSuccess) e = dev_alloc((void **)&ps->d_peak[b], (size_t)hc * in.P * sizeof(float));
            if (e == cudaSuccess) e = dev_alloc((void **)&ps->d_tau[b], (size_t)hc * in.P * sizeof(float));
        }
        if (e == cudaSuccess)
            e = dev_alloc((void **)&ps->d_spec, (size_t)std::min(hc, device_chunk(plan)) * in.M * in.B * 8);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ps->copy, cudaStreamNonBlocking);
        for (auto &ev : ps->ev)
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            pcm_destroy(plan);
            return e == cudaErrorMemoryAllocation ? fail(FCC_ERR_OOM, "fcc_tdoa_pcm_host staging")
                                                  : cuda_fail(e, "fcc_tdoa_pcm_host staging");
        }
    }
    if (ps->pcm_cap < pcm_bytes) {
        FCC_CUDA_TRY(cudaDeviceSynchronize());
        for (int b = 0; b < 2; ++b) {
            cudaFree(ps->d_pcm[b]);
            ps->d_pcm[b] = nullptr;
        }
        ps->pcm_cap = 0;
        for (int b = 0; b < 2; ++b) FCC_CUDA_TRY(dev_alloc(&ps->d_pcm[b], pcm_bytes));
        ps->pcm_cap = pcm_bytes;
    }
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaStream_t hs = ps->copy;
    // ev[b]: PCM of buffer b on the device; ev[2 + b]: buffer b free again
    FCC_CUDA_TRY(cudaEventRecord(ps->ev[4], cs));
    FCC_CUDA_TRY(cudaStreamWaitEvent(hs, ps->ev[4], 0));
    const unsigned char *src = static_cast<const unsigned char *>(h_pcm);
    long long chunk_id = 0;
    for (long long t0 = 0; t0 < T; t0 += hc, ++chunk_id) {
        const int b = (int)(chunk_id & 1);
        const long long n = std::min(hc, T - t0);
        const size_t bytes = ((size_t)(n - 1) * hop + in.N) * sb;
        if (chunk_id >= 2) FCC_CUDA_TRY(cudaStreamWaitEvent(hs, ps->ev[2 + b], 0));
        FCC_CUDA_TRY(cudaMemcpyAsync(ps->d_pcm[b], src + (size_t)t0 * hop * sb, bytes, cudaMemcpyHostToDevice, hs));
        FCC_CUDA_TRY(cudaEventRecord(ps->ev[b], hs));
        FCC_CUDA_TRY(cudaStreamWaitEvent(cs, ps->ev[b], 0));
        s = pcm_chunks(plan, static_cast<const unsigned char *>(ps->d_pcm[b]), type, n, hop, ps->d_idx[b],
                       ps->d_peak[b], h_tau_hat ? ps->d_tau[b] : nullptr, ps->d_spec,
                       std::min(hc, device_chunk(plan)), cs);
        if (s != FCC_OK) return s;
        const size_t o = (size_t)t0 * in.P, cnt = (size_t)n * in.P;
        FCC_CUDA_TRY(cudaMemcpyAsync(h_lag_idx + o, ps->d_idx[b], cnt * sizeof(int), cudaMemcpyDeviceToHost, cs));
        FCC_CUDA_TRY(cudaMemcpyAsync(h_peak + o, ps->d_peak[b], cnt * sizeof(float), cudaMemcpyDeviceToHost, cs));
        if (h_tau_hat)
            FCC_CUDA_TRY(cudaMemcpyAsync(h_tau_hat + o, ps->d_tau[b], cnt * sizeof(float), cudaMemcpyDeviceToHost, cs));
        FCC_CUDA_TRY(cudaEventRecord(ps->ev[2 + b], cs));
    }
    return fcc_plan_sync(plan, stream);
}

}  // extern "C"
