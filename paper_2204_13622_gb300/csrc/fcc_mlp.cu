// fcc_mlp.cu -- the learned TDoA head (an extension; the paper has no learned
// part): a 2K -> 128 -> 128 -> 2 MLP on a pair-frame's projection coefficients,
// y0 = sub-sample TDoA, y1 = confidence logit, exact erf GELU (erff in the
// training kernels; a fitted form within 5e-7 of it in the inference kernel),
// BF16 weights, FP32 accumulation and FP32 master weights for training.
//
// Kernels (hand-written, CUDA cores; one block = 128 threads, thread j <-> hidden
// unit j, tiles of 32 samples):
//   mlp_grad_kernel   persistent blocks; per tile: forward (keeping gelu and
//                     gelu' of both layers in shared memory), loss gradient,
//                     backward; parameter gradients accumulate per block and are
//                     written once per block;
//   mlp_reduce_kernel sums the per-block partials in a fixed order (bitwise
//                     reproducible gradients);
//   mlp_adam_kernel   Adam on the FP32 masters, refreshing the BF16 copies;
//   mlp_infer_tc_kernel  forward on the tensor cores + confidence gate: TDoA =
//                     y0 when sigmoid(y1) >= threshold, else the plain FCC estimate.
// Loss (mean over the batch): (y0 - t)^2 + lambda * BCE(sigmoid(y1), g), with the
// target g = [|y0 - t| <= |t_fcc - t|]: the confidence learns when the network
// beats the plain argmax + parabola.
#include <algorithm>
#include <cmath>
#include <cuda_bf16.h>
#include <new>
#include <vector>

#include "fcc_device.cuh"
#include "fcc_internal.h"
#include "fcc_mlp.h"

namespace fcc {
namespace {

constexpr int kH = 128;      // hidden width
constexpr int kTileS = 32;   // samples per tile
constexpr int kMaxIn = 32;   // 2K <= 32
constexpr int kLd = kH + 1;  // padded row of the activation tiles

__device__ __forceinline__ float gelu(float a) { return 0.5f * a * (1.f + erff(a * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float a)
{
    return 0.5f * (1.f + erff(a * 0.70710678118654752f)) + a * 0.39894228040143268f * expf(-0.5f * a * a);
}

// GELU for the inference kernel, two values at a time in packed FP32:
//   GELU(x) = x Phi(x) = max(x, 0) - t Phi(-t),  t = |x|,
//   Phi(-t) = exp(-t^2 / 2) S(t),  S(t) = sum_j c_j u^j,  u = 1 / (1 + 0.3 t),
// with t clamped to 7 (t Phi(-t) < 1e-11 beyond).  S(t) = Phi(-t) exp(t^2 / 2) is
// smooth and slowly varying; c_0..c_7 are its least-squares fit on Chebyshev
// points of u (csrc/fit_gelu.py, which also evaluates this order in FP32: the
// error against the exact-erf GELU is below 5e-7, 1.4e-7 of max(1, |x|)).  One
// reciprocal and one exp2 per value on the special-function unit, the rest in
// packed FMAs.  The training kernels keep gelu() above.
__device__ __forceinline__ float rcp_approx(float a)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float ex2_approx(float a)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ f2 gelu2(float a, float b)
{
    const f2 t = pk(fminf(fabsf(a), 7.f), fminf(fabsf(b), 7.f));
    float da, db;
    upk(fma2(pk(0.3f, 0.3f), t, pk(1.f, 1.f)), da, db);
    const f2 u = pk(rcp_approx(da), rcp_approx(db));
    f2 s = pk(3.266900021e-02f, 3.266900021e-02f);
    s = fma2(s, u, pk(-2.269355121e-01f, -2.269355121e-01f));
    s = fma2(s, u, pk(4.993950225e-01f, 4.993950225e-01f));
    s = fma2(s, u, pk(-3.028911948e-01f, -3.028911948e-01f));
    s = fma2(s, u, pk(3.103419967e-01f, 3.103419967e-01f));
    s = fma2(s, u, pk(5.813875278e-02f, 5.813875278e-02f));
    s = fma2(s, u, pk(1.300175062e-01f, 1.300175062e-01f));
    s = fma2(s, u, pk(-7.356064136e-04f, -7.356064136e-04f));
    constexpr float kHalfLog2e = -0.72134752044448170f;  // -1 / (2 ln 2)
    float qa, qb;
    upk(mul2(mul2(t, pk(kHalfLog2e, kHalfLog2e)), t), qa, qb);
    const f2 corr = mul2(mul2(t, pk(ex2_approx(qa), ex2_approx(qb))), s);
    return sub2(pk(fmaxf(a, 0.f), fmaxf(b, 0.f)), corr);
}

struct MlpW {
    const __nv_bfloat16 *W1, *W2, *W3;  // BF16 copies: [H][nin], [H][H], [2][H]
    const float *b1, *b2, *b3;          // FP32
    const float *scale;                 // per-input scale [nin]
    int nin;
};

// Shared-memory image of the weights (W2 also transposed for the backward).
struct MlpSmem {
    __nv_bfloat16 W2[kH * kH];
    __nv_bfloat16 W2T[kH * kH];
    __nv_bfloat16 W1[kH * kMaxIn];
    __nv_bfloat16 W3[2 * kH];
    float b1[kH], b2[kH], b3[2];
    float scale[kMaxIn];
    float X[kTileS][kMaxIn + 1];
    float H1[kTileS][kLd], G1[kTileS][kLd];  // gelu(a1), gelu'(a1)
    float H2[kTileS][kLd], G2[kTileS][kLd];  // gelu(a2), gelu'(a2) -> reused for da2
    float Y[kTileS][2], DY[kTileS][2];
};

__device__ void load_weights(MlpSmem &s, const MlpW &w)
{
    for (int e = threadIdx.x; e < kH * kH; e += blockDim.x) {
        const __nv_bfloat16 v = w.W2[e];
        s.W2[e] = v;
        s.W2T[(e % kH) * kH + e / kH] = v;
    }
    for (int e = threadIdx.x; e < kH * w.nin; e += blockDim.x) s.W1[e] = w.W1[e];
    for (int e = threadIdx.x; e < 2 * kH; e += blockDim.x) s.W3[e] = w.W3[e];
    for (int e = threadIdx.x; e < kH; e += blockDim.x) {
        s.b1[e] = w.b1[e];
        s.b2[e] = w.b2[e];
    }
    if (threadIdx.x < 2) s.b3[threadIdx.x] = w.b3[threadIdx.x];
    if (threadIdx.x < kMaxIn) s.scale[threadIdx.x] = threadIdx.x < w.nin ? w.scale[threadIdx.x] : 0.f;
}

// Forward of one tile of ns <= 32 samples (rows >= ns are zero).  Needs
// s.X loaded; leaves H1, G1, H2, G2, Y in shared memory.
__device__ void forward_tile(MlpSmem &s, int nin, bool want_grad)
{
    const int j = threadIdx.x;
    {
        float w[kMaxIn];
#pragma unroll
        for (int i = 0; i < kMaxIn; ++i) w[i] = i < nin ? __bfloat162float(s.W1[j * nin + i]) : 0.f;
        for (int r = 0; r < kTileS; ++r) {
            float a = s.b1[j];
#pragma unroll
            for (int i = 0; i < kMaxIn; ++i) a = fmaf(w[i], s.X[r][i], a);
            s.H1[r][j] = gelu(a);
            if (want_grad) s.G1[r][j] = gelu_d(a);
        }
    }
    __syncthreads();
    {
        float acc[kTileS];
#pragma unroll
        for (int r = 0; r < kTileS; ++r) acc[r] = s.b2[j];
        for (int i = 0; i < kH; ++i) {
            const float w = __bfloat162float(s.W2T[i * kH + j]);
#pragma unroll
            for (int r = 0; r < kTileS; ++r) acc[r] = fmaf(w, s.H1[r][i], acc[r]);
        }
#pragma unroll
        for (int r = 0; r < kTileS; ++r) {
            s.H2[r][j] = gelu(acc[r]);
            if (want_grad) s.G2[r][j] = gelu_d(acc[r]);
        }
    }
    __syncthreads();
    if (j < 2 * kTileS) {
        const int r = j >> 1, o = j & 1;
        float y = s.b3[o];
        for (int i = 0; i < kH; ++i) y = fmaf(__bfloat162float(s.W3[o * kH + i]), s.H2[r][i], y);
        s.Y[r][o] = y;
    }
    __syncthreads();
}

__device__ void load_x(MlpSmem &s, const float *feat, long long base, int ns, int nin)
{
    for (int e = threadIdx.x; e < kTileS * kMaxIn; e += blockDim.x) {
        const int r = e / kMaxIn, i = e % kMaxIn;
        s.X[r][i] = (r < ns && i < nin) ? feat[(size_t)(base + r) * nin + i] * s.scale[i] : 0.f;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kH) mlp_grad_kernel(MlpW w, const float *feat, const float *tau_true,
                                                      const float *tau_fcc, long long n, float lambda,
                                                      float *partial, long long n_params, float *loss_partial)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpSmem &s = *reinterpret_cast<MlpSmem *>(smem_raw);
    const int nin = w.nin, j = threadIdx.x;
    load_weights(s, w);
    __syncthreads();
    float gW1[kMaxIn], gb1 = 0.f, gb2 = 0.f, gW3_0 = 0.f, gW3_1 = 0.f, gb3_0 = 0.f, gb3_1 = 0.f, lsum = 0.f;
#pragma unroll
    for (int i = 0; i < kMaxIn; ++i) gW1[i] = 0.f;
    float *gW2 = reinterpret_cast<float *>(smem_raw + sizeof(MlpSmem));  // [H][kLd], row j owned by thread j
    for (int i = 0; i < kH; ++i) gW2[j * kLd + i] = 0.f;
    const float inv_n = 1.f / (float)n;
    const long long n_tiles = (n + kTileS - 1) / kTileS;
    for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const long long base = t * kTileS;
        const int ns = (int)min((long long)kTileS, n - base);
        load_x(s, feat, base, ns, nin);
        forward_tile(s, nin, true);
        // loss gradient at the outputs
        if (j < kTileS) {
            float dy0 = 0.f, dy1 = 0.f;
            if (j < ns) {
                const float y0 = s.Y[j][0], y1 = s.Y[j][1];
                const float tt = tau_true[base + j], tf = tau_fcc[base + j];
                const float e = y0 - tt;
                const float g = fabsf(e) <= fabsf(tf - tt) ? 1.f : 0.f;
                const float c = 1.f / (1.f + expf(-y1));
                const float bce = (y1 > 0.f ? y1 + log1pf(expf(-y1)) : log1pf(expf(y1))) - g * y1;
                lsum += e * e + lambda * bce;
                dy0 = 2.f * e * inv_n;
                dy1 = lambda * (c - g) * inv_n;
            }
            s.DY[j][0] = dy0;
            s.DY[j][1] = dy1;
        }
        __syncthreads();
        // layer 3 and da2 = (W3^T dy) * gelu'(a2)
        {
            const float w30 = __bfloat162float(s.W3[j]), w31 = __bfloat162float(s.W3[kH + j]);
            for (int r = 0; r < kTileS; ++r) {
                const float dy0 = s.DY[r][0], dy1 = s.DY[r][1];
                gW3_0 = fmaf(dy0, s.H2[r][j], gW3_0);
                gW3_1 = fmaf(dy1, s.H2[r][j], gW3_1);
                const float da2 = fmaf(w30, dy0, w31 * dy1) * s.G2[r][j];
                s.G2[r][j] = da2;
                gb2 += da2;
            }
            if (j == 0)
                for (int r = 0; r < kTileS; ++r) {
                    gb3_0 += s.DY[r][0];
                    gb3_1 += s.DY[r][1];
                }
        }
        __syncthreads();
        // dW2[j][i] += sum_r da2[r][j] h1[r][i];  dh1[r][i] = sum_j W2[j][i] da2[r][j]
        {
            float d2[kTileS];
#pragma unroll
            for (int r = 0; r < kTileS; ++r) d2[r] = s.G2[r][j];
            for (int i = 0; i < kH; ++i) {
                float acc = 0.f;
#pragma unroll
                for (int r = 0; r < kTileS; ++r) acc = fmaf(d2[r], s.H1[r][i], acc);
                gW2[j * kLd + i] += acc;
            }
        }
        {
            const int i = j;  // this thread now owns input unit i of layer 2
            float acc[kTileS];
#pragma unroll
            for (int r = 0; r < kTileS; ++r) acc[r] = 0.f;
            for (int jj = 0; jj < kH; ++jj) {
                const float wv = __bfloat162float(s.W2[jj * kH + i]);
#pragma unroll
                for (int r = 0; r < kTileS; ++r) acc[r] = fmaf(wv, s.G2[r][jj], acc[r]);
            }
#pragma unroll
            for (int r = 0; r < kTileS; ++r) {
                const float da1 = acc[r] * s.G1[r][i];
                gb1 += da1;
#pragma unroll
                for (int k = 0; k < kMaxIn; ++k) gW1[k] = fmaf(da1, s.X[r][k], gW1[k]);
            }
        }
        __syncthreads();
    }
    // per-block partial gradients, packed as W1, b1, W2, b2, W3, b3
    float *pp = partial + (size_t)blockIdx.x * n_params;
#pragma unroll
    for (int k = 0; k < kMaxIn; ++k)
        if (k < nin) pp[(size_t)j * nin + k] = gW1[k];
    float *pb1 = pp + (size_t)kH * nin, *pW2 = pb1 + kH, *pb2 = pW2 + (size_t)kH * kH, *pW3 = pb2 + kH,
          *pb3 = pW3 + 2 * kH;
    pb1[j] = gb1;
    for (int i = 0; i < kH; ++i) pW2[(size_t)j * kH + i] = gW2[j * kLd + i];
    pb2[j] = gb2;
    pW3[j] = gW3_0;
    pW3[kH + j] = gW3_1;
    if (j == 0) {
        pb3[0] = gb3_0;
        pb3[1] = gb3_1;
    }
    // block loss sum (threads < 32 hold per-sample sums)
    float l = lsum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if (j == 0) loss_partial[blockIdx.x] = l;
}

__global__ void mlp_reduce_kernel(const float *partial, int nb, long long n_params, float *grad,
                                  const float *loss_partial, float *loss, long long n)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n_params;
         k += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < nb; ++b) s += partial[(size_t)b * n_params + k];
        grad[k] = s;
    }
    if (loss && blockIdx.x == 0 && threadIdx.x == 0) {
        float s = 0.f;
        for (int b = 0; b < nb; ++b) s += loss_partial[b];
        *loss = s / (float)n;
    }
}

__global__ void mlp_adam_kernel(float *p, const float *g, float *m, float *v, long long n_params, float lr,
                                float c1, float c2, __nv_bfloat16 *W1b, __nv_bfloat16 *W2b, __nv_bfloat16 *W3b,
                                int nin)
{
    const long long nW1 = (long long)kH * nin, o2 = nW1 + kH, o3 = o2 + (long long)kH * kH + kH;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n_params;
         k += (long long)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = 0.9f * m[k] + 0.1f * gk;
        const float vk = 0.999f * v[k] + 0.001f * gk * gk;
        m[k] = mk;
        v[k] = vk;
        const float pk = p[k] - lr * (mk / c1) / (sqrtf(vk / c2) + 1e-8f);
        p[k] = pk;
        if (k < nW1) W1b[k] = __float2bfloat16_rn(pk);
        else if (k >= o2 && k < o2 + (long long)kH * kH) W2b[k - o2] = __float2bfloat16_rn(pk);
        else if (k >= o3 && k < o3 + 2 * kH) W3b[k - o3] = __float2bfloat16_rn(pk);
    }
}

// ---------------------------------------------------------------------------
// Inference on the tensor cores.  One CTA of 256 threads takes 128-sample tiles:
// warps w and w + 4 own TMEM lanes 32 (w % 4) .. + 31 (one sample per lane) and
// split the 128 hidden columns in halves.  Layer 1 and layer 2 are tcgen05.mma
// (kind::f16, BF16 x BF16 -> FP32 in TMEM, M = 128, N = 128); the activations
// enter as a two-term BF16 split a = hi + lo (hi = bf16(a), lo = bf16(a - hi)),
// so each layer is two MMA passes against the same BF16 weights and the
// products carry the activations to about 2^-17 -- the FP32 activations of the
// training kernels.  The epilogues read TMEM with tcgen05.ld (bias, GELU to
// FP32 accuracy with gelu2, the split for the next layer; layer 3 and the gate
// on the CUDA cores).
constexpr int kTcRows = 128;
constexpr int kTcThreads = 256;

struct TcMlpLayout {
    int K1;  // layer-1 K: n_in padded to a multiple of 16
    size_t w1, w2, abuf, w3, b1, b2, part, total;
};

__host__ __device__ inline TcMlpLayout tc_mlp_layout(int nin)
{
    TcMlpLayout L;
    L.K1 = (nin + 15) / 16 * 16;
    size_t o = 128;                       // mbarrier, TMEM address, abort flag
    L.w1 = o;
    o += (size_t)kH * L.K1 * 2;           // B of layer 1: [128][K1] bf16, K-major core matrices
    L.w2 = o;
    o += (size_t)kH * kH * 2;             // B of layer 2: [128][128]
    L.abuf = o;
    o += (size_t)kTcRows * 2 * kH * 2;    // A of layer 2: [128][hi 128 | lo 128]; A of layer 1 aliases it
    L.w3 = o;
    o += 2 * kH * 4;
    L.b1 = o;
    o += kH * 4;
    L.b2 = o;
    o += kH * 4;
    L.part = o;
    o += (size_t)kTcRows * 2 * 4 + 16;  // layer-3 partial sums of the second column half
    L.total = o;
    return L;
}

// Byte offset of element (r, k) of a K-major operand with K columns (bf16):
// 8-row x 16-byte core matrices, adjacent along K, then along rows.
__device__ __forceinline__ int kmaj(int r, int k, int K) { return ((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2; }

__device__ __forceinline__ uint32_t bf2(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// Write 8 consecutive K entries of row r (hi part at k, lo part at k + koff).
__device__ __forceinline__ void store_split8(unsigned char *A, int r, int k, int K, int koff, const float *v)
{
    // hi = bf16(v) packed two at a time; its FP32 values are the packed halves
    // moved to the top 16 bits, and lo = bf16(v - hi)
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        hi[j] = bf2(v[2 * j], v[2 * j + 1]);
        lo[j] = bf2(v[2 * j] - __uint_as_float(hi[j] << 16), v[2 * j + 1] - __uint_as_float(hi[j] & 0xffff0000u));
    }
    *reinterpret_cast<uint4 *>(A + kmaj(r, k, K)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<uint4 *>(A + kmaj(r, k + koff, K)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
}

__global__ void __launch_bounds__(kTcThreads) mlp_infer_tc_kernel(MlpW w, const float *feat, const float *tau_fcc,
                                                                  long long n, float threshold, float *tau_out,
                                                                  float *conf_out, float *raw_out, unsigned *err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int nin = w.nin;
    const TcMlpLayout L = tc_mlp_layout(nin);
    const int K1 = L.K1;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + 8);
    int *abort_flag = reinterpret_cast<int *>(smem + 12);
    unsigned char *W1s = smem + L.w1, *W2s = smem + L.w2, *A = smem + L.abuf;
    float *W3s = reinterpret_cast<float *>(smem + L.w3), *b1s = reinterpret_cast<float *>(smem + L.b1),
          *b2s = reinterpret_cast<float *>(smem + L.b2), *part = reinterpret_cast<float *>(smem + L.part);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int r = (warp & 3) * 32 + (tid & 31);  // sample row = TMEM lane
    const int half = warp >> 2;                  // hidden columns [64 half, 64 half + 64)

    // weights into shared memory, once per CTA
    for (int e = tid; e < kH * K1; e += blockDim.x) {
        const int o = e / K1, k = e % K1;
        *reinterpret_cast<__nv_bfloat16 *>(W1s + kmaj(o, k, K1)) =
            k < nin ? w.W1[o * nin + k] : __float2bfloat16_rn(0.f);
    }
    for (int e = tid; e < kH * kH; e += blockDim.x)
        *reinterpret_cast<__nv_bfloat16 *>(W2s + kmaj(e / kH, e % kH, kH)) = w.W2[e];
    for (int e = tid; e < 2 * kH; e += blockDim.x) W3s[e] = __bfloat162float(w.W3[e]);
    for (int e = tid; e < kH; e += blockDim.x) {
        b1s[e] = w.b1[e];
        b2s[e] = w.b2[e];
    }
    const float b30 = w.b3[0], b31 = w.b3[1];
    if (tid == 0) {
        mbar_init(bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "n"(kH));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t t_row = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(64 * half);
    // instruction descriptor: D FP32, A and B BF16, K-major, N = 128, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kH >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
    const uint32_t a_addr = smem_u32(A), w1_addr = smem_u32(W1s), w2_addr = smem_u32(W2s);
    unsigned phase = 0;
    bool failed = false;

    // one MMA pass set, committed to the barrier; every thread waits for it
    auto mma_and_wait = [&](int layer) -> bool {
        fence_proxy_async();  // our generic stores of A -> the tensor cores' reads
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (layer == 1) {
                const uint32_t sbo_a = (uint32_t)(2 * K1 / 8) * 128, sbo_b = (uint32_t)(K1 / 8) * 128;
                for (int j = 0; j < 2 * K1 / 16; ++j)
                    umma_f16(tmem, umma_desc(a_addr + j * 256, 128, sbo_a),
                             umma_desc(w1_addr + (j % (K1 / 16)) * 256, 128, sbo_b), idesc, j > 0);
            } else {
                const uint32_t sbo_a = (uint32_t)(2 * kH / 8) * 128, sbo_b = (uint32_t)(kH / 8) * 128;
                for (int j = 0; j < 2 * kH / 16; ++j)
                    umma_f16(tmem, umma_desc(a_addr + j * 256, 128, sbo_a),
                             umma_desc(w2_addr + (j % (kH / 16)) * 256, 128, sbo_b), idesc, j > 0);
            }
            umma_commit(bar);
        }
        const bool ok = mbar_wait(bar, phase);
        phase ^= 1u;
        if (!ok) atomicOr(abort_flag, 1);
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        return *abort_flag == 0;
    };

    const long long n_tiles = (n + kTcRows - 1) / kTcRows;
    // This thread's features of a tile: groups g of 8 at k = 8 half + 16 g (K1 is
    // 16 or 32), loaded a tile ahead so that the loads overlap the tile's MMAs and
    // epilogues; 16-byte loads where every row is 16-byte aligned.
    const int ng = K1 / 16;
    const bool vec = (nin % 4 == 0) && ((reinterpret_cast<uintptr_t>(feat) & 15) == 0);
    float sc[2][8];
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = 8 * half + 16 * g + j;
            sc[g][j] = (g < ng && k < nin) ? w.scale[k] : 0.f;
        }
    float xf[2][8];
    auto load_feat = [&](long long tt) {
        const long long s = tt * kTcRows + r;
        const bool live = tt < n_tiles && s < n;
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            const int k = 8 * half + 16 * g;
            if (g < ng && live && vec && k + 8 <= nin) {
                const float4 a = *reinterpret_cast<const float4 *>(feat + (size_t)s * nin + k);
                const float4 b = *reinterpret_cast<const float4 *>(feat + (size_t)s * nin + k + 4);
                xf[g][0] = a.x, xf[g][1] = a.y, xf[g][2] = a.z, xf[g][3] = a.w;
                xf[g][4] = b.x, xf[g][5] = b.y, xf[g][6] = b.z, xf[g][7] = b.w;
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    xf[g][j] = (g < ng && live && k + j < nin) ? feat[(size_t)s * nin + k + j] : 0.f;
            }
        }
    };
    load_feat(blockIdx.x);
    for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const long long s = t * kTcRows + r;
        const bool live = s < n;
        // ---- A of layer 1: scaled features split into hi | lo; the two halves
        // of the CTA take alternate groups of 8 features
#pragma unroll
        for (int g = 0; g < 2; ++g)
            if (g < ng) {
                float x[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) x[j] = xf[g][j] * sc[g][j];
                store_split8(A, r, 8 * half + 16 * g, 2 * K1, K1, x);
            }
        load_feat(t + gridDim.x);
        if (!mma_and_wait(1)) {
            failed = true;
            break;
        }
        // ---- epilogue 1: bias, GELU, split into the A of layer 2
#pragma unroll 1
        for (int c0 = 0; c0 < 64; c0 += 32) {
            const int c = 64 * half + c0;
            float v[32];
            tmem_ld32(t_row + c0, v);
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
                const float4 bb = *reinterpret_cast<const float4 *>(b1s + c + j);
                upk(gelu2(v[j] + bb.x, v[j + 1] + bb.y), v[j], v[j + 1]);
                upk(gelu2(v[j + 2] + bb.z, v[j + 3] + bb.w), v[j + 2], v[j + 3]);
            }
#pragma unroll
            for (int j = 0; j < 32; j += 8) store_split8(A, r, c + j, 2 * kH, kH, v + j);
        }
        if (!mma_and_wait(2)) {
            failed = true;
            break;
        }
        // ---- epilogue 2: bias, GELU, layer 3 over this half's columns
        float y0 = 0.f, y1 = 0.f;
#pragma unroll 1
        for (int c0 = 0; c0 < 64; c0 += 32) {
            const int c = 64 * half + c0;
            float v[32];
            tmem_ld32(t_row + c0, v);
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
                const float4 bb = *reinterpret_cast<const float4 *>(b2s + c + j);
                const float4 w0 = *reinterpret_cast<const float4 *>(W3s + c + j);
                const float4 w1 = *reinterpret_cast<const float4 *>(W3s + kH + c + j);
                float h0, h1, h2, h3;
                upk(gelu2(v[j] + bb.x, v[j + 1] + bb.y), h0, h1);
                upk(gelu2(v[j + 2] + bb.z, v[j + 3] + bb.w), h2, h3);
                y0 = fmaf(w0.x, h0, y0);
                y1 = fmaf(w1.x, h0, y1);
                y0 = fmaf(w0.y, h1, y0);
                y1 = fmaf(w1.y, h1, y1);
                y0 = fmaf(w0.z, h2, y0);
                y1 = fmaf(w1.z, h2, y1);
                y0 = fmaf(w0.w, h3, y0);
                y1 = fmaf(w1.w, h3, y1);
            }
        }
        if (half == 1) {
            part[2 * r] = y0;
            part[2 * r + 1] = y1;
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // partials visible; TMEM and A are free for the next tile
        if (half == 0 && live) {
            y0 = b30 + (y0 + part[2 * r]);
            y1 = b31 + (y1 + part[2 * r + 1]);
            const float c = 1.f / (1.f + expf(-y1));
            tau_out[s] = (c >= threshold || !tau_fcc) ? y0 : tau_fcc[s];
            if (conf_out) conf_out[s] = c;
            if (raw_out) raw_out[s] = y0;
        }
    }
    if (failed) {
        if (tid == 0) atomicOr(err, kErrTimeout);
        // the last MMAs may still be running: wait once more (bounded) before freeing TMEM
        if (!mbar_wait(bar, phase ^ 1u) && tid == 0) atomicOr(err, kErrTimeout);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kH));
}

__global__ void bf16_copy_kernel(const float *src, __nv_bfloat16 *dst, long long n)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        dst[k] = __float2bfloat16_rn(src[k]);
}

}  // namespace
}  // namespace fcc

struct fcc_mlp {
    int device = 0, nin = 0, num_sms = 0;
    long long n_params = 0;
    float lambda = 0.1f;
    float *scale = nullptr;  // [nin]
    long long step = 0;
    float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
    __nv_bfloat16 *Wb = nullptr;  // W1, W2, W3 BF16 copies, contiguous
    float *partial = nullptr, *loss_partial = nullptr;
    unsigned *d_err = nullptr;  // device error word (bounded waits of the inference kernel)
    int nb = 0;
};

using namespace fcc;

namespace {

MlpW weights(const fcc_mlp *h)
{
    MlpW w;
    w.W1 = h->Wb;
    w.W2 = h->Wb + (size_t)kH * h->nin;
    w.W3 = w.W2 + (size_t)kH * kH;
    w.b1 = h->p + (size_t)kH * h->nin;
    w.b2 = w.b1 + kH + (size_t)kH * kH;
    w.b3 = w.b2 + kH + 2 * kH;
    w.nin = h->nin;
    w.scale = h->scale;
    return w;
}

fcc_status_t refresh_bf16(fcc_mlp *h, cudaStream_t st)
{
    const long long nW1 = (long long)kH * h->nin;
    bf16_copy_kernel<<<64, 256, 0, st>>>(h->p, h->Wb, nW1);
    bf16_copy_kernel<<<64, 256, 0, st>>>(h->p + nW1 + kH, h->Wb + nW1, (long long)kH * kH);
    bf16_copy_kernel<<<8, 256, 0, st>>>(h->p + nW1 + kH + (long long)kH * kH + kH, h->Wb + nW1 + (long long)kH * kH,
                                        2 * kH);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FCC_OK : cuda_fail(e, "bf16 weight copy");
}

size_t grad_smem() { return sizeof(MlpSmem) + sizeof(float) * kH * kLd; }

fcc_status_t run_grad(fcc_mlp *h, const float *feat, const float *tt, const float *tf, long long n, float *loss,
                      cudaStream_t st)
{
    static bool attr[64] = {};
    if (!attr[h->device & 63]) {
        FCC_CUDA_TRY(cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem()));
        attr[h->device & 63] = true;
    }
    const long long tiles = (n + kTileS - 1) / kTileS;
    const int grid = (int)std::min<long long>(tiles, h->nb);
    mlp_grad_kernel<<<grid, kH, grad_smem(), st>>>(weights(h), feat, tt, tf, n, h->lambda, h->partial, h->n_params,
                                                   h->loss_partial);
    mlp_reduce_kernel<<<(int)((h->n_params + 255) / 256), 256, 0, st>>>(h->partial, grid, h->n_params, h->g,
                                                                        h->loss_partial, loss, n);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FCC_OK : cuda_fail(e, "mlp gradient kernels");
}

}  // namespace

extern "C" {

long long fcc_mlp_num_params(int n_in, int hidden)
{
    return (long long)hidden * n_in + hidden + (long long)hidden * hidden + hidden + 2LL * hidden + 2;
}

fcc_status_t fcc_mlp_create(int n_in, int hidden, const float *h_in_scale, double conf_weight, const float *h_params,
                            int device, fcc_mlp_t **out)
{
    if (!out || !h_params) return fail(FCC_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (hidden != kH) return fail(FCC_ERR_UNSUPPORTED, "hidden width must be 128");
    if (n_in < 1 || n_in > kMaxIn) return fail(FCC_ERR_UNSUPPORTED, "n_in must be in [1, 32]");
    if (!(conf_weight >= 0)) return fail(FCC_ERR_INVALID_ARG, "conf_weight < 0");
    int dev = device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return fail(FCC_ERR_CUDA, "no CUDA device");
    DeviceScope scope(dev);
    if (!scope.ok) return fail(FCC_ERR_CUDA, "cudaSetDevice failed");
    fcc_mlp *h = new (std::nothrow) fcc_mlp();
    if (!h) return fail(FCC_ERR_OOM, "host allocation");
    h->device = dev;
    h->nin = n_in;
    h->lambda = (float)conf_weight;
    h->n_params = fcc_mlp_num_params(n_in, hidden);
    cudaError_t e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    h->nb = std::max(1, h->num_sms);
    const size_t np_ = (size_t)h->n_params;
    const size_t nwb = (size_t)kH * n_in + (size_t)kH * kH + 2 * kH;
    if (e == cudaSuccess) e = cudaMalloc(&h->p, np_ * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->m, np_ * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->v, np_ * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->g, np_ * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->Wb, nwb * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&h->partial, (size_t)h->nb * np_ * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->loss_partial, (size_t)h->nb * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->scale, (size_t)n_in * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, sizeof(unsigned));
    if (e == cudaSuccess) {
        std::vector<float> sc(n_in, 1.f);
        if (h_in_scale) sc.assign(h_in_scale, h_in_scale + n_in);
        e = cudaMemcpy(h->scale, sc.data(), (size_t)n_in * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(h->p, h_params, np_ * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->m, 0, np_ * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(h->v, 0, np_ * sizeof(float));
    fcc_status_t st = e == cudaSuccess ? refresh_bf16(h, 0) : cuda_fail(e, "mlp allocation");
    if (st == FCC_OK) {
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) st = cuda_fail(e, "mlp init");
    }
    if (st != FCC_OK) {
        fcc_mlp_destroy(h);
        return st;
    }
    *out = h;
    return FCC_OK;
}

void fcc_mlp_destroy(fcc_mlp_t *h)
{
    if (!h) return;
    DeviceScope scope(h->device);
    cudaDeviceSynchronize();
    cudaFree(h->p);
    cudaFree(h->m);
    cudaFree(h->v);
    cudaFree(h->g);
    cudaFree(h->Wb);
    cudaFree(h->partial);
    cudaFree(h->loss_partial);
    cudaFree(h->scale);
    cudaFree(h->d_err);
    delete h;
}

fcc_status_t fcc_mlp_get_state(const fcc_mlp_t *h, float *params, float *m, float *v, long long *step)
{
    if (!h) return fail(FCC_ERR_INVALID_ARG, "null mlp");
    DeviceScope scope(h->device);
    const size_t b = (size_t)h->n_params * sizeof(float);
    FCC_CUDA_TRY(cudaDeviceSynchronize());
    if (params) FCC_CUDA_TRY(cudaMemcpy(params, h->p, b, cudaMemcpyDeviceToHost));
    if (m) FCC_CUDA_TRY(cudaMemcpy(m, h->m, b, cudaMemcpyDeviceToHost));
    if (v) FCC_CUDA_TRY(cudaMemcpy(v, h->v, b, cudaMemcpyDeviceToHost));
    if (step) *step = h->step;
    return FCC_OK;
}

fcc_status_t fcc_mlp_set_state(fcc_mlp_t *h, const float *params, const float *m, const float *v, long long step)
{
    if (!h || !params) return fail(FCC_ERR_INVALID_ARG, "null argument");
    if (step < 0) return fail(FCC_ERR_INVALID_ARG, "step < 0");
    DeviceScope scope(h->device);
    const size_t b = (size_t)h->n_params * sizeof(float);
    FCC_CUDA_TRY(cudaDeviceSynchronize());
    FCC_CUDA_TRY(cudaMemcpy(h->p, params, b, cudaMemcpyHostToDevice));
    if (m) FCC_CUDA_TRY(cudaMemcpy(h->m, m, b, cudaMemcpyHostToDevice));
    else FCC_CUDA_TRY(cudaMemset(h->m, 0, b));
    if (v) FCC_CUDA_TRY(cudaMemcpy(h->v, v, b, cudaMemcpyHostToDevice));
    else FCC_CUDA_TRY(cudaMemset(h->v, 0, b));
    h->step = step;
    fcc_status_t st = refresh_bf16(h, 0);
    if (st != FCC_OK) return st;
    FCC_CUDA_TRY(cudaDeviceSynchronize());
    return FCC_OK;
}

fcc_status_t fcc_mlp_gradient(fcc_mlp_t *h, const float *d_feat, const float *d_tau_true, const float *d_tau_fcc,
                              long long n, float *d_grad, float *d_loss, void *stream)
{
    if (!h || !d_feat || !d_tau_true || !d_tau_fcc || !d_grad) return fail(FCC_ERR_INVALID_ARG, "null argument");
    if (n <= 0) return fail(FCC_ERR_INVALID_ARG, "n <= 0");
    DeviceScope scope(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    fcc_status_t s = run_grad(h, d_feat, d_tau_true, d_tau_fcc, n, d_loss, st);
    if (s != FCC_OK) return s;
    FCC_CUDA_TRY(cudaMemcpyAsync(d_grad, h->g, (size_t)h->n_params * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return FCC_OK;
}

fcc_status_t fcc_mlp_train_step(fcc_mlp_t *h, const float *d_feat, const float *d_tau_true, const float *d_tau_fcc,
                                long long n, float lr, float *d_loss, void *stream)
{
    if (!h || !d_feat || !d_tau_true || !d_tau_fcc) return fail(FCC_ERR_INVALID_ARG, "null argument");
    if (n <= 0 || !(lr > 0)) return fail(FCC_ERR_INVALID_ARG, "n <= 0 or lr <= 0");
    DeviceScope scope(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    fcc_status_t s = run_grad(h, d_feat, d_tau_true, d_tau_fcc, n, d_loss, st);
    if (s != FCC_OK) return s;
    h->step += 1;
    const float c1 = 1.f - powf(0.9f, (float)h->step), c2 = 1.f - powf(0.999f, (float)h->step);
    const long long nW1 = (long long)kH * h->nin;
    mlp_adam_kernel<<<(int)((h->n_params + 255) / 256), 256, 0, st>>>(
        h->p, h->g, h->m, h->v, h->n_params, lr, c1, c2, h->Wb, h->Wb + nW1, h->Wb + nW1 + (long long)kH * kH, h->nin);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FCC_OK : cuda_fail(e, "mlp adam");
}

fcc_status_t fcc_mlp_infer(fcc_mlp_t *h, const float *d_feat, const float *d_tau_fcc, long long n, float threshold,
                           float *d_tau, float *d_conf, float *d_raw, void *stream)
{
    if (!h) return fail(FCC_ERR_INVALID_ARG, "null mlp");
    if (n < 0) return fail(FCC_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return FCC_OK;
    if (!d_feat || !d_tau) return fail(FCC_ERR_INVALID_ARG, "null argument");
    DeviceScope scope(h->device);
    const size_t smem = tc_mlp_layout(h->nin).total;
    static bool attr[64] = {};
    if (!attr[h->device & 63]) {
        FCC_CUDA_TRY(cudaFuncSetAttribute(mlp_infer_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)tc_mlp_layout(kMaxIn).total));  // the largest layout
        attr[h->device & 63] = true;
    }
    const long long tiles = (n + kTcRows - 1) / kTcRows;
    const int grid = (int)std::min<long long>(tiles, (long long)h->num_sms * 2);
    mlp_infer_tc_kernel<<<grid, kTcThreads, smem, static_cast<cudaStream_t>(stream)>>>(
        weights(h), d_feat, d_tau_fcc, n, threshold, d_tau, d_conf, d_raw, h->d_err);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FCC_OK : cuda_fail(e, "mlp inference");
}

fcc_status_t fcc_tdoa_learned(fcc_plan_t *plan, fcc_mlp_t *h, const void *d_spectra, long long T, float threshold,
                              int *d_lag_idx, float *d_peak, float *d_tau_fcc, float *d_coeffs, float *d_tau,
                              float *d_conf, void *stream)
{
    if (!plan || !h) return fail(FCC_ERR_INVALID_ARG, "null plan or mlp");
    if (T < 0) return fail(FCC_ERR_INVALID_ARG, "T < 0");
    if (T == 0) return FCC_OK;
    if (h->nin != 2 * plan->info.K) return fail(FCC_ERR_INVALID_ARG, "the head's n_in differs from 2K of the plan");
    if (h->device != plan->device) return fail(FCC_ERR_INVALID_ARG, "plan and head on different devices");
    if (!d_tau_fcc || !d_coeffs || !d_tau) return fail(FCC_ERR_INVALID_ARG, "null tau_fcc / coeffs / tau");
    fcc_status_t st = fcc_tdoa(plan, d_spectra, T, d_lag_idx, d_peak, d_tau_fcc, d_coeffs, nullptr, stream);
    if (st != FCC_OK) return st;
    return fcc_mlp_infer(h, d_coeffs, d_tau_fcc, T * plan->info.P, threshold, d_tau, d_conf, nullptr, stream);
}

fcc_status_t fcc_mlp_sync(fcc_mlp_t *h, void *stream)
{
    if (!h) return fail(FCC_ERR_INVALID_ARG, "null mlp");
    DeviceScope scope(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    FCC_CUDA_TRY(cudaStreamSynchronize(st));
    unsigned err = 0;
    FCC_CUDA_TRY(cudaMemcpyAsync(&err, h->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    FCC_CUDA_TRY(cudaMemsetAsync(h->d_err, 0, sizeof(unsigned), st));
    FCC_CUDA_TRY(cudaStreamSynchronize(st));
    if (err & kErrTimeout) return fail(FCC_ERR_TIMEOUT, "a device-side wait expired");
    return FCC_OK;
}

}  // extern "C"
