// fcc_smooth.cu -- FCC with the recursive cross-spectrum of Sec. 2, Eq. 1 for a
// smoothing factor alpha in (0, 1]:
//   R(t,f) = (1 - alpha) R(t-1,f) + alpha X_i(t,f) X_j(t,f)^*,   R_hat = R / |R|.
// The per-microphone normalisation of the alpha = 1 path no longer applies: the
// phase transform acts on each pair's smoothed R, and R carries state from frame
// to frame.  The frames are cut into chunks and the linear recursion is solved
// exactly in three passes:
//   1. chunk_sums_kernel  per chunk, one thread per bin holding all pairs'
//      running sums: the recursion run from zero over the chunk's frames (L_c);
//   2. carry_kernel       per (pair, bin), over the chunks in order: the state
//      entering chunk c, S_c = (1 - alpha)^len(c-1) S_{c-1} + L_{c-1} from the
//      caller's initial state, and the state after the last frame (returned);
//   3. fcc_smooth_kernel  per chunk: one warp per 2x2 pair slot.  Lane l owns
//      the fold records l, l + 32, ... of its four pairs and keeps their
//      smoothed R (both bins of each record, as R / alpha) in registers across
//      the chunk's frames; per frame it updates R, applies the phase transform
//      and folds (Eq. 8) into the warp's shared-memory rows.  Then each lane
//      projects one row over a quarter of the records onto the bases of its
//      parity (Eqs. 7, 9), and 8 lanes per pair reconstruct the lag grid,
//      argmax and refinement as the FP32 path.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "fcc_device.cuh"
#include "fcc_internal.h"
#include "fcc_smooth.h"

namespace fcc {
namespace {

constexpr int kSmoothStages = 2;

struct SmoothParams {
    const float2 *spectra;  // [T][M][B]
    long long T;
    int M, B, Q, P, n_slots;
    int chunk, n_chunks;    // frames per chunk
    float alpha, beta;      // beta = 1 - alpha
    const float2 *carry;    // [n_chunks][P][B]: the state entering each chunk
    const float *basis;     // folded form: [2][QP / 2][KH / 2][4] (parity, record pair, two bases x two records); zero past K and Q
    const float *recon;     // [center + 1][KH][4]
    const Slot *slots;
    int center, I, KE, KO;
    float delta;
    int *out_idx;
    float *out_peak;
    float *out_tau;
    float *out_coef;
    float *out_corr;        // nullable, [T][P][I]
    unsigned *err;
    long long wait_cycles;
    int inject;             // test hook: CTA 0 withholds the copy of its first frame
};

// Pass 1: the recursion run from zero over each chunk.  One CTA per chunk, one
// thread per bin f: per frame it loads the M microphones' X(f) once (coalesced
// across the CTA, so each frame is read from HBM once) and updates the running
// sums of all P pairs in registers.
template <int M>
__global__ void chunk_sums_kernel(const float2 *X, long long T, int B, int chunk, float alpha, float beta,
                                  float2 *sums)
{
    constexpr int P = M * (M - 1) / 2;
    const int c = blockIdx.x, f = threadIdx.x;
    if (f >= B) return;
    const long long t0 = (long long)c * chunk, t1 = min(T, t0 + chunk);
    f2 acc[P];
#pragma unroll
    for (int q = 0; q < P; ++q) acc[q] = 0ull;
    const f2 beta2 = pk(beta, beta);
    const float2 *xp = X + (size_t)t0 * M * B + f;
    for (long long t = t0; t < t1; ++t, xp += (size_t)M * B) {
        float2 x[M];
#pragma unroll
        for (int m = 0; m < M; ++m) x[m] = __ldg(xp + (size_t)m * B);
        int q = 0;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const f2 xa = pk(x[i].x, x[i].y), xw = pk(x[i].y, x[i].x);
#pragma unroll
            for (int j = i + 1; j < M; ++j, ++q) {
                // alpha x_i x_j^* = (xr yr + xi yi, xi yr - xr yi) alpha
                const f2 yr = pk(alpha * x[j].x, alpha * x[j].x), yi = pk(alpha * x[j].y, -alpha * x[j].y);
                acc[q] = fma2(beta2, acc[q], fma2(xw, yi, mul2(xa, yr)));
            }
        }
    }
#pragma unroll
    for (int q = 0; q < P; ++q) {
        float re, im;
        upk(acc[q], re, im);
        sums[((size_t)c * P + q) * B + f] = make_float2(re, im);
    }
}

// Pass 2: the state entering each chunk (written over the chunk sums) and the
// state after the last frame.  The chunk sums are loaded kCarryBatch at a time
// ahead of the dependent updates, so the loads overlap.
constexpr int kCarryBatch = 16;
__global__ void carry_kernel(float2 *sums_to_carry, int PB, int n_chunks, long long T, int chunk, float beta,
                             const float2 *state_in, float2 *state_out)
{
    const float decay_full = powf(beta, (float)chunk);
    const long long last_len = T - (long long)(n_chunks - 1) * chunk;
    const float decay_last = powf(beta, (float)last_len);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < PB; e += gridDim.x * blockDim.x) {
        float2 S = state_in ? state_in[e] : make_float2(0.f, 0.f);
        for (int c0 = 0; c0 < n_chunks; c0 += kCarryBatch) {
            float2 L[kCarryBatch];
#pragma unroll
            for (int u = 0; u < kCarryBatch; ++u)
                if (c0 + u < n_chunks) L[u] = sums_to_carry[(size_t)(c0 + u) * PB + e];
#pragma unroll
            for (int u = 0; u < kCarryBatch; ++u)
                if (c0 + u < n_chunks) {
                    const float decay = c0 + u == n_chunks - 1 ? decay_last : decay_full;
                    sums_to_carry[(size_t)(c0 + u) * PB + e] = S;
                    S.x = fmaf(decay, S.x, L[u].x);
                    S.y = fmaf(decay, S.y, L[u].y);
                }
        }
        if (state_out) state_out[e] = S;
    }
}

// Shared-memory layout of fcc_smooth_kernel, the same on host and device.
// Per warp: 8 rows (2 q + d: pair q's folded x_s for d = 0, x_d for d = 1) of
// QP = Q + 1 records rounded up to 4, at a row stride of QP * 8 + 16 bytes (an
// odd multiple of 16 modulo 128, so the 8 rows at one record fall into 8
// different 16-byte bank groups), then the pairs' 2 KH coefficients, then the
// four pairs' smoothed R at the lone bin N/4.
struct SmoothLayout {
    int QP, rows, row_bytes, warp_bytes;
    size_t basis_off, recon_off, warps_off, stages_off, stage_bytes, total;
    __host__ __device__ SmoothLayout(int Q, int KH, int center, int M, int B, int n_warps, bool FB)
    {
        // folded form: 8 rows (x_s, x_d of 4 pairs) of records 0..Q; split form:
        // 4 rows (R_hat of 4 pairs) of bins 0..2Q, whose weights stay in global memory
        QP = FB ? (2 * Q + 4) : ((Q + 4) & ~3);
        rows = FB ? 4 : 8;
        row_bytes = QP * 8 + 16;
        warp_bytes = (rows * row_bytes + 4 * 2 * KH * 8 + 4 * 8 + 127) & ~127;
        basis_off = 128 + 8 * sizeof(Slot);
        recon_off = basis_off + (FB ? 0 : (size_t)2 * KH * QP * 4);
        warps_off = (recon_off + (size_t)(center + 1) * 4 * KH * 4 + 127) & ~(size_t)127;
        stages_off = warps_off + (size_t)n_warps * warp_bytes;
        stage_bytes = ((size_t)M * B * 8 + 127) & ~(size_t)127;
        total = stages_off + kSmoothStages * stage_bytes;
    }
};

// Pass 3.  One warp per 2x2 pair slot; per frame:
//   state    lane l owns records l, l + 32, ... (both bins f and N/2 - f) of the
//            slot's four pairs and keeps their R in registers: Eq. 1 update,
//            R_hat = R / |R|, fold (Eq. 8), x_s and x_d written to the warp's rows;
//   project  (Eqs. 7, 9) in the folded form lane (rq, q, par) takes pair q's
//            x_s (par 0) or x_d (par 1) row over record pairs rq, rq + 4, ...
//            against all KH bases of that parity (each row element read once;
//            the shared-memory pipe is this pass's bound), and the four record
//            quarters add with two shuffles; in the split form lane (q, i)
//            forms coefficient(s) i * CPL.. over all bins;
//   search   8 lanes per pair split the lag steps of the reconstruction, then
//            argmax and refinement as the FP32 path.
// R / |R| without a branch: R is first scaled by the power of two that brings
// max(|Re R|, |Im R|) into [1, 2) (the scale is clamped to >= 2^-126, so the
// largest finite R lands in [2, 4)), which keeps |R|^2 normal for any finite
// R.  R = 0 gives 0 (the rsqrt argument is floored at FLT_MIN); a non-finite R
// flags the error word.
__device__ __forceinline__ f2 unit_scaled(float rx, float ry, bool &bad)
{
    const int eb = (int)(__float_as_uint(fmaxf(fabsf(rx), fabsf(ry))) & 0x7f800000u);
    const float sc = __int_as_float(max(0x7f000000 - eb, 0x00800000));
    const f2 ab = mul2(pk(rx, ry), pk(sc, sc));
    float a, b;
    upk(ab, a, b);
    const float s = fmaf(a, a, b * b);
    bad = bad || !(s < 64.f);
    const float r = rsqrtf(fmaxf(s, FLT_MIN));
    return mul2(ab, pk(r, r));
}

// R / |R| without the scaling, valid when |R|^2 is a normal FP32 number; ok is
// cleared otherwise (zero, tiny, huge or non-finite R), and the warp then redoes
// the frame with unit_scaled.  In the normal range both give the same value: the
// scaling is by a power of two, and |R|^2 by a power of four.
__device__ __forceinline__ f2 unit_fast(f2 R, bool &ok)
{
    float rx, ry;
    upk(R, rx, ry);
    const float s = fmaf(rx, rx, ry * ry);
    ok = ok && (s >= FLT_MIN) && (s <= FLT_MAX);
    const float r = rsqrtf(s);
    return mul2(R, pk(r, r));
}

// Eq. 1 on R / alpha: beta R + x y^*, with the cross spectrum
// x y^* = (xr yr + xi yi, xi yr - xr yi) folded into the FMA chain.
__device__ __forceinline__ f2 cross_update(f2 R, float2 x, float2 y, f2 beta2)
{
    float bx, by;
    upk(mul2(beta2, R), bx, by);
    return pk(fmaf(x.x, y.x, fmaf(x.y, y.y, bx)), fmaf(x.y, y.x, fmaf(-x.x, y.y, by)));
}

// FB (the split form): the rows hold R_hat at bins 0..N/2 unfolded, the
// projection pairs the cosine weight with Re and the sine weight with Im in one
// FFMA2 ((c_k, s_k) per coefficient), and the reconstruction table holds
// (2 U_c, 2 U_s) so the same S -/+ D evaluation gives y = 2 (U_c c - U_s s).
template <int KH, int RS, bool FB>
__global__ void __launch_bounds__(256, 2) fcc_smooth_kernel(const __grid_constant__ SmoothParams p)
{
    constexpr int CPL = KH > 4 ? 2 : 1;  // coefficients per projecting lane (split form)
    extern __shared__ __align__(128) unsigned char smem[];
    const SmoothLayout Ly(p.Q, KH, p.center, p.M, p.B, p.n_slots, FB);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *freed = full + kSmoothStages;
    Slot *slots = reinterpret_cast<Slot *>(smem + 128);
    float *basis = reinterpret_cast<float *>(smem + Ly.basis_off);  // [2 KH][QP]
    float *recon = reinterpret_cast<float *>(smem + Ly.recon_off);
    unsigned char *stages = smem + Ly.stages_off;
    const int frame_bytes = p.M * p.B * 8;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the host launches the instance with Q = 32 RS (N = 128 RS), so the row
    // geometry of SmoothLayout is known here and addresses fold into immediates
    constexpr int Q = 32 * RS, B = 2 * Q + 1;
    constexpr int QP = FB ? (2 * Q + 4) : ((Q + 4) & ~3);
    constexpr int ROWB = QP * 8 + 16;
    const unsigned FULLM = 0xffffffffu;
    const int nw = p.n_slots;  // one warp per slot
    if (threadIdx.x == 0) {
        for (int s = 0; s < kSmoothStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&freed[s], (unsigned)nw);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int e = threadIdx.x; e < p.n_slots; e += blockDim.x) slots[e] = p.slots[e];
    if (!FB)
        for (int e = threadIdx.x; e < 2 * KH * QP; e += blockDim.x) basis[e] = p.basis[e];
    for (int e = threadIdx.x; e < (p.center + 1) * 4 * KH; e += blockDim.x) recon[e] = p.recon[e];
    unsigned char *wreg = smem + Ly.warps_off + (size_t)warp * Ly.warp_bytes;
    // the padding entries past the last record (bin) stay zero (their weights are zero too)
    const int used = FB ? 2 * Q + 1 : Q + 1, npad = QP - used;
    for (int e = lane; e < Ly.rows * npad; e += 32)
        reinterpret_cast<float2 *>(wreg + (size_t)(e / npad) * ROWB)[used + e % npad] = make_float2(0.f, 0.f);
    fence_proxy_async();
    __syncthreads();

    const Slot sl = slots[warp];
    float2 *zbuf = reinterpret_cast<float2 *>(wreg + (size_t)Ly.rows * ROWB);  // [4][2 KH]
    f2 *Rl = reinterpret_cast<f2 *>(zbuf + 4 * 2 * KH);                 // [4]: pair q's, kept by lane q
    bool bad = false, failed = false;
    // This CTA's frames as one sequence g = i * chunk + k over its chunks
    // c_i = blockIdx.x + i * gridDim.x (only the global last chunk can be short,
    // and it is the last one of its CTA); frame g lives in stage g % S.
    const int my_chunks = p.n_chunks > (int)blockIdx.x ? (p.n_chunks - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    long long total_g = 0;
    if (my_chunks > 0) {
        const long long c_last = (long long)blockIdx.x + (long long)(my_chunks - 1) * gridDim.x;
        total_g = (long long)(my_chunks - 1) * p.chunk + min((long long)p.chunk, p.T - c_last * p.chunk);
    }
    auto frame_of = [&](long long g) {
        const long long i = g / p.chunk, k = g - i * p.chunk;
        return ((long long)blockIdx.x + i * gridDim.x) * p.chunk + k;
    };
    auto issue = [&](long long g) {
        const int s = (int)(g % kSmoothStages);
        mbar_arrive_expect_tx(&full[s], (unsigned)frame_bytes);
        bulk_g2s(stages + (size_t)s * Ly.stage_bytes,
                 reinterpret_cast<const unsigned char *>(p.spectra) + (size_t)frame_of(g) * frame_bytes,
                 (unsigned)frame_bytes, &full[s]);
    };
    long long issued = 0, g = 0;
    // the test hook withholds CTA 0's first frame: every warp's first wait runs out
    // (bounded), the launch finishes and the error word reports the timeout
    const long long withheld = (p.inject && blockIdx.x == 0) ? 0 : -1;
    if (threadIdx.x == 0)
        for (; issued < kSmoothStages && issued < total_g; ++issued)
            if (issued != withheld) issue(issued);
    const f2 beta2 = pk(p.beta, p.beta);
    for (int ci = 0; ci < my_chunks && !failed; ++ci) {
        const int c = (int)blockIdx.x + ci * (int)gridDim.x;
        const long long t0 = (long long)c * p.chunk;
        const int len = (int)min((long long)p.chunk, p.T - t0);
        // the state entering this chunk, R of the slot's four pairs at this lane's
        // records, held as R / alpha: then R / alpha <- beta R / alpha + X_i X_j^*
        // needs no scaling per frame, and the phase transform is unchanged
        const f2 ia2 = pk(1.f / p.alpha, 1.f / p.alpha);
        f2 R[4][RS][2];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int pq = sl.pair[q] >= 0 ? sl.pair[q] : 0;
            // no carry (alpha = 1): every chunk starts from R = 0
            const float2 *cs = p.carry ? p.carry + ((size_t)c * p.P + pq) * B : nullptr;
#pragma unroll
            for (int j = 0; j < RS; ++j) {
                const int fp = lane + 32 * j;
                const float2 u = cs ? cs[fp] : make_float2(0.f, 0.f), v = cs ? cs[2 * Q - fp] : make_float2(0.f, 0.f);
                R[q][j][0] = mul2(ia2, pk(u.x, u.y));
                R[q][j][1] = mul2(ia2, pk(v.x, v.y));
            }
            if (lane == q) {  // the lane that updates pair q's lone bin
                const float2 w = cs ? cs[Q] : make_float2(0.f, 0.f);
                Rl[q] = mul2(ia2, pk(w.x, w.y));
            }
        }
#pragma unroll 1
        for (int k = 0; k < len; ++k, ++g) {
            // refill the stage of frame g - 1 with frame g - 1 + S once every warp released it
            if (threadIdx.x == 0 && g > 0 && issued < total_g) {
                const long long h = g - 1;
                if (!mbar_wait(&freed[h % kSmoothStages], (unsigned)(h / kSmoothStages) & 1u, p.wait_cycles)) {
                    atomicOr(p.err, kErrTimeout);
                } else {
                    issue(issued);
                    ++issued;
                }
            }
            const int s = (int)(g % kSmoothStages);
            if (!mbar_wait(&full[s], (unsigned)(g / kSmoothStages) & 1u, p.wait_cycles)) {
                failed = true;
                break;
            }
            const unsigned char *st = stages + (size_t)s * Ly.stage_bytes;
            const float2 *row[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) row[r] = reinterpret_cast<const float2 *>(st + (size_t)sl.mic[r] * B * 8);
            // ---- state: Eq. 1, phase transform, fold (Eq. 8)
            auto put = [&](int q, int fp, f2 ua, f2 ub) {
                if (FB) {
                    reinterpret_cast<f2 *>(wreg + (size_t)q * ROWB)[fp] = ua;
                    reinterpret_cast<f2 *>(wreg + (size_t)q * ROWB)[2 * Q - fp] = ub;
                } else {
                    reinterpret_cast<f2 *>(wreg + (size_t)(2 * q) * ROWB)[fp] = add2(ua, ub);
                    reinterpret_cast<f2 *>(wreg + (size_t)(2 * q + 1) * ROWB)[fp] = sub2(ua, ub);
                }
            };
            bool ok = true;
#pragma unroll
            for (int j = 0; j < RS; ++j) {
                const int fp = lane + 32 * j;
                float2 xf[2], xb[2], yf[2], yb[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    xf[u] = row[u][fp];
                    xb[u] = row[u][2 * Q - fp];
                    yf[u] = row[2 + u][fp];
                    yb[u] = row[2 + u][2 * Q - fp];
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    R[q][j][0] = cross_update(R[q][j][0], xf[q >> 1], yf[q & 1], beta2);
                    R[q][j][1] = cross_update(R[q][j][1], xb[q >> 1], yb[q & 1], beta2);
                    put(q, fp, unit_fast(R[q][j][0], ok), unit_fast(R[q][j][1], ok));
                }
            }
            if (!__all_sync(FULLM, ok)) {
                // some |R|^2 of the frame is not a normal FP32 number: the whole warp
                // redoes the frame's phase transform in the scaled form
#pragma unroll
                for (int j = 0; j < RS; ++j)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float r0x, r0y, r1x, r1y;
                        upk(R[q][j][0], r0x, r0y);
                        upk(R[q][j][1], r1x, r1y);
                        put(q, lane + 32 * j, unit_scaled(r0x, r0y, bad), unit_scaled(r1x, r1y, bad));
                    }
            }
            if (lane < 4) {
                // the lone bin N/4, one pair per lane: x_s = R_hat(N/4), x_d = 0 (Eq. 8)
                const int q = lane;
                const float2 x = ((q & 2) ? row[1] : row[0])[Q], y = ((q & 1) ? row[3] : row[2])[Q];
                const f2 r = cross_update(Rl[q], x, y, beta2);
                Rl[q] = r;
                float rx, ry;
                upk(r, rx, ry);
                const f2 u = unit_scaled(rx, ry, bad);
                if (FB) {
                    reinterpret_cast<f2 *>(wreg + (size_t)q * ROWB)[Q] = u;
                } else {
                    reinterpret_cast<f2 *>(wreg + (size_t)(2 * q) * ROWB)[Q] = u;
                    reinterpret_cast<f2 *>(wreg + (size_t)(2 * q + 1) * ROWB)[Q] = 0ull;
                }
            }
            // the stage is read: release it (thread 0 refills it at the next frame)
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&freed[s]);
            // ---- project (Eqs. 7, 9): lanes 8 q .. 8 q + 7 form pair q's coefficients
            {
                const int q = lane >> 3, v0 = (lane & 7) * CPL;
                if (FB && v0 < 2 * KH) {
                    // (c_k, s_k) += (w_c, w_s) * (Re R_hat, Im R_hat), two bins per 16-byte load
                    const float4 *dat = reinterpret_cast<const float4 *>(wreg + (size_t)q * ROWB);
                    f2 acc[CPL];
#pragma unroll
                    for (int cc = 0; cc < CPL; ++cc) acc[cc] = 0ull;
#pragma unroll 4
                    for (int r2 = 0; r2 < QP / 2; ++r2) {
                        const float4 d = dat[r2];
#pragma unroll
                        for (int cc = 0; cc < CPL; ++cc) {
                            const float4 w = __ldg(reinterpret_cast<const float4 *>(p.basis) + (size_t)(v0 + cc) * (QP / 2) + r2);
                            acc[cc] = fma2(pk(w.x, w.y), pk(d.x, d.y), acc[cc]);
                            acc[cc] = fma2(pk(w.z, w.w), pk(d.z, d.w), acc[cc]);
                        }
                    }
#pragma unroll
                    for (int cc = 0; cc < CPL; ++cc) reinterpret_cast<f2 *>(zbuf)[q * 2 * KH + v0 + cc] = acc[cc];
                } else if (!FB) {
                    // lane (rq, qq, par): pair qq's row of parity par (x_s or x_d) over the
                    // record pairs u = rq, rq + 4, ... against all KH bases of that parity,
                    // so each row element is read once; a quarter-warp shares its record
                    // pairs, whose weights (grouped per record pair) it reads in one
                    // wavefront; the four record quarters add with two shuffles
                    const int rq = lane >> 3, qq = (lane >> 1) & 3, par = lane & 1;
                    const float4 *dat = reinterpret_cast<const float4 *>(wreg + (size_t)(2 * qq + par) * ROWB);
                    const float4 *wv = reinterpret_cast<const float4 *>(basis) + (size_t)par * (QP / 2) * (KH / 2);
                    f2 acc[KH];
#pragma unroll
                    for (int k = 0; k < KH; ++k) acc[k] = 0ull;
#pragma unroll 2
                    for (int u = rq; u < QP / 2; u += 4) {
                        const float4 d = dat[u];  // records 2u, 2u + 1 as (re, im, re, im)
                        const f2 d0 = pk(d.x, d.y), d1 = pk(d.z, d.w);
#pragma unroll
                        for (int k2 = 0; k2 < KH / 2; ++k2) {
                            // (w_{2k2}(2u), w_{2k2}(2u+1), w_{2k2+1}(2u), w_{2k2+1}(2u+1))
                            const float4 w = wv[(size_t)u * (KH / 2) + k2];
                            acc[2 * k2] = fma2(pk(w.y, w.y), d1, fma2(pk(w.x, w.x), d0, acc[2 * k2]));
                            acc[2 * k2 + 1] = fma2(pk(w.w, w.w), d1, fma2(pk(w.z, w.z), d0, acc[2 * k2 + 1]));
                        }
                    }
#pragma unroll
                    for (int k = 0; k < KH; ++k) {
                        acc[k] = add2(acc[k], __shfl_xor_sync(FULLM, acc[k], 8));
                        acc[k] = add2(acc[k], __shfl_xor_sync(FULLM, acc[k], 16));
                    }
#pragma unroll
                    for (int k = 0; k < KH; ++k)
                        if ((k & 3) == rq) reinterpret_cast<f2 *>(zbuf)[qq * 2 * KH + par * KH + k] = acc[k];
                }
            }
            __syncwarp();
            // ---- lag grid: the 8 lanes holding a pair split the steps m = gi, gi + 8, ...
            const int q = lane & 3, gi = lane >> 2;
            // the coefficients are read from the warp's buffer where used (the R state holds the registers)
            const f2 *zE = reinterpret_cast<const f2 *>(zbuf) + q * 2 * KH, *zO = zE + KH;
            const int pq = q == 0 ? sl.pair[0] : q == 1 ? sl.pair[1] : q == 2 ? sl.pair[2] : sl.pair[3];
            float best = -FLT_MAX;
            int bi = 0x7fffffff;
            if (pq >= 0) {
                float *corr = p.out_corr ? p.out_corr + ((size_t)(t0 + k) * p.P + pq) * p.I : nullptr;
                float S, D;
                int m = gi;
                if (gi == 0) {
                    eval_SD<KH>(recon, 0, zE, zO, S, D);
                    best = S - D;
                    bi = p.center;
                    if (corr) corr[p.center] = best;
                    m = 8;
                }
                for (; m <= p.center; m += 8) {
                    eval_SD<KH>(recon, m, zE, zO, S, D);
                    const float ym = S + D, yp = S - D;
                    if (ym >= best) {
                        best = ym;
                        bi = p.center - m;
                    }
                    if (yp > best) {
                        best = yp;
                        bi = p.center + m;
                    }
                    if (corr) {
                        corr[p.center - m] = ym;
                        corr[p.center + m] = yp;
                    }
                }
            }
#pragma unroll
            for (int off = 4; off < 32; off <<= 1) {
                const float ob = __shfl_xor_sync(FULLM, best, off);
                const int oi = __shfl_xor_sync(FULLM, bi, off);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (pq >= 0 && gi == 0) {
                const size_t o = (size_t)(t0 + k) * p.P + pq;
                p.out_idx[o] = bi;
                p.out_peak[o] = best;
                if (p.out_tau) {
                    float off = 0.f;
                    if (bi > 0 && bi < p.I - 1) {
                        const double y_m = y_at<KH>(recon, p.center, bi - 1, zE, zO);
                        const double y_p = y_at<KH>(recon, p.center, bi + 1, zE, zO);
                        const double num = y_m - y_p;
                        const double den = (y_m - 2.0 * (double)best) + y_p;
                        if (den < 0.0) off = fminf(0.5f, fmaxf(-0.5f, 0.5f * (float)num / (float)den));
                    }
                    p.out_tau[o] = ((float)(bi - p.center) + off) * p.delta;
                }
                if (!FB && p.out_coef) {
                    const int K = p.KE + p.KO;
                    float *cf = p.out_coef + o * 2 * K;
#pragma unroll
                    for (int v = 0; v < KH; ++v) {
                        float a, b2;
                        if (v < p.KE) {
                            upk(zE[v], a, b2);
                            cf[v] = a;
                            cf[p.KE + v] = b2;
                        }
                        if (v < p.KO) {
                            upk(zO[v], a, b2);
                            cf[2 * p.KE + v] = a;
                            cf[2 * p.KE + p.KO + v] = b2;
                        }
                    }
                }
            }
        }
        failed = __syncthreads_or(failed);
    }
    if (__any_sync(FULLM, bad) && lane == 0) atomicOr(p.err, kErrNonFinite);
    if (failed && threadIdx.x == 0) atomicOr(p.err, kErrTimeout);
    // never retire with a bulk copy in flight: frames issued but not consumed
    // (a withheld frame was never issued, so there is nothing to wait for)
    if (threadIdx.x == 0)
        for (long long h = g; h < issued; ++h)
            if (h != withheld &&
                !mbar_wait(&full[h % kSmoothStages], (unsigned)(h / kSmoothStages) & 1u, p.wait_cycles)) {
                atomicOr(p.err, kErrTimeout);
                break;
            }
}

}  // namespace
}  // namespace fcc

namespace fcc {
namespace {

struct SmoothPlan {
    int chunk, n_chunks, threads;
    size_t smem, work_bytes;
};

bool is_split(const fcc_plan *plan) { return plan->info.form == FCC_FORM_REIM_SPLIT; }

fcc_status_t smooth_geometry(const fcc_plan *plan, long long T, SmoothPlan &g)
{
    const fcc_plan_info_t &in = plan->info;
    const char *what = is_split(plan) ? "the smoothed split form" : "the smoothed path";
    if (in.prec != FCC_PREC_FP32) return fail(FCC_ERR_UNSUPPORTED, std::string(what) + " is FP32");
    if (in.M % 2) return fail(FCC_ERR_UNSUPPORTED, std::string(what) + " needs an even number of mics");
    if (plan->n_slots > 8) return fail(FCC_ERR_UNSUPPORTED, std::string(what) + " needs at most 8 mics");
    if (in.Q < 32 || in.Q > 128) return fail(FCC_ERR_UNSUPPORTED, std::string(what) + " needs 128 <= N <= 512");
    if (!plan->kh) return fail(FCC_ERR_UNSUPPORTED, "too many bases for the per-pair kernel");
    const long long target = 4LL * plan->num_sms;
    g.chunk = (int)std::max<long long>(64, (T + target - 1) / target);
    g.n_chunks = (int)((T + g.chunk - 1) / g.chunk);
    g.threads = 32 * plan->n_slots;
    const SmoothLayout Ly(in.Q, plan->kh, in.center, in.M, in.B, plan->n_slots, is_split(plan));
    g.smem = Ly.total;
    g.work_bytes = (size_t)g.n_chunks * in.P * in.B * sizeof(float2);
    return FCC_OK;
}

// grid = min(chunks, resident CTAs): the CTAs are persistent over chunks
template <int KH, int RS, bool FB>
fcc_status_t launch_smooth_inst(const SmoothParams &prm, int num_sms, int threads, size_t smem, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(fcc_smooth_kernel<KH, RS, FB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(fcc_smooth_kernel)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fcc_smooth_kernel<KH, RS, FB>, threads, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm < 1) return fail(FCC_ERR_UNSUPPORTED, "the per-pair kernel does not fit an SM");
    const int grid = (int)std::min<long long>(prm.n_chunks, (long long)num_sms * per_sm);
    fcc_smooth_kernel<KH, RS, FB><<<grid, threads, smem, st>>>(prm);
    e = cudaGetLastError();
    return e == cudaSuccess ? FCC_OK : cuda_fail(e, "fcc_smooth_kernel launch");
}

template <int KH, bool FB>
fcc_status_t launch_smooth_kh(int rs, const SmoothParams &prm, int num_sms, int threads, size_t smem, cudaStream_t st)
{
    switch (rs) {
    case 1: return launch_smooth_inst<KH, 1, FB>(prm, num_sms, threads, smem, st);
    case 2: return launch_smooth_inst<KH, 2, FB>(prm, num_sms, threads, smem, st);
    case 4: return launch_smooth_inst<KH, 4, FB>(prm, num_sms, threads, smem, st);
    default: return fail(FCC_ERR_UNSUPPORTED, "the per-pair kernel needs 128 <= N <= 512");
    }
}

template <bool FB>
fcc_status_t launch_smooth_form(int kh, int rs, const SmoothParams &prm, int num_sms, int threads, size_t smem,
                                cudaStream_t st)
{
    switch (kh) {
    case 2: return launch_smooth_kh<2, FB>(rs, prm, num_sms, threads, smem, st);
    case 4: return launch_smooth_kh<4, FB>(rs, prm, num_sms, threads, smem, st);
    case 6: return launch_smooth_kh<6, FB>(rs, prm, num_sms, threads, smem, st);
    case 8: return launch_smooth_kh<8, FB>(rs, prm, num_sms, threads, smem, st);
    default: return fail(FCC_ERR_UNSUPPORTED, "too many bases for the per-pair kernel");
    }
}

}  // namespace

// Folded-form weights in the per-pair kernel's layout: row v < KH = even basis v
// over records 0..Q, row KH + v = odd basis v (zero at Q); padding records zero.
// Built when the plan is created, so the smoothed path never allocates.
fcc_status_t prepare_per_pair(fcc_plan *plan)
{
    if (plan->d_smooth_basis) return FCC_OK;
    const fcc_plan_info_t &in = plan->info;
    const int kh = plan->kh, Q = in.Q;
    const SmoothLayout Ly(Q, kh, in.center, in.M, in.B, plan->n_slots, false);
    // [parity][record pair u][k / 2][(k, 2u), (k, 2u + 1), (k + 1, 2u), (k + 1, 2u + 1)]:
    // the kernel's lane reads one float4 per two bases and two records
    std::vector<float> bas((size_t)2 * kh * Ly.QP, 0.f);
    auto put = [&](int par, int k, int f, double w) {
        const int u = f / 2, r = f % 2;
        bas[(((size_t)par * (Ly.QP / 2) + u) * (kh / 2) + k / 2) * 4 + (k % 2) * 2 + r] = (float)w;
    };
    for (int k = 0; k < in.K_even; ++k)
        for (int f = 0; f <= Q; ++f) put(0, k, f, plan->Pe[(size_t)k * (Q + 1) + f]);
    for (int k = 0; k < in.K_odd; ++k)
        for (int f = 0; f < Q; ++f) put(1, k, f, plan->Po[(size_t)k * Q + f]);
    float *d = nullptr;
    FCC_CUDA_TRY(dev_alloc((void **)&d, bas.size() * sizeof(float)));
    cudaError_t e = cudaMemcpy(d, bas.data(), bas.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "cudaMemcpy(per-pair weights)");
    }
    plan->d_smooth_basis = d;
    return FCC_OK;
}

namespace {

// The per-pair kernel over T frames: `carry` (may be null: every chunk starts
// from R = 0, which is exact for alpha = 1) holds the state entering each chunk.
fcc_status_t run_per_pair(const fcc_plan *plan, const SmoothPlan &g, const float2 *spectra, long long T, float a,
                          float b, const float2 *carry, int *idx, float *peak, float *tau, float *coef, float *corr,
                          cudaStream_t s)
{
    const fcc_plan_info_t &in = plan->info;
    SmoothParams prm{};
    prm.spectra = spectra;
    prm.T = T;
    prm.M = in.M;
    prm.B = in.B;
    prm.Q = in.Q;
    prm.P = in.P;
    prm.n_slots = plan->n_slots;
    prm.chunk = g.chunk;
    prm.n_chunks = g.n_chunks;
    prm.alpha = a;
    prm.beta = b;
    prm.carry = carry;
    prm.basis = plan->d_smooth_basis;
    prm.recon = plan->d_recon;
    prm.slots = plan->d_slots;
    prm.center = in.center;
    prm.I = in.I;
    prm.KE = in.K_even;
    prm.KO = in.K_odd;
    prm.delta = (float)in.delta;
    prm.out_idx = idx;
    prm.out_peak = peak;
    prm.out_tau = tau;
    prm.out_coef = coef;
    prm.out_corr = corr;
    prm.err = plan->d_err;
    DebugHooks &dh = debug_hooks();
    prm.wait_cycles = dh.wait_cycles;
    prm.inject = 0;
    if (dh.withhold_copies > 0) {
        --dh.withhold_copies;
        prm.inject = 1;
    }
    const int rs = in.Q / 32;
    return is_split(plan) ? launch_smooth_form<true>(plan->kh, rs, prm, plan->num_sms, g.threads, g.smem, s)
                          : launch_smooth_form<false>(plan->kh, rs, prm, plan->num_sms, g.threads, g.smem, s);
}

}  // namespace

// Split-form weights for the per-pair kernel (Eq. 1 smoothing), built once when
// the plan is created: [2 KH][2Q + 4] (cosine, sine) pairs, sigma v_k of C and
// of S over bins 0..N/2, zero past K_c / K_s and in the padding.  The
// reconstruction table is the FP32 kernel's split-form table (pack_tables).
fcc_status_t prepare_reim(fcc_plan *plan)
{
    const fcc_plan_info_t &in = plan->info;
    const int kh = plan->kh, B = in.B, Kc = in.K_even, Ks = in.K_odd;
    const SmoothLayout Ly(in.Q, kh, in.center, in.M, in.B, std::max(plan->n_slots, 1), true);
    std::vector<float> w((size_t)2 * kh * Ly.QP * 2, 0.f);
    for (int k = 0; k < 2 * kh; ++k)
        for (int f = 0; f < B; ++f) {
            w[((size_t)k * Ly.QP + f) * 2] = k < Kc ? (float)plan->Pe[(size_t)k * B + f] : 0.f;
            w[((size_t)k * Ly.QP + f) * 2 + 1] = k < Ks ? (float)plan->Po[(size_t)k * B + f] : 0.f;
        }
    float *dw = nullptr;
    cudaError_t e = dev_alloc((void **)&dw, w.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(dw, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dw);
        return cuda_fail(e, "split-form per-pair weights");
    }
    cudaFree(plan->d_smooth_basis);
    plan->d_smooth_basis = dw;
    return FCC_OK;
}

}  // namespace fcc

using namespace fcc;

extern "C" {

fcc_status_t fcc_smooth_workspace(const fcc_plan_t *plan, long long T, long long *bytes)
{
    if (!plan || !bytes) return fail(FCC_ERR_INVALID_ARG, "null argument");
    if (T < 0) return fail(FCC_ERR_INVALID_ARG, "T < 0");
    SmoothPlan g{};
    fcc_status_t st = smooth_geometry(plan, std::max<long long>(T, 1), g);
    if (st != FCC_OK) return st;
    *bytes = T == 0 ? 0 : (long long)g.work_bytes;
    return FCC_OK;
}

fcc_status_t fcc_tdoa_smoothed(fcc_plan_t *plan, const void *d_spectra, long long T, double alpha, void *d_state,
                               void *d_work, long long work_bytes, int *d_lag_idx, float *d_peak, float *d_tau_hat,
                               float *d_coeffs, float *d_corr, void *stream)
{
    if (!plan) return fail(FCC_ERR_INVALID_ARG, "null plan");
    if (!(alpha > 0.0 && alpha <= 1.0)) return fail(FCC_ERR_INVALID_ARG, "alpha must be in (0, 1]");
    if (T < 0) return fail(FCC_ERR_INVALID_ARG, "T < 0");
    SmoothPlan g{};
    fcc_status_t st = smooth_geometry(plan, std::max<long long>(T, 1), g);
    if (st != FCC_OK) return st;
    if (T == 0) return FCC_OK;
    if (!d_spectra || !d_lag_idx || !d_peak || !d_work) return fail(FCC_ERR_INVALID_ARG, "null spectra/outputs/work");
    if (d_coeffs && is_split(plan)) return fail(FCC_ERR_UNSUPPORTED, "the split form has no coefficient output");
    if (reinterpret_cast<uintptr_t>(d_spectra) & 15) return fail(FCC_ERR_INVALID_ARG, "spectra not 16-byte aligned");
    if ((reinterpret_cast<uintptr_t>(d_state) | reinterpret_cast<uintptr_t>(d_work)) & 7)
        return fail(FCC_ERR_INVALID_ARG, "state / workspace not 8-byte aligned");
    if (work_bytes < (long long)g.work_bytes) return fail(FCC_ERR_INVALID_ARG, "workspace too small");
    const fcc_plan_info_t &in = plan->info;
    DeviceScope scope(plan->device);
    if (!scope.ok) return fail(FCC_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float a = (float)alpha, b = (float)(1.0 - alpha);
    float2 *work = static_cast<float2 *>(d_work);
    const int PB = in.P * in.B;
    // pass 1 and pass 2
    {
        const int threads = (in.B + 31) / 32 * 32;
        const float2 *X = static_cast<const float2 *>(d_spectra);
        switch (in.M) {
        case 2: chunk_sums_kernel<2><<<g.n_chunks, threads, 0, s>>>(X, T, in.B, g.chunk, a, b, work); break;
        case 4: chunk_sums_kernel<4><<<g.n_chunks, threads, 0, s>>>(X, T, in.B, g.chunk, a, b, work); break;
        case 6: chunk_sums_kernel<6><<<g.n_chunks, threads, 0, s>>>(X, T, in.B, g.chunk, a, b, work); break;
        case 8: chunk_sums_kernel<8><<<g.n_chunks, threads, 0, s>>>(X, T, in.B, g.chunk, a, b, work); break;
        default: return fail(FCC_ERR_UNSUPPORTED, "the smoothed path needs 2, 4, 6 or 8 mics");
        }
        carry_kernel<<<(PB + 127) / 128, 128, 0, s>>>(work, PB, g.n_chunks, T, g.chunk, b,
                                                      static_cast<const float2 *>(d_state),
                                                      static_cast<float2 *>(d_state));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "smoothing carry kernels");
    }
    if (!plan->d_smooth_basis) return fail(FCC_ERR_UNSUPPORTED, "the plan has no per-pair tables");
    return run_per_pair(plan, g, static_cast<const float2 *>(d_spectra), T, a, b, work, d_lag_idx, d_peak, d_tau_hat,
                        d_coeffs, d_corr, s);
}

}  // extern "C"
