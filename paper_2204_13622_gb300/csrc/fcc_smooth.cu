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
//   3. fcc_smooth_kernel  per chunk: one warp per 2x2 pair slot, lane l owns the
//      fold records l, l + 32, ... of its four pairs and keeps their smoothed R
//      (both bins of each record) in registers across the chunk's frames; per
//      frame it updates R, applies the phase transform, folds (Eq. 8) and
//      projects (Eqs. 7, 9); the 32 lanes reduce the projections with shuffles
//      and reconstruct the lag grid, argmax and refinement as the FP32 path.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "fcc_device.cuh"
#include "fcc_internal.h"
#include "fcc_smooth.h"

namespace fcc {
namespace {

constexpr int kSmoothStages = 4;

struct SmoothParams {
    const float2 *spectra;  // [T][M][B]
    long long T;
    int M, B, Q, P, n_slots;
    int chunk, n_chunks;    // frames per chunk
    float alpha, beta;      // beta = 1 - alpha
    const float2 *carry;    // [n_chunks][P][B]: the state entering each chunk
    const float *basis;     // [Q + 1][2 KH]: even weights, then odd (zero at N/4)
    const float *recon;     // [center + 1][KH][4]
    const Slot *slots;
    int center, I, KE, KO;
    float delta;
    int *out_idx;
    float *out_peak;
    float *out_tau;
    float *out_coef;
    unsigned *err;
    long long wait_cycles;
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
// state after the last frame.
__global__ void carry_kernel(float2 *sums_to_carry, int PB, int n_chunks, long long T, int chunk, float beta,
                             const float2 *state_in, float2 *state_out)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < PB; e += gridDim.x * blockDim.x) {
        float2 S = state_in ? state_in[e] : make_float2(0.f, 0.f);
        for (int c = 0; c < n_chunks; ++c) {
            const long long len = min((long long)chunk, T - (long long)c * chunk);
            const float decay = powf(beta, (float)len);
            const float2 Lc = sums_to_carry[(size_t)c * PB + e];
            sums_to_carry[(size_t)c * PB + e] = S;
            S.x = fmaf(decay, S.x, Lc.x);
            S.y = fmaf(decay, S.y, Lc.y);
        }
        if (state_out) state_out[e] = S;
    }
}

// R_hat = R / |R| (0 where R = 0; non-finite R flags the error word).
__device__ __forceinline__ f2 unit_of(float rx, float ry, bool &bad)
{
    const float s = fmaf(rx, rx, ry * ry);
    if (s >= FLT_MIN && s <= FLT_MAX) {
        const float r = rsqrtf(s);
        return mul2(pk(rx, ry), pk(r, r));
    }
    bool b2 = false;
    const float2 u = unit_phase_slow(make_float2(rx, ry), b2);
    bad = bad || b2;
    return pk(u.x, u.y);
}

template <int KH, int RS>
__global__ void __launch_bounds__(256, 1) fcc_smooth_kernel(const __grid_constant__ SmoothParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int frame_bytes = p.M * p.B * 8;
    const size_t stage_bytes = ((size_t)frame_bytes + 127) & ~(size_t)127;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *freed = full + kSmoothStages;
    Slot *slots = reinterpret_cast<Slot *>(smem + 128);
    float *basis = reinterpret_cast<float *>(smem + 128 + 8 * sizeof(Slot));
    const int nbasis = (p.Q + 1) * 2 * KH;
    float *recon = basis + nbasis;
    const size_t tab_end = (128 + 8 * sizeof(Slot) + (size_t)(nbasis + (p.center + 1) * 4 * KH) * 4 + 127) & ~(size_t)127;
    unsigned char *stages = smem + tab_end;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Q = p.Q, B = p.B, M = p.M;
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
    for (int e = threadIdx.x; e < nbasis; e += blockDim.x) basis[e] = p.basis[e];
    for (int e = threadIdx.x; e < (p.center + 1) * 4 * KH; e += blockDim.x) recon[e] = p.recon[e];
    fence_proxy_async();
    __syncthreads();

    const Slot sl = slots[warp];
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
        bulk_g2s(stages + (size_t)s * stage_bytes,
                 reinterpret_cast<const unsigned char *>(p.spectra) + (size_t)frame_of(g) * frame_bytes,
                 (unsigned)frame_bytes, &full[s]);
    };
    long long issued = 0, g = 0;
    if (threadIdx.x == 0)
        for (; issued < kSmoothStages && issued < total_g; ++issued) issue(issued);
    for (int ci = 0; ci < my_chunks && !failed; ++ci) {
        const int c = (int)blockIdx.x + ci * (int)gridDim.x;
        const long long t0 = (long long)c * p.chunk;
        const int len = (int)min((long long)p.chunk, p.T - t0);
        // the state entering this chunk: R of the slot's four pairs at this lane's records
        f2 R[4][RS][2], Rl[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int pq = sl.pair[q] >= 0 ? sl.pair[q] : 0;
            const float2 *cs = p.carry + ((size_t)c * p.P + pq) * B;
#pragma unroll
            for (int j = 0; j < RS; ++j) {
                const int fp = lane + 32 * j;
                const float2 u = cs[fp], v = cs[2 * Q - fp];
                R[q][j][0] = pk(u.x, u.y);
                R[q][j][1] = pk(v.x, v.y);
            }
            const float2 w = cs[Q];
            Rl[q] = pk(w.x, w.y);
        }
        const f2 beta2 = pk(p.beta, p.beta), alpha2 = pk(p.alpha, p.alpha);
        for (int k = 0; k < len; ++k, ++g) {
            const int s = (int)(g % kSmoothStages);
            const unsigned par = (unsigned)(g / kSmoothStages) & 1u;
            if (!mbar_wait(&full[s], par, p.wait_cycles)) {
                failed = true;
                break;
            }
            const unsigned char *st = stages + (size_t)s * stage_bytes;
            f2 accE[4][KH], accO[4][KH];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int v = 0; v < KH; ++v) accE[q][v] = accO[q][v] = 0ull;
            const float2 *row[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) row[r] = reinterpret_cast<const float2 *>(st + (size_t)sl.mic[r] * B * 8);
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
                const float4 *bw = reinterpret_cast<const float4 *>(basis + (size_t)fp * 2 * KH);
                float w[2 * KH];
#pragma unroll
                for (int v = 0; v < KH / 2; ++v) {
                    const float4 e = bw[v];
                    w[4 * v] = e.x;
                    w[4 * v + 1] = e.y;
                    w[4 * v + 2] = e.z;
                    w[4 * v + 3] = e.w;
                }
                // packed operands: x as (re, im) and (im, re), y as (re, re) and (im, -im),
                // so x y^* is one FMUL2 + one FFMA2 (scaled by alpha on the y side)
                f2 xa[2][2], xw[2][2], yr[2][2], yi[2][2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    xa[u][0] = pk(xf[u].x, xf[u].y);
                    xw[u][0] = pk(xf[u].y, xf[u].x);
                    xa[u][1] = pk(xb[u].x, xb[u].y);
                    xw[u][1] = pk(xb[u].y, xb[u].x);
                    yr[u][0] = pk(p.alpha * yf[u].x, p.alpha * yf[u].x);
                    yi[u][0] = pk(p.alpha * yf[u].y, -p.alpha * yf[u].y);
                    yr[u][1] = pk(p.alpha * yb[u].x, p.alpha * yb[u].x);
                    yi[u][1] = pk(p.alpha * yb[u].y, -p.alpha * yb[u].y);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int ix = q >> 1, iy = q & 1;
                    // Eq. 1 at f and N/2 - f (alpha X_i X_j^*), then the phase transform of R
                    const f2 a = fma2(xw[ix][0], yi[iy][0], mul2(xa[ix][0], yr[iy][0]));
                    const f2 b = fma2(xw[ix][1], yi[iy][1], mul2(xa[ix][1], yr[iy][1]));
                    R[q][j][0] = fma2(beta2, R[q][j][0], a);
                    R[q][j][1] = fma2(beta2, R[q][j][1], b);
                    float r0x, r0y, r1x, r1y;
                    upk(R[q][j][0], r0x, r0y);
                    upk(R[q][j][1], r1x, r1y);
                    const f2 ua = unit_of(r0x, r0y, bad), ub = unit_of(r1x, r1y, bad);
                    const f2 xs = add2(ua, ub), xd = sub2(ua, ub);  // Eq. 8
#pragma unroll
                    for (int v = 0; v < KH; ++v) {
                        accE[q][v] = fma2(pk(w[v], w[v]), xs, accE[q][v]);
                        accO[q][v] = fma2(pk(w[KH + v], w[KH + v]), xd, accO[q][v]);
                    }
                }
            }
            if (lane == 0) {
                // the lone bin N/4: x_s = R_hat(N/4), no odd part (Eq. 8)
                const float *bq = basis + (size_t)Q * 2 * KH;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 x = row[q >> 1][Q], y = row[2 + (q & 1)][Q];
                    const f2 a = pk(fmaf(x.x, y.x, x.y * y.y), fmaf(x.y, y.x, -(x.x * y.y)));
                    Rl[q] = fma2(beta2, Rl[q], mul2(alpha2, a));
                    float rx, ry;
                    upk(Rl[q], rx, ry);
                    const f2 ua = unit_of(rx, ry, bad);
#pragma unroll
                    for (int v = 0; v < KH; ++v) accE[q][v] = fma2(pk(bq[v], bq[v]), ua, accE[q][v]);
                }
            }
            // the stage is read: release it and refill it with frame g + S
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&freed[s]);
            if (threadIdx.x == 0 && issued < total_g) {
                if (!mbar_wait(&freed[s], par, p.wait_cycles)) {
                    atomicOr(p.err, kErrTimeout);
                } else {
                    issue(issued);
                    ++issued;
                }
            }
            // reduce-scatter over the 32 lanes: lane (l & 3) keeps pair (l & 3)
            f2 zE[KH], zO[KH];
            {
                const bool hi = (lane & 2) != 0;
                f2 rE[2][KH], rO[2][KH];
#pragma unroll
                for (int pp = 0; pp < 2; ++pp)
#pragma unroll
                    for (int v = 0; v < KH; ++v) {
                        float m0, m1, o0, o1;
                        upk(hi ? accE[pp + 2][v] : accE[pp][v], m0, m1);
                        upk(hi ? accE[pp][v] : accE[pp + 2][v], o0, o1);
                        rE[pp][v] = pk(m0 + __shfl_xor_sync(FULLM, o0, 2), m1 + __shfl_xor_sync(FULLM, o1, 2));
                        upk(hi ? accO[pp + 2][v] : accO[pp][v], m0, m1);
                        upk(hi ? accO[pp][v] : accO[pp + 2][v], o0, o1);
                        rO[pp][v] = pk(m0 + __shfl_xor_sync(FULLM, o0, 2), m1 + __shfl_xor_sync(FULLM, o1, 2));
                    }
                const bool b0 = (lane & 1) != 0;
#pragma unroll
                for (int v = 0; v < KH; ++v) {
                    float m0, m1, o0, o1;
                    upk(b0 ? rE[1][v] : rE[0][v], m0, m1);
                    upk(b0 ? rE[0][v] : rE[1][v], o0, o1);
                    float e0 = m0 + __shfl_xor_sync(FULLM, o0, 1), e1 = m1 + __shfl_xor_sync(FULLM, o1, 1);
                    upk(b0 ? rO[1][v] : rO[0][v], m0, m1);
                    upk(b0 ? rO[0][v] : rO[1][v], o0, o1);
                    float d0 = m0 + __shfl_xor_sync(FULLM, o0, 1), d1 = m1 + __shfl_xor_sync(FULLM, o1, 1);
#pragma unroll
                    for (int o = 4; o < 32; o <<= 1) {
                        e0 += __shfl_xor_sync(FULLM, e0, o);
                        e1 += __shfl_xor_sync(FULLM, e1, o);
                        d0 += __shfl_xor_sync(FULLM, d0, o);
                        d1 += __shfl_xor_sync(FULLM, d1, o);
                    }
                    zE[v] = pk(e0, e1);
                    zO[v] = pk(d0, d1);
                }
            }
            // lag grid: the 8 lanes holding a pair split the steps m = gi, gi + 8, ...
            const int q = lane & 3, gi = lane >> 2;
            const int pq = q == 0 ? sl.pair[0] : q == 1 ? sl.pair[1] : q == 2 ? sl.pair[2] : sl.pair[3];
            float best = -FLT_MAX;
            int bi = 0x7fffffff;
            if (pq >= 0) {
                float S, D;
                int m = gi;
                if (gi == 0) {
                    eval_SD<KH>(recon, 0, zE, zO, S, D);
                    best = S - D;
                    bi = p.center;
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
                if (p.out_coef) {
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
    if (threadIdx.x == 0)
        for (long long h = g; h < issued; ++h)
            if (!mbar_wait(&full[h % kSmoothStages], (unsigned)(h / kSmoothStages) & 1u, p.wait_cycles)) {
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

fcc_status_t smooth_geometry(const fcc_plan *plan, long long T, SmoothPlan &g)
{
    const fcc_plan_info_t &in = plan->info;
    if (in.prec != FCC_PREC_FP32) return fail(FCC_ERR_UNSUPPORTED, "the smoothed path is FP32");
    if (in.M % 2) return fail(FCC_ERR_UNSUPPORTED, "the smoothed path needs an even number of mics");
    if (plan->n_slots > 8) return fail(FCC_ERR_UNSUPPORTED, "the smoothed path needs at most 8 mics");
    if (in.Q < 32 || in.Q > 128) return fail(FCC_ERR_UNSUPPORTED, "the smoothed path needs 128 <= N <= 512");
    if (!plan->kh) return fail(FCC_ERR_UNSUPPORTED, "more than 8 bases of one parity");
    const long long target = 4LL * plan->num_sms;
    g.chunk = (int)std::max<long long>(64, (T + target - 1) / target);
    g.n_chunks = (int)((T + g.chunk - 1) / g.chunk);
    g.threads = 32 * plan->n_slots;
    const int frame_bytes = in.M * in.B * 8;
    const size_t stage = ((size_t)frame_bytes + 127) & ~(size_t)127;
    const size_t tabs = (128 + 8 * sizeof(Slot) + (size_t)((in.Q + 1) * 2 * plan->kh + (in.center + 1) * 4 * plan->kh) * 4 +
                         127) & ~(size_t)127;
    g.smem = tabs + kSmoothStages * stage;
    g.work_bytes = (size_t)g.n_chunks * in.P * in.B * sizeof(float2);
    return FCC_OK;
}

// grid = min(chunks, resident CTAs): the CTAs are persistent over chunks
template <int KH, int RS>
fcc_status_t launch_smooth_inst(const SmoothParams &prm, int num_sms, int threads, size_t smem, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(fcc_smooth_kernel<KH, RS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(fcc_smooth_kernel)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fcc_smooth_kernel<KH, RS>, threads, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm < 1) return fail(FCC_ERR_UNSUPPORTED, "the smoothed kernel does not fit an SM");
    const int grid = (int)std::min<long long>(prm.n_chunks, (long long)num_sms * per_sm);
    fcc_smooth_kernel<KH, RS><<<grid, threads, smem, st>>>(prm);
    e = cudaGetLastError();
    return e == cudaSuccess ? FCC_OK : cuda_fail(e, "fcc_smooth_kernel launch");
}

template <int KH>
fcc_status_t launch_smooth_kh(int rs, const SmoothParams &prm, int num_sms, int threads, size_t smem, cudaStream_t st)
{
    switch (rs) {
    case 1: return launch_smooth_inst<KH, 1>(prm, num_sms, threads, smem, st);
    case 2: return launch_smooth_inst<KH, 2>(prm, num_sms, threads, smem, st);
    case 4: return launch_smooth_inst<KH, 4>(prm, num_sms, threads, smem, st);
    default: return fail(FCC_ERR_UNSUPPORTED, "the smoothed path needs 128 <= N <= 512");
    }
}

}  // namespace
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
                               float *d_coeffs, void *stream)
{
    if (!plan) return fail(FCC_ERR_INVALID_ARG, "null plan");
    if (!(alpha > 0.0 && alpha <= 1.0)) return fail(FCC_ERR_INVALID_ARG, "alpha must be in (0, 1]");
    if (T < 0) return fail(FCC_ERR_INVALID_ARG, "T < 0");
    SmoothPlan g{};
    fcc_status_t st = smooth_geometry(plan, std::max<long long>(T, 1), g);
    if (st != FCC_OK) return st;
    if (T == 0) return FCC_OK;
    if (!d_spectra || !d_lag_idx || !d_peak || !d_work) return fail(FCC_ERR_INVALID_ARG, "null spectra/outputs/work");
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
    // basis in the smoothed kernel's layout: row f = (even weights, odd weights)
    if (!plan->d_smooth_basis) {
        const int kh = plan->kh, Q = in.Q;
        std::vector<float> bas((size_t)(Q + 1) * 2 * kh, 0.f);
        for (int f = 0; f <= Q; ++f) {
            for (int k = 0; k < in.K_even; ++k) bas[(size_t)f * 2 * kh + k] = (float)plan->Pe[(size_t)k * (Q + 1) + f];
            if (f < Q)
                for (int k = 0; k < in.K_odd; ++k) bas[(size_t)f * 2 * kh + kh + k] = (float)plan->Po[(size_t)k * Q + f];
        }
        float *d = nullptr;
        FCC_CUDA_TRY(cudaMalloc(&d, bas.size() * sizeof(float)));
        FCC_CUDA_TRY(cudaMemcpy(d, bas.data(), bas.size() * sizeof(float), cudaMemcpyHostToDevice));
        const_cast<fcc_plan *>(plan)->d_smooth_basis = d;
    }
    SmoothParams prm{};
    prm.spectra = static_cast<const float2 *>(d_spectra);
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
    prm.carry = work;
    prm.basis = plan->d_smooth_basis;
    prm.recon = plan->d_recon;
    prm.slots = plan->d_slots;
    prm.center = in.center;
    prm.I = in.I;
    prm.KE = in.K_even;
    prm.KO = in.K_odd;
    prm.delta = (float)in.delta;
    prm.out_idx = d_lag_idx;
    prm.out_peak = d_peak;
    prm.out_tau = d_tau_hat;
    prm.out_coef = d_coeffs;
    prm.err = plan->d_err;
    prm.wait_cycles = debug_hooks().wait_cycles;
    const int rs = in.Q / 32;
    switch (plan->kh) {
    case 2: return launch_smooth_kh<2>(rs, prm, plan->num_sms, g.threads, g.smem, s);
    case 4: return launch_smooth_kh<4>(rs, prm, plan->num_sms, g.threads, g.smem, s);
    case 6: return launch_smooth_kh<6>(rs, prm, plan->num_sms, g.threads, g.smem, s);
    case 8: return launch_smooth_kh<8>(rs, prm, plan->num_sms, g.threads, g.smem, s);
    default: return fail(FCC_ERR_UNSUPPORTED, "more than 8 bases of one parity");
    }
}

}  // extern "C"
