// fcc_fp32.cu -- the FP32 FCC hot path for sm_103a.
//
// One persistent kernel does, per frame tile:
//   1. stage   : a warp-specialised producer copies whole frame tiles of spectra
//                (contiguous [F][M][B] complex64) into a ring of shared-memory
//                stages with one cp.async.bulk per tile, completed on an mbarrier
//                (bounded waits everywhere; no multicast);
//   2. PHAT    : the consumer group normalises each bin of each microphone in
//                place, u = X / |X| (0 for |X| = 0).  Because
//                X_i X_j^* / |X_i X_j^*| = u_i u_j^*, this is the phase transform
//                of Sec. 2 (eq. 1 with alpha = 1) for every pair at M (not P)
//                reciprocal square roots per bin;
//   3. fold +
//      project: each lane owns a 2x2 block of the pair triangle (mics {i1,i2} x
//                {j1,j2}, 4 pairs sharing 4 microphone rows) and one chunk of the
//                frequency axis; per bin pair (f, N/2-f) it forms the four cross
//                spectra in registers, folds them into x_s / x_d (Eq. 8) and
//                accumulates the real and imaginary parts against the cropped
//                even and odd bases (Eqs. 7, 9).  No pair spectrum leaves
//                registers;
//   4. reduce  : the chunk lanes of a slot combine their partial projections
//                with a reduce-scatter over warp shuffles, so lane q ends up
//                holding the 2K coefficients of pair q of the block;
//   5. output  : y(tau) on the lag grid from the 2K coefficients (using the
//                grid's symmetry, one pass over tau >= 0 yields y(tau) and
//                y(-tau)), argmax with the lowest index winning ties, the peak,
//                and (optionally) the FP64 three-point quadratic refinement.
// HBM traffic is the spectra read once plus the per-pair results.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdlib>

#include "fcc_internal.h"

namespace fcc {
namespace {


// Registers are split per SM sub-partition (16K each, warps assigned round
// robin), so the register cap and the warp count must fit together:
// KH = 8 keeps up to 224 registers with at most 8 warps (7 compute + producer);
// smaller KH cap registers at 168 and allow 8 compute warps + producer.
__host__ __device__ constexpr int max_compute_warps(int kh) { return kh == 8 ? 7 : 8; }
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase; false if it did not complete in time.
__device__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    long long t0 = clock64();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > kWaitCycles) return false;
        __nanosleep(64);
    }
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// u = x / |x| with u = 0 for x = 0; scaled slow path for |x|^2 outside the
// normal FP32 range; flags NaN / Inf.
__device__ __forceinline__ float2 unit_phase(float2 x, bool &bad)
{
    float s = fmaf(x.x, x.x, x.y * x.y);
    if (s >= FLT_MIN && s <= FLT_MAX) {
        float r = rsqrtf(s);
        return make_float2(x.x * r, x.y * r);
    }
    if (!(fabsf(x.x) <= FLT_MAX) || !(fabsf(x.y) <= FLT_MAX)) {  // NaN or Inf
        bad = true;
        return make_float2(0.f, 0.f);
    }
    float m = fmaxf(fabsf(x.x), fabsf(x.y));
    if (m == 0.f) return make_float2(0.f, 0.f);
    float a = x.x / m, b = x.y / m;
    float r = rsqrtf(fmaf(a, a, b * b));
    return make_float2(a * r, b * r);
}

struct SmemLayout {
    size_t bar_off, slot_off, basis_off, stage_off, stage_bytes, total;
};

__host__ __device__ inline SmemLayout smem_layout(int S, int n_slots, int Q, int kh, int F,
                                                  int frame_bytes)
{
    SmemLayout L;
    size_t o = 0;
    L.bar_off = o;
    o += 3 * (size_t)S * 8;
    o = (o + 15) & ~(size_t)15;
    L.slot_off = o;
    o += (size_t)n_slots * sizeof(Slot);
    o = (o + 15) & ~(size_t)15;
    L.basis_off = o;
    o += (size_t)(Q + 1) * 2 * kh * sizeof(float);
    o = (o + 127) & ~(size_t)127;
    L.stage_off = o;
    L.stage_bytes = (((size_t)F * frame_bytes) + 127) & ~(size_t)127;
    o += (size_t)S * L.stage_bytes;
    L.total = o;
    return L;
}

// y at lag index center+m (sign -1) or center-m (sign +1) from the 2K
// coefficients: S(m) -/+ D(m) (see the recon table layout in pack_tables).
template <int KH>
__device__ __forceinline__ void eval_SD(const float *__restrict__ recon, int m, const float *z,
                                        float &S, float &D)
{
    const float *g = recon + (size_t)m * 4 * KH;
    float s = 0.f, d = 0.f;
#pragma unroll
    for (int k = 0; k < KH; ++k) {
        s = fmaf(__ldg(g + k), z[k], s);
        s = fmaf(__ldg(g + KH + k), z[2 * KH + k], s);
        d = fmaf(__ldg(g + 2 * KH + k), z[KH + k], d);
        d = fmaf(__ldg(g + 3 * KH + k), z[3 * KH + k], d);
    }
    S = s;
    D = d;
}

template <int KH>
__device__ __forceinline__ float y_at(const float *__restrict__ recon, int center, int i, const float *z)
{
    int m = i >= center ? i - center : center - i;
    float S, D;
    eval_SD<KH>(recon, m, z, S, D);
    return i >= center ? S - D : S + D;
}

template <int KH>
__global__ void __maxnreg__(KH == 8 ? 224 : 168) fcc_fp32_kernel(const Fp32Params p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const SmemLayout lay = smem_layout(p.S, p.n_slots, p.Q, KH, p.F, p.frame_floats * 4);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + lay.bar_off);
    uint64_t *empty = full + p.S;
    uint64_t *normd = empty + p.S;  // group-wide "stage normalised" barrier
    Slot *slots = reinterpret_cast<Slot *>(smem + lay.slot_off);
    float *basis = reinterpret_cast<float *>(smem + lay.basis_off);
    unsigned char *stages = smem + lay.stage_off;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_compute_warps = p.G * p.GW;
    const int n_local = (p.n_tiles > (int)blockIdx.x)
                            ? (p.n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x
                            : 0;

    // ---- prologue: barriers, slot table and bases into shared memory
    if (threadIdx.x == 0) {
        for (int s = 0; s < p.S; ++s) {
            mbar_init(&full[s], p.bulk ? 1u : 32u);
            mbar_init(&empty[s], (unsigned)p.GW);
            mbar_init(&normd[s], (unsigned)p.GW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int e = threadIdx.x; e < p.n_slots; e += blockDim.x) slots[e] = p.slots[e];
    {
        const int nb = (p.Q + 1) * 2 * KH;
        for (int e = threadIdx.x; e < nb; e += blockDim.x) basis[e] = p.basis[e];
    }
    fence_proxy_async();
    __syncthreads();

    if (warp == n_compute_warps) {
        // ================= producer warp =================
        const size_t frame_bytes = (size_t)p.frame_floats * 4;
        int issued = 0;
        bool ok = true;
        for (int k = 0; k < n_local && ok; ++k) {
            const int s = k % p.S;
            const unsigned par = ((unsigned)(k / p.S) & 1u) ^ 1u;
            if (!mbar_wait(&empty[s], par)) {
                ok = false;
                break;
            }
            const long long tile = (long long)blockIdx.x + (long long)k * gridDim.x;
            const long long f0 = tile * p.F;
            const int nf = (int)min((long long)p.F, p.T - f0);
            const char *src = reinterpret_cast<const char *>(p.spectra) + (size_t)f0 * frame_bytes;
            unsigned char *dst = stages + (size_t)s * lay.stage_bytes;
            const size_t bytes = (size_t)nf * frame_bytes;
            if (p.bulk) {
                if (lane == 0) {
                    mbar_arrive_expect_tx(&full[s], (unsigned)bytes);
                    bulk_g2s(dst, src, (unsigned)bytes, &full[s]);
                }
            } else {
                const size_t n8 = bytes / 8;
                const unsigned long long *s8 = reinterpret_cast<const unsigned long long *>(src);
                unsigned long long *d8 = reinterpret_cast<unsigned long long *>(dst);
                for (size_t e = lane; e < n8; e += 32) d8[e] = __ldg(s8 + e);
                mbar_arrive(&full[s]);
            }
            ++issued;
        }
        if (!ok && lane == 0) atomicOr(p.err, kErrTimeout);
        // never leave a bulk copy in flight when the CTA retires
        if (p.bulk && lane == 0) {
            for (int k = max(0, issued - p.S); k < issued; ++k)
                if (!mbar_wait(&full[k % p.S], (unsigned)(k / p.S) & 1u)) atomicOr(p.err, kErrTimeout);
        }
        return;
    }

    // ================= consumer groups =================
    const int group = warp / p.GW;
    const int lane_g = (warp % p.GW) * 32 + lane;
    const int gthreads = p.GW * 32;
    const int fl = lane_g / p.lanes_frame;
    const int rem = lane_g - fl * p.lanes_frame;
    const int slot_id = rem / p.C;
    const int chunk = rem - slot_id * p.C;
    const int QC = p.Q / p.C;
    const int B = p.B;
    const int half = 2 * p.Q;  // N/2
    const unsigned FULLM = 0xffffffffu;

    for (int k = group; k < n_local; k += p.G) {
        const int s = k % p.S;
        if (!mbar_wait(&full[s], (unsigned)(k / p.S) & 1u)) {
            if (lane == 0) atomicOr(p.err, kErrTimeout);
            break;
        }
        const long long tile = (long long)blockIdx.x + (long long)k * gridDim.x;
        const long long f0 = tile * p.F;
        const int nf = (int)min((long long)p.F, p.T - f0);
        float2 *st = reinterpret_cast<float2 *>(stages + (size_t)s * lay.stage_bytes);

        // ---- 2. PHAT normalisation in place
        {
            bool bad = false;
            const int ne = nf * p.M * B;
            for (int e = lane_g; e < ne; e += gthreads) st[e] = unit_phase(st[e], bad);
            if (__any_sync(FULLM, bad) && lane == 0) atomicOr(p.err, kErrNonFinite);
        }
        __syncwarp();
        if (p.GW > 1) {
            // every warp of the group must see the whole tile normalised
            if (lane == 0) mbar_arrive(&normd[s]);
            if (!mbar_wait(&normd[s], (unsigned)(k / p.S) & 1u)) {
                if (lane == 0) atomicOr(p.err, kErrTimeout);
                break;
            }
        }

        // ---- 3. fold + projection over this lane's frequency chunk
        const bool active = (fl < nf) && (slot_id < p.n_slots);
        float acc[4][4 * KH];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int v = 0; v < 4 * KH; ++v) acc[q][v] = 0.f;
        Slot sl;
        if (active) {
            sl = slots[slot_id];
            const float2 *U = st + (size_t)fl * p.M * B;
            const float2 *ui1 = U + sl.mic[0] * B;
            const float2 *ui2 = U + sl.mic[1] * B;
            const float2 *uj1 = U + sl.mic[2] * B;
            const float2 *uj2 = U + sl.mic[3] * B;
            const int fbase = chunk * QC;
            const int r0 = p.rot * chunk;
#pragma unroll 2
            for (int it = 0; it < QC; ++it) {
                const int f = fbase + ((it + r0) & (QC - 1));
                const int fm = half - f;
                const float2 xa[2] = {ui1[f], ui2[f]};
                const float2 ya[2] = {uj1[f], uj2[f]};
                const float2 xb[2] = {ui1[fm], ui2[fm]};
                const float2 yb[2] = {uj1[fm], uj2[fm]};
                // basis row of bin f: even bases in [0, KH), odd bases in [KH, 2KH)
                float row[2 * KH];
                const float4 *b4 = reinterpret_cast<const float4 *>(basis + (size_t)f * 2 * KH);
#pragma unroll
                for (int v = 0; v < KH / 2; ++v) {
                    const float4 w = b4[v];
                    row[4 * v] = w.x;
                    row[4 * v + 1] = w.y;
                    row[4 * v + 2] = w.z;
                    row[4 * v + 3] = w.w;
                }
                const float *be = row, *bo = row + KH;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 x1 = xa[q >> 1], y1 = ya[q & 1];
                    const float2 x2 = xb[q >> 1], y2 = yb[q & 1];
                    // a = x1 y1^*, b = x2 y2^*  (cross spectra at f and N/2 - f)
                    const float ar = fmaf(x1.x, y1.x, x1.y * y1.y);
                    const float ai = fmaf(x1.y, y1.x, -(x1.x * y1.y));
                    const float br = fmaf(x2.x, y2.x, x2.y * y2.y);
                    const float bi = fmaf(x2.y, y2.x, -(x2.x * y2.y));
                    const float sr = ar + br, si = ai + bi;  // x_s (Eq. 8)
                    const float dr = ar - br, di = ai - bi;  // x_d (Eq. 8)
#pragma unroll
                    for (int v = 0; v < KH; ++v) {
                        acc[q][v] = fmaf(be[v], sr, acc[q][v]);
                        acc[q][KH + v] = fmaf(be[v], si, acc[q][KH + v]);
                        acc[q][2 * KH + v] = fmaf(bo[v], dr, acc[q][2 * KH + v]);
                        acc[q][3 * KH + v] = fmaf(bo[v], di, acc[q][3 * KH + v]);
                    }
                }
            }
            if (chunk == 0) {
                // f = N/4: x_s = R_hat(N/4); x_d's entry meets only zeros of the odd bases
                const int f = p.Q;
                const float2 xa[2] = {ui1[f], ui2[f]};
                const float2 ya[2] = {uj1[f], uj2[f]};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 x1 = xa[q >> 1], y1 = ya[q & 1];
                    const float sr = fmaf(x1.x, y1.x, x1.y * y1.y);
                    const float si = fmaf(x1.y, y1.x, -(x1.x * y1.y));
#pragma unroll
                    for (int v = 0; v < KH; ++v) {
                        const float b = basis[(size_t)f * 2 * KH + v];
                        acc[q][v] = fmaf(b, sr, acc[q][v]);
                        acc[q][KH + v] = fmaf(b, si, acc[q][KH + v]);
                    }
                }
            }
        }
        // release the stage: order our generic-proxy writes before the next bulk copy
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);

        // ---- 4. reduce-scatter of the chunk partials: lane (chunk & 3) keeps pair (chunk & 3)
        float z[4 * KH];
        {
            const bool hi = (chunk & 2) != 0;
            float r1[2][4 * KH];
#pragma unroll
            for (int pp = 0; pp < 2; ++pp)
#pragma unroll
                for (int v = 0; v < 4 * KH; ++v) {
                    const float mine = hi ? acc[pp + 2][v] : acc[pp][v];
                    const float other = hi ? acc[pp][v] : acc[pp + 2][v];
                    r1[pp][v] = mine + __shfl_xor_sync(FULLM, other, 2);
                }
            const bool b0 = (chunk & 1) != 0;
#pragma unroll
            for (int v = 0; v < 4 * KH; ++v) {
                const float mine = b0 ? r1[1][v] : r1[0][v];
                const float other = b0 ? r1[0][v] : r1[1][v];
                z[v] = mine + __shfl_xor_sync(FULLM, other, 1);
            }
            for (int o = 4; o < p.C; o <<= 1) {
#pragma unroll
                for (int v = 0; v < 4 * KH; ++v) z[v] += __shfl_xor_sync(FULLM, z[v], o);
            }
        }

        // ---- 5. reconstruction on the grid, argmax, peak, refinement
        const int q = chunk & 3;
        const int pq = q == 0 ? sl.pair[0] : q == 1 ? sl.pair[1] : q == 2 ? sl.pair[2] : sl.pair[3];
        if (active && chunk < 4 && pq >= 0) {
            const long long t = f0 + fl;
            const size_t o = (size_t)t * p.P + pq;
            float *corr = p.out_corr ? p.out_corr + o * p.I : nullptr;
            float S, D;
            eval_SD<KH>(p.recon, 0, z, S, D);
            float best = S - D;
            int bi = p.center;
            if (corr) corr[p.center] = best;
            for (int m = 1; m <= p.center; ++m) {
                eval_SD<KH>(p.recon, m, z, S, D);
                const float ym = S + D, yp = S - D;  // y(center - m), y(center + m)
                if (ym >= best) {  // lower index than everything seen so far
                    best = ym;
                    bi = p.center - m;
                }
                if (yp > best) {  // higher index than everything seen so far
                    best = yp;
                    bi = p.center + m;
                }
                if (corr) {
                    corr[p.center - m] = ym;
                    corr[p.center + m] = yp;
                }
            }
            p.out_idx[o] = bi;
            p.out_peak[o] = best;
            if (p.out_tau) {
                double tau = (double)(bi - p.center) * (double)p.delta;
                if (bi > 0 && bi < p.I - 1) {
                    const double y_m = y_at<KH>(p.recon, p.center, bi - 1, z);
                    const double y_p = y_at<KH>(p.recon, p.center, bi + 1, z);
                    const double den = y_m - 2.0 * (double)best + y_p;
                    if (den < 0.0) {
                        double d = 0.5 * (y_m - y_p) / den;
                        d = fmin(0.5, fmax(-0.5, d));
                        tau += (double)p.delta * d;
                    }
                }
                p.out_tau[o] = (float)tau;
            }
            if (p.out_coef) {
                const int K = p.KE + p.KO;
                float *cf = p.out_coef + o * 2 * K;
#pragma unroll
                for (int v = 0; v < KH; ++v) {
                    if (v < p.KE) {
                        cf[v] = z[v];
                        cf[p.KE + v] = z[KH + v];
                    }
                    if (v < p.KO) {
                        cf[2 * p.KE + v] = z[2 * KH + v];
                        cf[2 * p.KE + p.KO + v] = z[3 * KH + v];
                    }
                }
            }
        }
    }
}

template <int KH>
fcc_status_t launch_kh(const fcc_plan *plan, const Fp32Params &prm, cudaStream_t st, int grid)
{
    static bool attr_set[64] = {};
    int dev = plan->device;
    if (!attr_set[dev & 63]) {
        cudaError_t e = cudaFuncSetAttribute(fcc_fp32_kernel<KH>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(fcc_fp32_kernel)");
        attr_set[dev & 63] = true;
    }
    const int threads = (prm.G * prm.GW + 1) * 32;
    fcc_fp32_kernel<KH><<<grid, threads, plan->geo.smem_bytes, st>>>(prm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fcc_fp32_kernel launch");
    return FCC_OK;
}

}  // namespace

// Choose chunks per slot (C), warps per group (GW), groups (G), frames per
// stage (F) and the ring depth (S) for this plan's M, N and K.  Tile k lives in
// stage k % S and is processed by group k % G; S is a multiple of G so that
// every stage is only ever filled for, and released by, one group -- each
// group then sees a plain single-consumer ring and the mbarrier phase parity
// it waits on can never be two phases stale.  The environment variables
// FCC_FP32_GROUPS and FCC_FP32_STAGES_PER_GROUP pin G and S/G (tuning only).
fcc_status_t choose_fp32_geometry(fcc_plan *plan)
{
    const fcc_plan_info_t &in = plan->info;
    const int kh = plan->kh;
    const int n_slots = plan->n_slots;
    const int frame_bytes = in.M * in.B * 8;
    int smem_max = 0;
    FCC_CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, plan->device));
    smem_max = std::min(smem_max, 232448);
    const char *eg = getenv("FCC_FP32_GROUPS");
    const char *es = getenv("FCC_FP32_STAGES_PER_GROUP");
    const int want_g = eg ? atoi(eg) : 0, want_sg = es ? atoi(es) : 0;
    Fp32Geometry best{};
    double best_score = -1.0;
    for (int C = 4; C <= 16 && C <= in.Q; C <<= 1) {
        const int lanes = n_slots * C;
        for (int GW = 1; GW <= max_compute_warps(kh); GW <<= 1) {
            if (lanes > GW * 32) continue;
            const int F = (GW * 32) / lanes;
            for (int G = max_compute_warps(kh) / GW; G >= 1; --G) {
                if (want_g && G != want_g) continue;
                for (int Sg = 3; Sg >= 1; --Sg) {
                    if (want_sg && Sg != want_sg) continue;
                    const int S = G * Sg;
                    const SmemLayout L = smem_layout(S, n_slots, in.Q, kh, F, frame_bytes);
                    if (L.total > (size_t)smem_max) continue;
                    // lane utilisation x warps in flight; a group with a second
                    // stage can prefetch while it computes; fewer chunks reduce
                    // the shuffle reduction
                    const double util = (double)(F * lanes) / (GW * 32);
                    const double score = util * (G * GW) * (Sg >= 2 ? 1.0 : 0.8) * (1.0 - 0.02 * (C / 4 - 1));
                    if (score > best_score) {
                        best_score = score;
                        best = Fp32Geometry{C, lanes, GW, G, F, S, 5, L.total};
                    }
                    break;  // the deepest ring that fits for this G
                }
            }
        }
    }
    if (best_score < 0) return fail(FCC_ERR_UNSUPPORTED, "frame too large for the shared-memory ring");
    plan->geo = best;
    return FCC_OK;
}

fcc_status_t launch_fp32(const fcc_plan *plan, const float2 *spectra, long long T, int *idx,
                         float *peak, float *tau, float *coef, float *corr, cudaStream_t st)
{
    const fcc_plan_info_t &in = plan->info;
    const Fp32Geometry &g = plan->geo;
    Fp32Params prm{};
    prm.spectra = spectra;
    prm.T = T;
    prm.M = in.M;
    prm.B = in.B;
    prm.Q = in.Q;
    prm.N = in.N;
    prm.P = in.P;
    prm.n_slots = plan->n_slots;
    prm.C = g.C;
    prm.lanes_frame = g.lanes_frame;
    prm.GW = g.GW;
    prm.G = g.G;
    prm.F = g.F;
    prm.S = g.S;
    prm.rot = g.rot;
    const long long n_tiles = (T + g.F - 1) / g.F;
    if (n_tiles > 0x7fffffffLL) return fail(FCC_ERR_UNSUPPORTED, "too many frames for one call");
    prm.n_tiles = (int)n_tiles;
    prm.frame_floats = in.M * in.B * 2;
    const size_t frame_bytes = (size_t)in.M * in.B * 8;
    prm.bulk = (frame_bytes % 16 == 0) && ((reinterpret_cast<uintptr_t>(spectra) & 15) == 0);
    prm.center = in.center;
    prm.I = in.I;
    prm.KE = in.K_even;
    prm.KO = in.K_odd;
    prm.tau0 = (float)(-in.L);
    prm.delta = (float)in.delta;
    prm.basis = plan->d_basis;
    prm.recon = plan->d_recon;
    prm.slots = plan->d_slots;
    prm.out_idx = idx;
    prm.out_peak = peak;
    prm.out_tau = tau;
    prm.out_coef = coef;
    prm.out_corr = corr;
    prm.err = plan->d_err;
    const int grid = (int)std::min<long long>(n_tiles, (long long)plan->num_sms);
    switch (plan->kh) {
    case 2: return launch_kh<2>(plan, prm, st, grid);
    case 4: return launch_kh<4>(plan, prm, st, grid);
    case 6: return launch_kh<6>(plan, prm, st, grid);
    case 8: return launch_kh<8>(plan, prm, st, grid);
    default: return fail(FCC_ERR_UNSUPPORTED, "more than 8 bases of one parity");
    }
}

}  // namespace fcc
