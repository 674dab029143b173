// fcc_fp32_tiles.cuh -- the per-tile pipeline of the FP32 FCC kernels (stage,
// per-microphone PHAT and folded re-lay, cross spectra + projection,
// reduce-scatter, reconstruction + argmax + refinement), shared by the folded
// kernels (fcc_fp32.cu) and the split-form kernel (fcc_fp32_reim.cu).
#pragma once

#include <cfloat>

#include "fcc_device.cuh"
#include "fcc_internal.h"

namespace fcc {
namespace {

constexpr int kMaxRowSlots = 8;                  // fold records per lane per row (RS): N <= 1024

// Registers are split per SM sub-partition (16K each), so the warp count and
// the register cap must fit together: KH >= 6 keeps up to 255 registers with 8
// warps; smaller KH caps registers at 168 with 12 warps.
__host__ __device__ constexpr int max_compute_warps(int kh) { return kh >= 6 ? 8 : 12; }


struct SmemLayout {
    size_t bar_off, slot_off, basis_off, recon_off, stage_off, stage_bytes, total;
};

__host__ __device__ inline SmemLayout smem_layout(int S, int n_slots, int Q, int kh, int C, int BS, int center,
                                                  int F, int frame_bytes)
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
    o += (size_t)(Q + C + 1) * BS * sizeof(float);
    o = (o + 15) & ~(size_t)15;
    L.recon_off = o;
    o += (size_t)(center + 1) * 4 * kh * sizeof(float);
    o = (o + 127) & ~(size_t)127;
    L.stage_off = o;
    L.stage_bytes = (((size_t)F * frame_bytes) + 127) & ~(size_t)127;
    o += (size_t)S * L.stage_bytes;
    L.total = o;
    return L;
}


// Byte offsets, inside a tile, of row R's fold records and of its lone bin N/4.
__device__ __forceinline__ int rec_off(int R, int B) { return R * B * 8 + ((R & 1) ? 8 : 0); }
__device__ __forceinline__ int lone_off(int R, int B, int Q) { return R * B * 8 + ((R & 1) ? 0 : 16 * Q); }


// The whole per-tile pipeline for one plan: this CTA processes tiles
// tile_base + k * tile_stride, k = 0 .. n_local - 1, with the geometry and tables
// of `p` laid out from `smem`.  Warps beyond the plan's G * GW only help load the
// tables.  Every barrier this call initialises is idle again when it returns
// (all copies it issued have landed).
// RS = fold records per lane per row = max(1, N / 128) (N/4 records over 32 lanes).
// FB = the split form (cosine bases on Re x, sine bases on Im x, Eq. 3 without
// the Eq. 8 fold): the same records feed 2 KH coefficient pairs (c_v, s_v),
// accE holding v < KH and accO holding KH + v, and the reconstruction table
// holds (2 U_c, 2 U_s) so that the same S -/+ D evaluation gives
// y(+/-tau) = 2 (U_c c -/+ U_s s).
// Lag grid on the tensor cores (LG = single-plan launches; folded form, KH >= 6,
// p.npad > 0, one pair per lane (C = 4) and groups of at most four warps).  Per
// group the lanes write their coefficients into tensor memory as A rows (row =
// 32 (warp % 4) + lane), each row scaled by a power of two that puts its largest
// |z| in [2^14, 2^15) and split into three FP16 terms z1 + z2 + z3 (z minus the
// three is below 2^-33 |z|max); one elected lane issues S = A_re W_S and D =
// A_im W_D as six kind::f16 passes each (z1 w1, z2 w1, z1 w2, z1 w3, z2 w2,
// z3 w1) against the same three-term split of the weights, resident in shared
// memory (lag steps m = 1 .. npad, scaled by 2^rshift so that every |w| <
// 2^15), with FP32 accumulators.  What the six leave out is below 2^-30 of
// sum_k |z_k w_k|, plus at most 2^-25 per FP16 subnormal term (below 2^-38 of
// the largest |z| or |w|).
// The products are thus those of FP32 operands and better; the sums are FP32
// sums, as in eval_SD.  The lanes read S and D back for the argmax (the same
// outward scan and tie rule as the CUDA-core path), then evaluate y at the
// chosen lag and its two neighbours with eval_SD, so that the peak and the
// refinement are those of the CUDA-core path at that lag.  Rows whose
// coefficients are zero, tiny or not finite take the CUDA-core scan.
constexpr int kMmaHeader = 128;  // per group two barriers, then the tensor-memory slot
constexpr int kMmaParts = 3;     // FP16 terms per coefficient and per weight

template <int KH, int RS, bool FB, bool LG = false>
__device__ __forceinline__ void fp32_tiles(const Fp32Params &p, unsigned char *smem, long long tile_base,
                                           long long tile_stride, int n_local)
{
    const int frame_bytes = p.frame_floats * 4;
    const SmemLayout lay = smem_layout(p.S, p.n_slots, p.Q, KH, p.C, p.BS, p.center, p.F, frame_bytes);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + lay.bar_off);
    uint64_t *normd = full + p.S;   // group: every row of the tile re-laid
    uint64_t *freed = normd + p.S;  // group: every warp left the tile's rows
    Slot *slots = reinterpret_cast<Slot *>(smem + lay.slot_off);
    float *basis = reinterpret_cast<float *>(smem + lay.basis_off);
    float *recon = reinterpret_cast<float *>(smem + lay.recon_off);
    unsigned char *stages = smem + lay.stage_off;
    constexpr bool kMmaRecon = LG && !FB && KH >= 6;
    const bool mma = kMmaRecon && p.npad > 0;
    uint64_t *afull = reinterpret_cast<uint64_t *>(smem + lay.total);  // group: every A row written
    uint64_t *dfull = afull + p.G;                                       // group: S and D complete
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + lay.total + 16 * p.G);
    unsigned char *rtab = smem + lay.total + kMmaHeader;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int group = warp / p.GW, wig = warp - group * p.GW;
    const bool member = group < p.G;  // this warp belongs to one of the plan's groups
    const bool leader = member && wig == 0 && lane == 0;

    // ---- prologue: barriers, tables into shared memory
    if (threadIdx.x == 0) {
        for (int s = 0; s < p.S; ++s) {
            mbar_init(&full[s], p.bulk ? 1u : (unsigned)(p.GW * 32));
            mbar_init(&normd[s], (unsigned)p.GW);
            mbar_init(&freed[s], (unsigned)p.GW);
        }
        if (mma)
            for (int g = 0; g < p.G; ++g) {
                mbar_init(&afull[g], (unsigned)p.GW);
                mbar_init(&dfull[g], 1u);
            }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int e = threadIdx.x; e < p.n_slots; e += blockDim.x) slots[e] = p.slots[e];
    for (int e = threadIdx.x; e < (p.Q + p.C + 1) * p.BS; e += blockDim.x) basis[e] = p.basis[e];
    for (int e = threadIdx.x; e < (p.center + 1) * 4 * KH; e += blockDim.x) recon[e] = p.recon[e];
    uint32_t tmem = 0;
    if (mma) {
        const uint4 *src = reinterpret_cast<const uint4 *>(p.rbases);
        uint4 *dst = reinterpret_cast<uint4 *>(rtab);
        for (int e = threadIdx.x; e < p.npad * 4 * kMmaParts; e += blockDim.x) dst[e] = src[e];  // 2 x 3 x npad x 32 B
        __syncwarp();
        if (warp == 0) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                         "r"(512u));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    fence_proxy_async();
    __syncthreads();
    if (mma) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tmem = *tmem_slot;
    }
    unsigned rpar = 0;  // phase parity of this group's afull / dfull (one phase per tile)
    int r_issued = 0;   // reconstruction commits issued by this group's leader

    auto tile_src = [&](int k, int &nf) {
        const long long tile = tile_base + (long long)k * tile_stride;
        const long long f0 = tile * p.F;
        nf = (int)min((long long)p.F, p.T - f0);
        return f0;
    };
    // Issue the bulk copy of this CTA's tile k into its stage (group leader only);
    // `inflight` marks the stages whose copy the leader has not yet seen land.
    unsigned inflight = 0;
    auto issue = [&](int k) {
        int nf;
        const long long f0 = tile_src(k, nf);
        const int s = k % p.S;
        const unsigned bytes = (unsigned)nf * (unsigned)frame_bytes;
        mbar_arrive_expect_tx(&full[s], bytes);
        inflight |= 1u << s;
        bulk_g2s(stages + (size_t)s * lay.stage_bytes,
                 reinterpret_cast<const unsigned char *>(p.spectra) + (size_t)f0 * frame_bytes, bytes, &full[s]);
    };

    // prime this group's stages (the test hook withholds the copy of the plan's
    // first tile, so that group's first wait runs out and the timeout path is
    // taken)
    const int Sg = p.S / p.G;
    if (p.bulk && leader)
        for (int j = 0; j < Sg; ++j)
            if (group + j * p.G < n_local && !(p.inject && tile_base == 0 && group == 0 && j == 0))
                issue(group + j * p.G);

    // lane -> (frame in tile, slot, chunk).  A frame takes n_blocks whole warps;
    // inside a warp the lanes are chunk-major (lane = chunk * SB + slot), so the
    // 32 / SB lanes of a quarter-warp share one chunk and read one basis row.
    const int lane_g = wig * 32 + lane;
    const int fl = lane_g / p.lanes_frame;
    const int rem = lane_g - fl * p.lanes_frame;
    const int chunk = (rem & 31) / p.SB;
    const int slot_id = (rem >> 5) * p.SB + (rem & 31) % p.SB;
    const int QC = p.Q / p.C;
    const int B = p.B, Q = p.Q, M = p.M;
    const unsigned FULLM = 0xffffffffu;
    int k_done = group - p.G;  // last tile fully consumed by this group

    for (int k = group; member && k < n_local; k += p.G) {
        const int s = k % p.S;
        const unsigned par = (unsigned)(k / p.S) & 1u;
        int nf;
        const long long f0 = tile_src(k, nf);
        unsigned char *st = stages + (size_t)s * lay.stage_bytes;
        if (!p.bulk) {
            // plain-load staging (frame size not a multiple of 16 bytes)
            const size_t n8 = (size_t)nf * frame_bytes / 8;
            const unsigned long long *src = reinterpret_cast<const unsigned long long *>(
                reinterpret_cast<const unsigned char *>(p.spectra) + (size_t)f0 * frame_bytes);
            unsigned long long *dst = reinterpret_cast<unsigned long long *>(st);
            for (size_t e = lane_g; e < n8; e += p.GW * 32) dst[e] = __ldg(src + e);
            mbar_arrive(&full[s]);
        }
        if (!mbar_wait(&full[s], par, p.wait_cycles)) {
            if (lane == 0) atomicOr(p.err, kErrTimeout);
            break;
        }
        if (leader) inflight &= ~(1u << s);

        // ---- 2. PHAT + folded re-lay, one row per warp at a time
        {
            bool bad = false;
            const int rows = nf * M;
            for (int R = wig; R < rows; R += p.GW) {
                const float2 *raw = reinterpret_cast<const float2 *>(st + (size_t)R * B * 8);
                float2 a[RS], b[RS], lone = make_float2(0.f, 0.f);
                bool ok = true;
#pragma unroll
                for (int j = 0; j < RS; ++j) {
                    const int fp = lane + 32 * j;
                    if (RS > 1 || fp < Q) {
                        bool o1, o2;
                        a[j] = unit_phase_fast(raw[fp], o1);
                        b[j] = unit_phase_fast(raw[2 * Q - fp], o2);
                        ok = ok && o1 && o2;
                    }
                }
                if (lane == 0) {
                    bool o;
                    lone = unit_phase_fast(raw[Q], o);
                    ok = ok && o;
                }
                if (!__all_sync(FULLM, ok)) {  // rare: zero, tiny, huge or non-finite bins
#pragma unroll
                    for (int j = 0; j < RS; ++j) {
                        const int fp = lane + 32 * j;
                        if (RS > 1 || fp < Q) {
                            a[j] = unit_phase_slow(raw[fp], bad);
                            b[j] = unit_phase_slow(raw[2 * Q - fp], bad);
                        }
                    }
                    if (lane == 0) lone = unit_phase_slow(raw[Q], bad);
                }
                __syncwarp();  // the whole row is read before any of it is rewritten
                float4 *recs = reinterpret_cast<float4 *>(st + rec_off(R, B));
                const int sw = rec_swz(R, Q);
#pragma unroll
                for (int j = 0; j < RS; ++j) {
                    const int fp = lane + 32 * j;
                    if (RS > 1 || fp < Q) recs[fp ^ sw] = make_float4(a[j].x, a[j].y, b[j].x, b[j].y);
                }
                if (lane == 0) *reinterpret_cast<float2 *>(st + lone_off(R, B, Q)) = lone;
                __syncwarp();
            }
            if (__any_sync(FULLM, bad) && lane == 0) atomicOr(p.err, kErrNonFinite);
        }
        if (p.GW > 1) {
            if (lane == 0) mbar_arrive(&normd[s]);
            if (!mbar_wait(&normd[s], par, p.wait_cycles)) {
                if (lane == 0) atomicOr(p.err, kErrTimeout);
                break;
            }
        }

        // ---- 3. fold + projection over this lane's chunk of bin pairs
        const bool active = (fl < nf) && (slot_id < p.n_slots);
        f2 accE[4][KH], accO[4][KH];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int v = 0; v < KH; ++v) accE[q][v] = accO[q][v] = 0ull;
        Slot sl{};
        if (active) {
            sl = slots[slot_id];
            const int R0 = fl * M;
            const float4 *bas = reinterpret_cast<const float4 *>(basis);
            // basis row stride in float4 (odd): folded KH even + KH odd weights;
            // split form 2 KH coefficient rows of (C(f), S(f), C(N/2-f), S(N/2-f))
            constexpr int BS4 = FB ? 2 * KH + 1 : (((KH / 2) % 2 == 0) ? KH / 2 + 1 : KH / 2);
            const float4 *bchunk = bas + (size_t)chunk * (QC + 1) * BS4;  // one pad row per chunk
            auto body = [&](const float4 (&X)[2], const float4 (&Y)[2], const float4 *brow) {
                // packed operands: x as (re, im) and swapped (im, re) per X microphone
                // and bin, y as (re, re) and (im, -im) per Y microphone and bin, so
                // that x y^* = (xr yr + xi yi, xi yr - xr yi) is one FMUL2 + one FFMA2
                f2 xa[2][2], xw[2][2], yr[2][2], yi[2][2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    xa[u][0] = pk(X[u].x, X[u].y);
                    xw[u][0] = pk(X[u].y, X[u].x);
                    xa[u][1] = pk(X[u].z, X[u].w);
                    xw[u][1] = pk(X[u].w, X[u].z);
                    yr[u][0] = pk(Y[u].x, Y[u].x);
                    yi[u][0] = pk(Y[u].y, -Y[u].y);
                    yr[u][1] = pk(Y[u].z, Y[u].z);
                    yi[u][1] = pk(Y[u].w, -Y[u].w);
                }
                if constexpr (FB) {
                    // cross spectra of the four pairs at f and N/2 - f, then per
                    // coefficient v: (c_v, s_v) += (C_v, S_v) (Re, Im) at both bins
                    f2 a[4], b[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int ix = q >> 1, iy = q & 1;
                        a[q] = fma2(xw[ix][0], yi[iy][0], mul2(xa[ix][0], yr[iy][0]));
                        b[q] = fma2(xw[ix][1], yi[iy][1], mul2(xa[ix][1], yr[iy][1]));
                    }
#pragma unroll
                    for (int v = 0; v < KH; ++v) {
                        const float4 e = brow[v], o = brow[KH + v];
                        const f2 ef = pk(e.x, e.y), eg = pk(e.z, e.w), of = pk(o.x, o.y), og = pk(o.z, o.w);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            accE[q][v] = fma2(eg, b[q], fma2(ef, a[q], accE[q][v]));
                            accO[q][v] = fma2(og, b[q], fma2(of, a[q], accO[q][v]));
                        }
                    }
                } else {
                    f2 bE[KH], bO[KH];
                    float w[2 * KH];
#pragma unroll
                    for (int v = 0; v < KH / 2; ++v) {
                        const float4 e = brow[v];
                        w[4 * v] = e.x;
                        w[4 * v + 1] = e.y;
                        w[4 * v + 2] = e.z;
                        w[4 * v + 3] = e.w;
                    }
#pragma unroll
                    for (int v = 0; v < KH; ++v) {
                        bE[v] = pk(w[v], w[v]);
                        bO[v] = pk(w[KH + v], w[KH + v]);
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int ix = q >> 1, iy = q & 1;
                        // cross spectra at f and N/2 - f: a = x(f) y(f)^*, b = x(N/2-f) y(N/2-f)^*
                        const f2 a = fma2(xw[ix][0], yi[iy][0], mul2(xa[ix][0], yr[iy][0]));
                        const f2 b = fma2(xw[ix][1], yi[iy][1], mul2(xa[ix][1], yr[iy][1]));
                        const f2 xs = add2(a, b), xd = sub2(a, b);  // Eq. 8
#pragma unroll
                        for (int v = 0; v < KH; ++v) {
                            accE[q][v] = fma2(bE[v], xs, accE[q][v]);
                            accO[q][v] = fma2(bO[v], xd, accO[q][v]);
                        }
                    }
                }
            };
            const int cb = chunk * QC;
            const int st_off = (int)(st - smem);
            // Each lane takes its slot's microphones in the order of its role in
            // the reduce-scatter: chunk bit 1 swaps the two X microphones, chunk
            // bit 0 the two Y microphones, so accumulator q always holds the pair
            // this lane keeps (q = 0) or hands on, with no selects.
            const int sx = (chunk >> 1) & 1, sy = chunk & 1;
            const int mr[4] = {sx ? sl.mic[1] : sl.mic[0], sx ? sl.mic[0] : sl.mic[1],
                               sy ? sl.mic[3] : sl.mic[2], sy ? sl.mic[2] : sl.mic[3]};
            int sw[4], rb[4];  // byte offsets from the shared-memory base
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                sw[r] = rec_swz(R0 + mr[r], Q);
                rb[r] = st_off + rec_off(R0 + mr[r], B) + 16 * cb;
            }
            if ((QC & 7) == 0) {
                // 8 records at a time: record cb+t8+j of a swizzled row is at
                // cb+t8+(j^4), i.e. +4 records for j < 4 and -4 for j >= 4
                int lo[4], hi[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    lo[r] = rb[r] + 16 * sw[r];
                    hi[r] = rb[r] - 16 * sw[r];
                }
                // two 8-record blocks per iteration pay for KH = 8 (16-mic grid: 8 %
                // faster) and cost the 4-basis kernels (8-mic circle: 11 % slower)
                constexpr int kBlockUnroll = KH >= 8 ? 2 : 1;
#pragma unroll kBlockUnroll
                for (int t8 = 0; t8 < QC; t8 += 8) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int o = 16 * (t8 + j);
                        float4 X[2], Y[2];
                        X[0] = *reinterpret_cast<const float4 *>(smem + (j < 4 ? lo[0] : hi[0]) + o);
                        X[1] = *reinterpret_cast<const float4 *>(smem + (j < 4 ? lo[1] : hi[1]) + o);
                        Y[0] = *reinterpret_cast<const float4 *>(smem + (j < 4 ? lo[2] : hi[2]) + o);
                        Y[1] = *reinterpret_cast<const float4 *>(smem + (j < 4 ? lo[3] : hi[3]) + o);
                        body(X, Y, bchunk + (size_t)(t8 + j) * BS4);
                    }
                }
            } else {
#pragma unroll 1
                for (int t = 0; t < QC; ++t) {
                    float4 X[2], Y[2];
                    X[0] = *reinterpret_cast<const float4 *>(smem + rb[0] + 16 * (((cb + t) ^ sw[0]) - cb));
                    X[1] = *reinterpret_cast<const float4 *>(smem + rb[1] + 16 * (((cb + t) ^ sw[1]) - cb));
                    Y[0] = *reinterpret_cast<const float4 *>(smem + rb[2] + 16 * (((cb + t) ^ sw[2]) - cb));
                    Y[1] = *reinterpret_cast<const float4 *>(smem + rb[3] + 16 * (((cb + t) ^ sw[3]) - cb));
                    body(X, Y, bchunk + (size_t)t * BS4);
                }
            }
            if (chunk == 0) {
                // bin N/4: x_s = R_hat(N/4); the odd bases vanish there (Eq. 8)
                float2 X[2], Y[2];
                X[0] = *reinterpret_cast<const float2 *>(st + lone_off(R0 + sl.mic[0], B, Q));
                X[1] = *reinterpret_cast<const float2 *>(st + lone_off(R0 + sl.mic[1], B, Q));
                Y[0] = *reinterpret_cast<const float2 *>(st + lone_off(R0 + sl.mic[2], B, Q));
                Y[1] = *reinterpret_cast<const float2 *>(st + lone_off(R0 + sl.mic[3], B, Q));
                const float4 *brow = bas + (size_t)p.C * (QC + 1) * BS4;
                if constexpr (FB) {
                    // split form: row v holds (C_v(N/4), S_v(N/4), 0, 0)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float2 x = X[q >> 1], y = Y[q & 1];
                        const f2 xs = pk(fmaf(x.x, y.x, x.y * y.y), fmaf(x.y, y.x, -(x.x * y.y)));
#pragma unroll
                        for (int v = 0; v < KH; ++v) {
                            const float4 e = brow[v], o = brow[KH + v];
                            accE[q][v] = fma2(pk(e.x, e.y), xs, accE[q][v]);
                            accO[q][v] = fma2(pk(o.x, o.y), xs, accO[q][v]);
                        }
                    }
                } else {
                    f2 bE[KH];
#pragma unroll
                    for (int v = 0; v < KH / 4 + (KH % 4 ? 1 : 0); ++v) {
                        const float4 e = brow[v];
                        if (4 * v < KH) bE[4 * v] = pk(e.x, e.x);
                        if (4 * v + 1 < KH) bE[4 * v + 1] = pk(e.y, e.y);
                        if (4 * v + 2 < KH) bE[4 * v + 2] = pk(e.z, e.z);
                        if (4 * v + 3 < KH) bE[4 * v + 3] = pk(e.w, e.w);
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float2 x = X[q >> 1], y = Y[q & 1];
                        const f2 xs = pk(fmaf(x.x, y.x, x.y * y.y), fmaf(x.y, y.x, -(x.x * y.y)));
#pragma unroll
                        for (int v = 0; v < KH; ++v) accE[q][v] = fma2(bE[v], xs, accE[q][v]);
                    }
                }
            }
        }
        // ---- release the stage and refill it with this group's tile k + S
        fence_proxy_async();  // our generic writes precede the next bulk write
        __syncwarp();
        if (p.bulk) {
            if (p.GW > 1) {
                if (lane == 0) mbar_arrive(&freed[s]);
                if (leader && k + p.S < n_local) {
                    if (!mbar_wait(&freed[s], par, p.wait_cycles)) {
                        atomicOr(p.err, kErrTimeout);
                    } else {
                        issue(k + p.S);
                    }
                }
            } else if (lane == 0 && k + p.S < n_local) {
                issue(k + p.S);
            }
        } else if (p.GW > 1) {
            // plain staging: the group's next copy must not start before every
            // warp has left this stage
            if (lane == 0) mbar_arrive(&freed[s]);
            if (!mbar_wait(&freed[s], par, p.wait_cycles)) {
                if (lane == 0) atomicOr(p.err, kErrTimeout);
                break;
            }
        }
        k_done = k;

        // ---- 4. reduce-scatter of the chunk partials: lane (chunk & 3) keeps pair (chunk & 3)
        f2 zE[KH], zO[KH];
        {
            // level 1 (lanes 2 SB apart): keep accumulators 0, 1, hand on 2, 3
            f2 rE[2][KH], rO[2][KH];
#pragma unroll
            for (int pp = 0; pp < 2; ++pp)
#pragma unroll
                for (int v = 0; v < KH; ++v) {
                    float m0, m1, o0, o1;
                    upk(accE[pp][v], m0, m1);
                    upk(accE[pp + 2][v], o0, o1);
                    rE[pp][v] = pk(m0 + __shfl_xor_sync(FULLM, o0, 2 * p.SB), m1 + __shfl_xor_sync(FULLM, o1, 2 * p.SB));
                    upk(accO[pp][v], m0, m1);
                    upk(accO[pp + 2][v], o0, o1);
                    rO[pp][v] = pk(m0 + __shfl_xor_sync(FULLM, o0, 2 * p.SB), m1 + __shfl_xor_sync(FULLM, o1, 2 * p.SB));
                }
            // level 2 (lanes SB apart): keep 0, hand on 1; then plain sums over the other chunks
#pragma unroll
            for (int v = 0; v < KH; ++v) {
                float m0, m1, o0, o1;
                upk(rE[0][v], m0, m1);
                upk(rE[1][v], o0, o1);
                float e0 = m0 + __shfl_xor_sync(FULLM, o0, p.SB), e1 = m1 + __shfl_xor_sync(FULLM, o1, p.SB);
                upk(rO[0][v], m0, m1);
                upk(rO[1][v], o0, o1);
                float d0 = m0 + __shfl_xor_sync(FULLM, o0, p.SB), d1 = m1 + __shfl_xor_sync(FULLM, o1, p.SB);
                for (int o = 4 * p.SB; o < 32; o <<= 1) {
                    e0 += __shfl_xor_sync(FULLM, e0, o);
                    e1 += __shfl_xor_sync(FULLM, e1, o);
                    d0 += __shfl_xor_sync(FULLM, d0, o);
                    d1 += __shfl_xor_sync(FULLM, d1, o);
                }
                zE[v] = pk(e0, e1);
                zO[v] = pk(d0, d1);
            }
        }

        // ---- 5. reconstruction on the grid, argmax, peak, refinement
        const int q = chunk & 3;
        const int pq = q == 0 ? sl.pair[0] : q == 1 ? sl.pair[1] : q == 2 ? sl.pair[2] : sl.pair[3];
        // The pair's y(tau) values at bi - 1 and bi + 1 (FP64 differences) give the
        // three-point parabola; the coefficients go out when asked for.
        auto emit = [&](size_t o, int bi, float best) {
            p.out_idx[o] = bi;
            p.out_peak[o] = best;
            if (p.out_tau) {
                float off = 0.f;
                if (bi > 0 && bi < p.I - 1) {
                    // three-point parabola; the differences, where the
                    // cancellation happens, are exact in FP64
                    const double y_m = y_at<KH>(recon, p.center, bi - 1, zE, zO);
                    const double y_p = y_at<KH>(recon, p.center, bi + 1, zE, zO);
                    const double num = y_m - y_p;
                    const double den = (y_m - 2.0 * (double)best) + y_p;
                    if (den < 0.0) off = fminf(0.5f, fmaxf(-0.5f, 0.5f * (float)num / (float)den));
                }
                p.out_tau[o] = ((float)(bi - p.center) + off) * p.delta;
            }
            if (!FB && p.out_coef) {  // the split form has no coefficient output
                const int K = p.KE + p.KO;
                float *cf = p.out_coef + o * 2 * K;
#pragma unroll
                for (int v = 0; v < KH; ++v) {
                    float a, b;
                    if (v < p.KE) {
                        upk(zE[v], a, b);
                        cf[v] = a;
                        cf[p.KE + v] = b;
                    }
                    if (v < p.KO) {
                        upk(zO[v], a, b);
                        cf[2 * p.KE + v] = a;
                        cf[2 * p.KE + p.KO + v] = b;
                    }
                }
            }
        };
        // One outward scan over lag steps m = m0, m0 + stride, ...: y(center - m)
        // is below every index this lane has seen (wins ties), y(center + m)
        // above every one (loses ties).
        auto scan = [&](int m0, int stride, float &best, int &bi, float *corr) {
            float S, D;
            for (int m = m0; m <= p.center; m += stride) {
                eval_SD<KH>(recon, m, zE, zO, S, D);
                const float ym = S + D, yp = S - D;  // y(center - m), y(center + m)
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
        };
        if (mma) {
            // ---- 5'. the lag grid on the tensor cores (C = 4: one pair per lane)
            __syncwarp();  // tcgen05.st / ld are warp-wide
            const bool mine = active && pq >= 0;
            const uint32_t lrow = (uint32_t)((warp & 3) * 32) << 16;  // this lane's tensor-memory row
            const uint32_t gcol = tmem + (uint32_t)(group * (64 + 2 * p.npad));
            float mx = 0.f, zs = 0.f;
#pragma unroll
            for (int v = 0; v < KH; ++v) {
                float a0, a1, b0, b1;
                upk(zE[v], a0, a1);
                upk(zO[v], b0, b1);
                mx = fmaxf(mx, fmaxf(fmaxf(fabsf(a0), fabsf(a1)), fmaxf(fabsf(b0), fabsf(b1))));
                zs += (fabsf(a0) + fabsf(a1)) + (fabsf(b0) + fabsf(b1));
            }
            // a NaN fails the first test, an infinity or a tiny or zero row the others
            const bool fine = mine && zs < 0x1p100f && mx >= 0x1p-90f;
            const unsigned eb = (__float_as_uint(mx) >> 23) & 0xffu;        // mx in [2^(eb-127), 2^(eb-126))
            const float zsc = fine ? __uint_as_float((268u - eb) << 23) : 0.f;  // 2^(141 - eb)
#pragma unroll 1
            for (int part = 0; part < 2; ++part) {  // Re (S) then Im (D): z1, z2, z3, 8 columns each
                uint32_t a[24];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float v[2];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int kk = 2 * j + e;
                        float x = 0.f, y = 0.f;
                        if (kk < 8) {
                            if (kk < KH) upk(zE[kk], x, y);
                        } else if (kk - 8 < KH) {
                            upk(zO[kk - 8], x, y);
                        }
                        v[e] = (part ? y : x) * zsc;
                    }
                    // each difference is exact in FP32
                    a[j] = f16x2(v[0], v[1]);
                    const float r0 = v[0] - lo16(a[j]), r1 = v[1] - hi16(a[j]);
                    a[8 + j] = f16x2(r0, r1);
                    a[16 + j] = f16x2(r0 - lo16(a[8 + j]), r1 - hi16(a[8 + j]));
                }
                st8(lrow + gcol + 24 * part, a);
                st8(lrow + gcol + 24 * part + 8, a + 8);
                st8(lrow + gcol + 24 * part + 16, a + 16);
                // tcgen05.st reads its registers asynchronously: a[] is not reused before the wait
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&afull[group]);
            if (leader) {
                // every A row of the group written (so every lane has also read the
                // previous tile's S and D)
                if (mbar_wait(&afull[group], rpar, p.wait_cycles)) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    // F32 accumulators, FP16 A and B, N = npad, M = 128
                    const uint32_t idesc = (1u << 4) | ((uint32_t)(p.npad >> 3) << 17) | (8u << 24);
                    const uint32_t rb = smem_u32(rtab), tb = (uint32_t)p.npad * 32;
#pragma unroll
                    for (int sd = 0; sd < 2; ++sd) {
                        // S from the real parts (A columns 0..23), D from the imaginary ones (24..47)
                        const uint32_t d = gcol + 64 + (uint32_t)(sd * p.npad), a0 = gcol + 24 * sd;
                        const uint32_t w0 = rb + (uint32_t)(3 * sd) * tb;
                        mma_f16_ta(d, a0, umma_desc(w0, 128, 256), idesc, false);            // z1 w1
                        mma_f16_ta(d, a0 + 8, umma_desc(w0, 128, 256), idesc, true);         // z2 w1
                        mma_f16_ta(d, a0, umma_desc(w0 + tb, 128, 256), idesc, true);        // z1 w2
                        mma_f16_ta(d, a0, umma_desc(w0 + 2 * tb, 128, 256), idesc, true);    // z1 w3
                        mma_f16_ta(d, a0 + 8, umma_desc(w0 + tb, 128, 256), idesc, true);    // z2 w2
                        mma_f16_ta(d, a0 + 16, umma_desc(w0, 128, 256), idesc, true);        // z3 w1
                    }
                    umma_commit(&dfull[group]);
                    ++r_issued;
                } else {
                    atomicOr(p.err, kErrTimeout);  // the group's dfull waits run out too
                }
            }
            // lag step 0 in FP32 while the tensor cores run
            float S0, D0;
            eval_SD<KH>(recon, 0, zE, zO, S0, D0);
            const float y0 = S0 - D0;
            if (!__all_sync(FULLM, mbar_wait(&dfull[group], rpar, p.wait_cycles))) {
                if (lane == 0) atomicOr(p.err, kErrTimeout);
                break;
            }
            rpar ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const float fs = zsc * __uint_as_float((uint32_t)(127 + p.rshift) << 23);  // the MMA values' scale
            const float inv = fine ? __frcp_rn(fs) : 0.f;
            const size_t o = mine ? (size_t)(f0 + fl) * p.P + pq : 0;
            float *corr = (mine && p.out_corr) ? p.out_corr + o * p.I : nullptr;
            // the outward scan of the CUDA-core path over the MMA values (scaled by fs),
            // four columns at a time with the next four loading; rolled, so that the
            // epilogue stays small beside the record loop in the instruction cache
            float best = y0 * fs;
            int bi = p.center;
            auto take = [&](const float (&sv)[4], const float (&dv)[4], int c0) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int m = c0 + j + 1;
                    const float ym = sv[j] + dv[j], yp = sv[j] - dv[j];  // y(center - m), y(center + m)
                    if (m <= p.center) {
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
            };
            const uint32_t tS = lrow + gcol + 64, tD = tS + (uint32_t)p.npad;
            {
                float sa[4], da[4], sb[4], db[4];
                tmem_ld4_nw(tS, sa);
                tmem_ld4_nw(tD, da);
                tmem_wait_ld4(sa, da);
#pragma unroll 1
                for (int c0 = 0; c0 < p.npad; c0 += 8) {  // npad is a multiple of 32
                    tmem_ld4_nw(tS + (uint32_t)(c0 + 4), sb);
                    tmem_ld4_nw(tD + (uint32_t)(c0 + 4), db);
                    take(sa, da, c0);
                    __syncwarp();
                    tmem_wait_ld4(sb, db);
                    if (c0 + 8 < p.npad) {
                        tmem_ld4_nw(tS + (uint32_t)(c0 + 8), sa);
                        tmem_ld4_nw(tD + (uint32_t)(c0 + 8), da);
                    }
                    take(sb, db, c0 + 4);
                    __syncwarp();
                    tmem_wait_ld4(sa, da);
                }
            }
            if (p.out_corr) {
                // the correlation output (tests, diagnostics): every lag from the MMA values
#pragma unroll 1
                for (int c0 = 0; c0 < p.npad; c0 += 16) {
                    float sv[16], dv[16];
                    __syncwarp();
                    tmem_ld16_nw(tS + (uint32_t)c0, sv);
                    tmem_ld16_nw(tD + (uint32_t)c0, dv);
                    tmem_wait_ld(sv, dv);
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        const int m = c0 + jj + 1;
                        if (corr && m <= p.center) {
                            corr[p.center - m] = (sv[jj] + dv[jj]) * inv;
                            corr[p.center + m] = (sv[jj] - dv[jj]) * inv;
                        }
                    }
                }
            }
            if (mine) {
                if (fine) {
                    // the chosen lag's value in FP32, as the CUDA-core scan computes it
                    const int m = bi >= p.center ? bi - p.center : p.center - bi;
                    float S, D;
                    eval_SD<KH>(recon, m, zE, zO, S, D);
                    best = bi >= p.center ? S - D : S + D;
                    if (corr) {
                        corr[p.center] = y0;
                        corr[bi] = best;
                    }
                } else {
                    best = y0;
                    bi = p.center;
                    if (corr) corr[p.center] = y0;
                    scan(1, 1, best, bi, corr);
                }
                emit(o, bi, best);
            }
            continue;
        }
        if (p.C == 4) {
            // one chunk lane per pair
            if (active && pq >= 0) {
                const size_t o = (size_t)(f0 + fl) * p.P + pq;
                float *corr = p.out_corr ? p.out_corr + o * p.I : nullptr;
                float S, D;
                eval_SD<KH>(recon, 0, zE, zO, S, D);
                float best = S - D;
                int bi = p.center;
                if (corr) corr[p.center] = best;
                scan(1, 1, best, bi, corr);
                emit(o, bi, best);
            }
        } else {
            // the C / 4 chunk lanes holding the same pair (the reduction leaves
            // its coefficients in all of them) split the lag steps m = gi,
            // gi + C/4, ... and combine their maxima with shuffles: value first,
            // then the lower lag index, as one outward scan would
            const int G4 = p.C >> 2, gi = chunk >> 2;
            const bool mine = active && pq >= 0;
            const size_t o = mine ? (size_t)(f0 + fl) * p.P + pq : 0;
            float best = -FLT_MAX;
            int bi = 0x7fffffff;
            if (mine) {
                float *corr = p.out_corr ? p.out_corr + o * p.I : nullptr;
                int m0 = gi;
                if (gi == 0) {
                    float S, D;
                    eval_SD<KH>(recon, 0, zE, zO, S, D);
                    best = S - D;
                    bi = p.center;
                    if (corr) corr[p.center] = best;
                    m0 = G4;
                }
                scan(m0, G4, best, bi, corr);
            }
            for (int off = 4 * p.SB; off < 32; off <<= 1) {
                const float ob = __shfl_xor_sync(FULLM, best, off);
                const int oi = __shfl_xor_sync(FULLM, bi, off);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (mine && gi == 0) emit(o, bi, best);
        }
    }
    // never retire with one of this group's bulk copies still in flight: wait,
    // with the full bound whatever the test hook set, for every copy that was
    // issued and not yet seen landing (a withheld or never-issued tile has no
    // copy to wait for)
    if (p.bulk && leader) {
        for (int k = k_done + p.G; k < n_local && k <= k_done + p.S; k += p.G)
            if ((inflight >> (k % p.S)) & 1u)
                if (!mbar_wait(&full[k % p.S], (unsigned)(k / p.S) & 1u, kWaitCycles)) atomicOr(p.err, kErrTimeout);
    }
    if (mma) {
        // never free tensor memory under a reconstruction MMA still running
        if (leader && r_issued > 0 && !mbar_wait(&dfull[group], (unsigned)(r_issued - 1) & 1u, kWaitCycles))
            atomicOr(p.err, kErrTimeout);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (warp == 0) {
            __syncwarp();
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
        }
    }
}

}  // namespace
}  // namespace fcc
