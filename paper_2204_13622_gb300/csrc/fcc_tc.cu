// fcc_tc.cu -- the BF16 / FP16 precision forms of the FCC hot path on the
// 5th-generation tensor cores (tcgen05, sm_103a).
//
// The projection of Eq. 9 is a dense contraction over the folded bins:
//   z_e^c[n] = sum_k A_e[row, 2k + c] * pe_n(k),   z_o^c[n] = sum_k A_o[row, 2k + c] * po_n(k),
// where row is one microphone pair of the tile, c = 0 / 1 the real / imaginary
// part and A_e = (Re x_s, Im x_s), A_o = (Re x_d, Im x_d) interleaved along k
// (Eq. 8).  Written as D = A B with B[(k,c), (c',n)] = p_n(k) [c = c'], one
// tcgen05.mma (M = 128 rows, N = 16 = (c', n), K = 16) per 8 bins and part.
//
// Roles in a CTA (persistent over frame tiles of TS = F * slots <= 32 slots):
//   * 8 producer warps: PHAT of the staged raw frames into FP16 unit-phase
//     records (FP32 arithmetic; the raw stage is released right after), then
//     per 32-bin chunk the cross spectra of their 2x2 pair blocks in FP32,
//     folded and rounded to BF16 / FP16 into the chunk's A tiles (shared
//     memory, K-major 8x16-byte core matrices; row = q * 32 + slot so that a
//     quarter-warp's 16-byte stores cover one core matrix);
//   * 1 MMA warp: allocates TMEM, issues the MMAs of each chunk when its A
//     tiles are full (FP32 accumulators, two TMEM buffers so that a tile's
//     epilogue overlaps the next tile's MMAs) and commits them to mbarriers;
//   * 1 copy warp: streams raw frame tiles with one cp.async.bulk per tile.
// Epilogue (8 warps of their own, two per TMEM lane quadrant = pair q of every
// slot, a tile behind the producers): tcgen05.ld of the pair's 2K
// coefficients, the lone bin N/4 (from the producers, through shared memory)
// added in FP32, then the lag-grid reconstruction, split between the two warps
// of the quadrant, argmax and refinement as the FP32 path.  On long lag grids
// the reconstruction is itself a contraction on the tensor cores: per lag step
// m, S(m) and D(m) (y(center -/+ m) = S +/- D) are the real and imaginary
// coefficient parts against the step's weights, written by the epilogue as an
// FP16 hi / lo A operand in tensor memory and multiplied by resident FP16 hi / lo
// weight tables (three passes, about 22 bits), one MMA group per tile issued
// by an epilogue thread; the warps then read S and D back with tcgen05.ld.
// Every wait is bounded; TMEM is released on every exit path.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdlib>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fcc_device.cuh"
#include "fcc_internal.h"

namespace fcc {
namespace {

constexpr int kProdWarps = 8;                 // producer warps (one 4-bin group each)
constexpr int kEpiWarps = 8;                 // epilogue warps: two per TMEM lane quadrant (pair q)
constexpr int kEpi0 = kProdWarps + 2;         // first epilogue warp
constexpr int kThreadsTC = (kProdWarps + 2 + kEpiWarps) * 32;
constexpr int kChunkRec = 4 * kProdWarps;     // bins per chunk (32)
constexpr int kChunkCols = 2 * kChunkRec;     // A columns per part per chunk (64)
constexpr int kPartBytes = 128 * kChunkCols * 2;  // one part of one chunk (16 KB)
constexpr int kNTile = 16;                    // MMA N: (c', n) with n < 8
constexpr int kTmemCols = 64;                 // two (even, odd) accumulator buffers
// With the reconstruction on the tensor cores: A2 (the coefficients as FP16
// hi / lo, 4 x 8 columns) at kA2Col, then S (npad columns) and D (npad) at kD2Col.
constexpr int kTmemColsRecon = 512;
constexpr int kA2Col = 64;
constexpr int kD2Col = 96;
constexpr int kMaxNpad = (kTmemColsRecon - kD2Col) / 2;  // 208

struct TcLayout {
    size_t bar, slot, bas_e, bas_o, peq, recon, rbase, lone, comb, abuf, ubuf, raw, total;
    int ustride;  // bytes per unit-phase row
};

__host__ __device__ inline TcLayout tc_layout(int n_slots, int Q, int kh, int center, int rows_tile, int F,
                                              int frame_bytes, int npad)
{
    TcLayout L;
    size_t o = 0;
    L.bar = o;
    o += 32 * 8 + 16;  // mbarriers + TMEM address
    o = (o + 15) & ~(size_t)15;
    L.slot = o;
    o += (size_t)n_slots * sizeof(Slot);
    o = (o + 127) & ~(size_t)127;
    L.bas_e = o;
    o += (size_t)kNTile * 2 * Q * 2;
    L.bas_o = o;
    o += (size_t)kNTile * 2 * Q * 2;
    L.peq = o;
    o += 8 * sizeof(float);
    o = (o + 15) & ~(size_t)15;
    L.recon = o;  // the FP32 reconstruction table, for the CUDA-core scan only
    if (!npad) o += (size_t)(center + 1) * 4 * kh * sizeof(float);
    o = (o + 127) & ~(size_t)127;
    L.rbase = o;  // the FP16 tables of the tensor-core reconstruction
    o += (size_t)4 * npad * 16 * 2;
    o = (o + 15) & ~(size_t)15;
    L.lone = o;  // [2][4][32] float2: the lone bin's cross spectrum per tile parity, pair, slot
    o += 2 * 4 * 32 * 8;
    L.comb = o;  // [2][4][32] (float, int): the second half's maximum per tile parity, pair, slot
    o += 2 * 4 * 32 * 8;
    o = (o + 127) & ~(size_t)127;
    L.abuf = o;
    o += 2 * 2 * (size_t)kPartBytes;
    L.ustride = Q * 8 + 24;  // 8-byte records + lone + pad: rows fall on distinct bank pairs
    L.ubuf = o;
    o += (size_t)rows_tile * L.ustride;
    o = (o + 127) & ~(size_t)127;
    L.raw = o;
    o += (((size_t)F * frame_bytes) + 127) & ~(size_t)127;
    L.total = o;
    return L;
}

template <int PREC>
__device__ __forceinline__ uint32_t pack16(float lo, float hi)
{
    if constexpr (PREC == FCC_PREC_BF16) {
        __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&h);
    } else {
        __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&h);
    }
}

__device__ __forceinline__ float4 rec_f32(uint2 r)
{
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&r.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&r.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

// Barriers (indices into the mbarrier array).
enum {
    kFull = 0,     // raw tile landed (tx)
    kRawEmpty,     // producers done reading the raw tile
    kUReady,       // unit-phase records written
    kUFree,        // producers done reading the unit-phase records
    kAFull0,       // A buffer 0 / 1 written by the producers
    kAFull1,
    kAEmpty0,      // MMAs reading A buffer 0 / 1 done (tcgen05.commit)
    kAEmpty1,
    kDFull0,       // accumulator buffer 0 / 1 complete (tcgen05.commit)
    kDFull1,
    kDEmpty0,      // accumulator buffer 0 / 1 read by the epilogue
    kDEmpty1,
    kLoneFull0,    // the lone bin of tile parity 0 / 1 written by producers 0..3
    kLoneFull1,
    kLoneFree0,    // ... read by the epilogue warps
    kLoneFree1,
    kCombFull0,    // the second half's maxima of tile parity 0 / 1 written
    kCombFull1,
    kCombFree0,    // ... read by the first half
    kCombFree1,
    kA2Full,       // reconstruction: the coefficients written as the A operand (4 warps)
    kD2Full,       // reconstruction MMAs complete (tcgen05.commit)
    kD2Free,       // S and D read by the 8 epilogue warps
    kNumBars
};

template <int KH, int RS, int PREC>
__global__ void __launch_bounds__(kThreadsTC, 1) fcc_tc_kernel(const TcParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int frame_bytes = p.M * p.B * 8;
    const int rows_tile = p.F * p.M;
    const TcLayout lay = tc_layout(p.n_slots, p.Q, KH, p.center, rows_tile, p.F, frame_bytes, p.npad);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + lay.bar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + lay.bar + kNumBars * 8);
    Slot *slots = reinterpret_cast<Slot *>(smem + lay.slot);
    float *peq = reinterpret_cast<float *>(smem + lay.peq);
    float *recon = reinterpret_cast<float *>(smem + lay.recon);
    float2 *lone_buf = reinterpret_cast<float2 *>(smem + lay.lone);
    float *comb_s = reinterpret_cast<float *>(smem + lay.comb);
    int *comb_i = reinterpret_cast<int *>(smem + lay.comb) + 2 * 4 * 32;
    unsigned char *abuf = smem + lay.abuf;
    unsigned char *ubuf = smem + lay.ubuf;
    unsigned char *raw = smem + lay.raw;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Q = p.Q, B = p.B, M = p.M;
    const int nch = Q / kChunkRec;
    const int n_local = (p.n_tiles > (int)blockIdx.x)
                            ? (p.n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x
                            : 0;

    if (threadIdx.x == 0) {
        mbar_init(&bar[kFull], 1);
        mbar_init(&bar[kRawEmpty], kProdWarps);
        mbar_init(&bar[kUReady], kProdWarps);
        mbar_init(&bar[kUFree], kProdWarps);
        mbar_init(&bar[kAFull0], kProdWarps);
        mbar_init(&bar[kAFull1], kProdWarps);
        mbar_init(&bar[kAEmpty0], 1);
        mbar_init(&bar[kAEmpty1], 1);
        mbar_init(&bar[kDFull0], 1);
        mbar_init(&bar[kDFull1], 1);
        mbar_init(&bar[kDEmpty0], kEpiWarps);
        mbar_init(&bar[kDEmpty1], kEpiWarps);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bar[kLoneFull0 + b], 4);
            mbar_init(&bar[kLoneFree0 + b], kEpiWarps);
            mbar_init(&bar[kCombFull0 + b], kEpiWarps / 2);
            mbar_init(&bar[kCombFree0 + b], kEpiWarps / 2);
        }
        mbar_init(&bar[kA2Full], kEpiWarps / 2);
        mbar_init(&bar[kD2Full], 1);
        mbar_init(&bar[kD2Free], kEpiWarps);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int e = threadIdx.x; e < p.n_slots; e += blockDim.x) slots[e] = p.slots[e];
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(p.bases);
        uint4 *dst = reinterpret_cast<uint4 *>(smem + lay.bas_e);
        const int n16 = 2 * kNTile * 2 * Q * 2 / 16;
        for (int e = threadIdx.x; e < n16; e += blockDim.x) dst[e] = src[e];
    }
    for (int e = threadIdx.x; e < 8; e += blockDim.x) peq[e] = p.peq[e];
    if (p.npad) {
        const uint4 *src = reinterpret_cast<const uint4 *>(p.rbases);
        uint4 *dst = reinterpret_cast<uint4 *>(smem + lay.rbase);
        for (int e = threadIdx.x; e < 4 * p.npad * 16 * 2 / 16; e += blockDim.x) dst[e] = src[e];
    } else {
        for (int e = threadIdx.x; e < (p.center + 1) * 4 * KH; e += blockDim.x) recon[e] = p.recon[e];
    }
    fence_proxy_async();
    const uint32_t tcols = p.npad ? (uint32_t)kTmemColsRecon : (uint32_t)kTmemCols;
    if (warp == kProdWarps) {  // the MMA warp owns the tensor memory
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    auto tile_src = [&](int k, int &nf) {
        const long long tile = (long long)blockIdx.x + (long long)k * gridDim.x;
        const long long f0 = tile * p.F;
        nf = (int)min((long long)p.F, p.T - f0);
        return f0;
    };

    if (warp == kProdWarps + 1) {
        // ================= copy warp =================
        if (lane == 0) {
            int issued = 0;
            for (int k = 0; k < n_local; ++k) {
                if (!mbar_wait(&bar[kRawEmpty], ((unsigned)k & 1u) ^ 1u)) {
                    atomicOr(p.err, kErrTimeout);
                    break;
                }
                int nf;
                const long long f0 = tile_src(k, nf);
                const unsigned bytes = (unsigned)nf * (unsigned)frame_bytes;
                mbar_arrive_expect_tx(&bar[kFull], bytes);
                bulk_g2s(raw, reinterpret_cast<const unsigned char *>(p.spectra) + (size_t)f0 * frame_bytes, bytes,
                         &bar[kFull]);
                issued = k + 1;
            }
            // never retire with the last bulk copy still in flight
            if (issued > 0 && !mbar_wait(&bar[kFull], (unsigned)(issued - 1) & 1u)) atomicOr(p.err, kErrTimeout);
        }
    } else if (warp == kProdWarps) {
        // ================= MMA warp =================
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (PREC == FCC_PREC_BF16 ? (1u << 7) | (1u << 10) : 0u) |
                                   ((uint32_t)(kNTile >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
            const uint32_t a_base = smem_u32(abuf);
            const uint32_t be = smem_u32(smem + lay.bas_e), bo = smem_u32(smem + lay.bas_o);
            const uint32_t b_sbo = (uint32_t)(2 * Q / 8) * 128;
            long long cc = 0;  // chunks issued so far
            bool ok = true;
            for (int k = 0; k < n_local && ok; ++k) {
                const int db = k & 1;
                if (!mbar_wait(&bar[kDEmpty0 + db], ((unsigned)(k >> 1) & 1u) ^ 1u)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d_e = tmem + db * 32, d_o = d_e + 16;
                for (int ch = 0; ch < nch; ++ch, ++cc) {
                    const int b = (int)(cc & 1);
                    if (!mbar_wait(&bar[kAFull0 + b], (unsigned)(cc >> 1) & 1u)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t ae = a_base + b * 2 * kPartBytes, ao = ae + kPartBytes;
#pragma unroll
                    for (int ks = 0; ks < kChunkCols / 16; ++ks) {
                        const uint32_t koff = ks * 2 * 128;
                        const uint32_t kb = (uint32_t)(ch * (kChunkCols / 8) + ks * 2) * 128;
                        const bool acc = (ch > 0) || (ks > 0);
                        umma_f16(d_e, umma_desc(ae + koff, 128, 1024), umma_desc(be + kb, 128, b_sbo), idesc, acc);
                        umma_f16(d_o, umma_desc(ao + koff, 128, 1024), umma_desc(bo + kb, 128, b_sbo), idesc, acc);
                    }
                    umma_commit(&bar[kAEmpty0 + b]);
                }
                if (ok) umma_commit(&bar[kDFull0 + db]);
            }
            if (!ok) atomicOr(p.err, kErrTimeout);
            // retire only when the last MMAs have completed
            if (cc > 0) {
                const int b = (int)((cc - 1) & 1);
                if (!mbar_wait(&bar[kAEmpty0 + b], (unsigned)((cc - 1) >> 1) & 1u)) atomicOr(p.err, kErrTimeout);
            }
        }
    } else if (warp < kProdWarps) {
        // ================= producer warps =================
        const int g = warp;         // bin group within a chunk
        const int sp = lane;        // slot within the tile
        const int TS = p.F * p.n_slots;
        const bool live = sp < TS;
        const int fl = live ? sp / p.n_slots : 0;
        Slot sl{};
        if (live) sl = slots[sp - fl * p.n_slots];
        const unsigned FULLM = 0xffffffffu;
        long long cc = 0;
        for (int k = 0; k < n_local; ++k) {
            int nf;
            const long long f0 = tile_src(k, nf);
            const unsigned par = (unsigned)k & 1u;
            // unit-phase records may be rewritten once the previous tile is done with them
            if (!mbar_wait(&bar[kUFree], par ^ 1u) || !mbar_wait(&bar[kFull], par)) {
                if (lane == 0) atomicOr(p.err, kErrTimeout);
                break;
            }
            // ---- PHAT (FP32) into FP16 folded records: row R = (frame, mic)
            {
                bool bad = false;
                for (int R = warp; R < nf * M; R += kProdWarps) {
                    const float2 *xr = reinterpret_cast<const float2 *>(raw + (size_t)R * B * 8);
                    uint2 *rec = reinterpret_cast<uint2 *>(ubuf + (size_t)R * lay.ustride);
#pragma unroll
                    for (int j = 0; j < RS; ++j) {
                        const int fp = lane + 32 * j;
                        if (RS > 1 || fp < Q) {
                            bool o1, o2;
                            float2 a = unit_phase_fast(xr[fp], o1);
                            float2 b = unit_phase_fast(xr[2 * Q - fp], o2);
                            if (!(o1 && o2)) {
                                a = unit_phase_slow(xr[fp], bad);
                                b = unit_phase_slow(xr[2 * Q - fp], bad);
                            }
                            const __half2 ha = __floats2half2_rn(a.x, a.y), hb = __floats2half2_rn(b.x, b.y);
                            rec[fp] = make_uint2(*reinterpret_cast<const uint32_t *>(&ha),
                                                 *reinterpret_cast<const uint32_t *>(&hb));
                        }
                    }
                    if (lane == 0) {
                        bool o;
                        float2 c = unit_phase_fast(xr[Q], o);
                        if (!o) c = unit_phase_slow(xr[Q], bad);
                        const __half2 hc = __floats2half2_rn(c.x, c.y);
                        *reinterpret_cast<__half2 *>(ubuf + (size_t)R * lay.ustride + 8 * Q) = hc;
                    }
                }
                if (__any_sync(FULLM, bad) && lane == 0) atomicOr(p.err, kErrNonFinite);
            }
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&bar[kRawEmpty]);  // raw tile consumed: the copy warp may refill it
                mbar_arrive(&bar[kUReady]);
            }
            if (!mbar_wait(&bar[kUReady], par)) {
                if (lane == 0) atomicOr(p.err, kErrTimeout);
                break;
            }
            // ---- A tiles, one 32-bin chunk at a time
            const int R0 = fl * M;
            const uint2 *u0 = reinterpret_cast<const uint2 *>(ubuf + (size_t)(R0 + sl.mic[0]) * lay.ustride);
            const uint2 *u1 = reinterpret_cast<const uint2 *>(ubuf + (size_t)(R0 + sl.mic[1]) * lay.ustride);
            const uint2 *u2 = reinterpret_cast<const uint2 *>(ubuf + (size_t)(R0 + sl.mic[2]) * lay.ustride);
            const uint2 *u3 = reinterpret_cast<const uint2 *>(ubuf + (size_t)(R0 + sl.mic[3]) * lay.ustride);
            // the lone bin N/4 of this thread's own pair (q = warp for warps 0..3), for
            // the epilogue warps: its buffer (tile parity) is free once they read it
            // two tiles ago
            bool ok = true;
            if (warp < 4) {
                const int db = k & 1;
                if (!__all_sync(0xffffffffu, mbar_wait(&bar[kLoneFree0 + db], ((unsigned)(k >> 1) & 1u) ^ 1u))) {
                    ok = false;
                } else {
                    float lone_r = 0.f, lone_i = 0.f;
                    if (live) {
                        const int q = warp;
                        const __half2 hx = *reinterpret_cast<const __half2 *>(
                            ubuf + (size_t)(R0 + sl.mic[q >> 1]) * lay.ustride + 8 * Q);
                        const __half2 hy = *reinterpret_cast<const __half2 *>(
                            ubuf + (size_t)(R0 + sl.mic[2 + (q & 1)]) * lay.ustride + 8 * Q);
                        const float2 x = __half22float2(hx), y = __half22float2(hy);
                        lone_r = fmaf(x.x, y.x, x.y * y.y);
                        lone_i = fmaf(x.y, y.x, -(x.x * y.y));
                    }
                    lone_buf[(db * 4 + warp) * 32 + sp] = make_float2(lone_r, lone_i);
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&bar[kLoneFull0 + db]);
                }
            }
            for (int ch = 0; ch < nch && ok; ++ch, ++cc) {
                const int b = (int)(cc & 1);
                if (!mbar_wait(&bar[kAEmpty0 + b], ((unsigned)(cc >> 1) & 1u) ^ 1u)) {
                    ok = false;
                    break;
                }
                uint32_t we[4][4], wo[4][4];  // [pair][bin]: packed (re, im) of x_s / x_d
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int kk = ch * kChunkRec + 4 * g + r;
                    const float4 X[2] = {rec_f32(u0[kk]), rec_f32(u1[kk])};
                    const float4 Y[2] = {rec_f32(u2[kk]), rec_f32(u3[kk])};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 x = X[q >> 1], y = Y[q & 1];
                        const float ar = fmaf(x.x, y.x, x.y * y.y), ai = fmaf(x.y, y.x, -(x.x * y.y));
                        const float br = fmaf(x.z, y.z, x.w * y.w), bi = fmaf(x.w, y.z, -(x.z * y.w));
                        we[q][r] = pack16<PREC>(ar + br, ai + bi);  // x_s (Eq. 8)
                        wo[q][r] = pack16<PREC>(ar - br, ai - bi);  // x_d
                    }
                }
                unsigned char *ae = abuf + b * 2 * kPartBytes, *ao = ae + kPartBytes;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int row = 32 * q + sp;
                    const int off = ((row >> 3) * (kChunkCols / 8) + g) * 128 + (row & 7) * 16;
                    const uint4 ve = live ? make_uint4(we[q][0], we[q][1], we[q][2], we[q][3]) : make_uint4(0, 0, 0, 0);
                    const uint4 vo = live ? make_uint4(wo[q][0], wo[q][1], wo[q][2], wo[q][3]) : make_uint4(0, 0, 0, 0);
                    *reinterpret_cast<uint4 *>(ae + off) = ve;
                    *reinterpret_cast<uint4 *>(ao + off) = vo;
                }
                fence_proxy_async();  // generic-proxy stores -> tensor-core reads
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar[kAFull0 + b]);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[kUFree]);
            if (!ok) {
                if (lane == 0) atomicOr(p.err, kErrTimeout);
                break;
            }
        }
    } else {
        // ================= epilogue warps =================
        // Warp w reads TMEM lane quadrant w % 4, i.e. pair q of every slot; the two
        // warps of a quadrant split the lag steps (half h = 0: m < mid, including
        // m = 0; h = 1: the rest) and h = 0 takes the larger of the two maxima
        // (lowest index on a tie) and writes the outputs (every wait's outcome is
        // made warp-uniform before the warp acts on it).  They run a tile behind
        // the producers (two accumulator buffers), so reconstruction overlaps
        // the next tile's PHAT and A tiles.
        const int q = warp & 3, h = (warp - kEpi0) >> 2;
        const int sp = lane;
        const int TS = p.F * p.n_slots;
        const bool live = sp < TS;
        const int fl = live ? sp / p.n_slots : 0;
        Slot sl{};
        if (live) sl = slots[sp - fl * p.n_slots];
        const int pq = q == 0 ? sl.pair[0] : q == 1 ? sl.pair[1] : q == 2 ? sl.pair[2] : sl.pair[3];
        const int mid = (p.center + 1) / 2;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        const float *rtab = p.npad ? p.recon : recon;  // FP32 rows for the refinement
        int r_issued = 0;  // tiles whose reconstruction MMAs this thread issued
        bool ok = true;
        for (int k = 0; k < n_local; ++k) {
            int nf;
            const long long f0 = tile_src(k, nf);
            const int db = k & 1;
            const unsigned par = (unsigned)(k >> 1) & 1u;
            if (!__all_sync(0xffffffffu, mbar_wait(&bar[kDFull0 + db], par))) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float de[16], dd[16];
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + db * 32;
            tmem_ld16(taddr, de);
            tmem_ld16(taddr + 16, dd);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[kDEmpty0 + db]);
            if (!__all_sync(0xffffffffu, mbar_wait(&bar[kLoneFull0 + db], par))) {
                ok = false;
                break;
            }
            const float2 lone = lone_buf[(db * 4 + q) * 32 + sp];
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[kLoneFree0 + db]);
            const bool act = live && fl < nf && pq >= 0;
            f2 zE[KH], zO[KH];
#pragma unroll
            for (int v = 0; v < KH; ++v) {
                zE[v] = pk(fmaf(peq[v], lone.x, de[v]), fmaf(peq[v], lone.y, de[8 + v]));
                zO[v] = pk(dd[v], dd[8 + v]);
            }
            const size_t o = act ? (size_t)(f0 + fl) * p.P + pq : 0;
            float *corr = (act && p.out_corr) ? p.out_corr + o * p.I : nullptr;
            float best = -FLT_MAX;
            int bi = 0x7fffffff;
            // the scan over lag steps m of this warp's half: y(center - m) = S + D is below
            // every index seen so far (wins ties), y(center + m) = S - D above (loses ties)
            auto take = [&](int m, float S, float D) {
                if (m == 0) {
                    best = S - D;
                    bi = p.center;
                    if (corr) corr[p.center] = best;
                    return;
                }
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
            };
            const int m_lo = h == 0 ? 0 : mid, m_hi = h == 0 ? mid : p.center + 1;
            if (p.npad) {
                // ---- the reconstruction on the tensor cores: per lag step m,
                // S(m) = sum_k A_re[k] G_S[m][k] and D(m) = sum_k A_im[k] G_D[m][k] with
                // A_re = (Re zE, Re zO), A_im = (Im zE, Im zO) (16 parts each, zero past
                // KH), as three FP16 passes A_hi G_hi + A_lo G_hi + A_hi G_lo (about 22
                // bits), FP32 accumulation into tensor memory
                if (h == 0) {
                    // A_re hi, A_re lo, A_im hi, A_im lo: 8 packed pairs each, the real parts
                    // first, then the imaginary parts (16 registers at a time)
                    const uint32_t ta = tmem + lane_base + kA2Col;
#pragma unroll
                    for (int part = 0; part < 2; ++part) {
                        uint32_t a[16];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            float v[2];
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                const int k = 2 * j + e;
                                float x = 0.f, y = 0.f;
                                if (k < 8) {
                                    if (k < KH) upk(zE[k], x, y);
                                } else if (k - 8 < KH) {
                                    upk(zO[k - 8], x, y);
                                }
                                v[e] = act ? (part ? y : x) : 0.f;
                            }
                            a[j] = f16x2(v[0], v[1]);
                            a[8 + j] = f16x2(v[0] - lo16(a[j]), v[1] - hi16(a[j]));
                        }
                        st8(ta + 16 * part, a);
                        st8(ta + 16 * part + 8, a + 8);
                        // tcgen05.st reads its registers asynchronously: a[] is not reused
                        // before the wait
                        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    }
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&bar[kA2Full]);
                }
                if (warp == kEpi0 && lane == 0) {
                    // the issuer: every A2 row written, and S / D of the previous tile read
                    bool go = mbar_wait(&bar[kA2Full], (unsigned)k & 1u);
                    if (go && k > 0) go = mbar_wait(&bar[kD2Free], (unsigned)(k - 1) & 1u);
                    if (go) {
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t idesc = (1u << 4) | ((uint32_t)(p.npad >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
                        const uint32_t rb = smem_u32(smem + lay.rbase), tb = (uint32_t)p.npad * 32;
                        const uint32_t dS = tmem + kD2Col, dD = dS + (uint32_t)p.npad, aa = tmem + kA2Col;
                        mma_f16_ta(dS, aa, umma_desc(rb, 128, 256), idesc, false);
                        mma_f16_ta(dS, aa + 8, umma_desc(rb, 128, 256), idesc, true);
                        mma_f16_ta(dS, aa, umma_desc(rb + tb, 128, 256), idesc, true);
                        mma_f16_ta(dD, aa + 16, umma_desc(rb + 2 * tb, 128, 256), idesc, false);
                        mma_f16_ta(dD, aa + 24, umma_desc(rb + 2 * tb, 128, 256), idesc, true);
                        mma_f16_ta(dD, aa + 16, umma_desc(rb + 3 * tb, 128, 256), idesc, true);
                        umma_commit(&bar[kD2Full]);
                        ++r_issued;
                    }
                    // on a timeout the other warps' D2Full waits run out too
                }
                if (!__all_sync(0xffffffffu, mbar_wait(&bar[kD2Full], (unsigned)k & 1u))) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int c0 = m_lo & ~15; c0 < m_hi; c0 += 16) {
                    float sv[16], dv[16];
                    tmem_ld16(tmem + lane_base + kD2Col + (uint32_t)c0, sv);
                    tmem_ld16(tmem + lane_base + kD2Col + (uint32_t)(p.npad + c0), dv);
                    if (act) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int m = c0 + j;
                            if (m >= m_lo && m < m_hi) take(m, sv[j], dv[j]);
                        }
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar[kD2Free]);
            } else if (act) {
                float S, D;
                for (int m = m_lo; m < m_hi; ++m) {
                    eval_SD<KH>(recon, m, zE, zO, S, D);
                    take(m, S, D);
                }
            }
            const int ci = (db * 4 + q) * 32 + sp;
            if (h == 1) {
                if (!__all_sync(0xffffffffu, mbar_wait(&bar[kCombFree0 + db], par ^ 1u))) {
                    ok = false;
                    break;
                }
                comb_s[ci] = best;
                comb_i[ci] = bi;
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar[kCombFull0 + db]);
                continue;
            }
            if (!__all_sync(0xffffffffu, mbar_wait(&bar[kCombFull0 + db], par))) {
                ok = false;
                break;
            }
            const float ob = comb_s[ci];
            const int oi = comb_i[ci];
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[kCombFree0 + db]);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
            if (act) {
                p.out_idx[o] = bi;
                p.out_peak[o] = best;
                if (p.out_tau) {
                    float off = 0.f;
                    if (bi > 0 && bi < p.I - 1) {
                        const double y_m = y_at<KH>(rtab, p.center, bi - 1, zE, zO);
                        const double y_p = y_at<KH>(rtab, p.center, bi + 1, zE, zO);
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
        // never free tensor memory under a reconstruction MMA still running
        if (r_issued > 0 && !mbar_wait(&bar[kD2Full], (unsigned)(r_issued - 1) & 1u, kWaitCycles))
            atomicOr(p.err, kErrTimeout);
        if (!ok && lane == 0) atomicOr(p.err, kErrTimeout);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == kProdWarps)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
}

template <int KH, int RS, int PREC>
fcc_status_t launch_tc_inst(const fcc_plan *plan, const TcParams &prm, cudaStream_t st, int grid)
{
    static bool attr_set[64] = {};
    const int dev = plan->device;
    if (!attr_set[dev & 63]) {
        cudaError_t e = cudaFuncSetAttribute(fcc_tc_kernel<KH, RS, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             232448);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(fcc_tc_kernel)");
        attr_set[dev & 63] = true;
    }
    fcc_tc_kernel<KH, RS, PREC><<<grid, kThreadsTC, plan->tc_smem, st>>>(prm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fcc_tc_kernel launch");
    return FCC_OK;
}

template <int KH, int PREC>
fcc_status_t launch_tc_kh(const fcc_plan *plan, const TcParams &prm, cudaStream_t st, int grid)
{
    switch (prm.Q / 32) {
    case 1: return launch_tc_inst<KH, 1, PREC>(plan, prm, st, grid);
    case 2: return launch_tc_inst<KH, 2, PREC>(plan, prm, st, grid);
    case 4: return launch_tc_inst<KH, 4, PREC>(plan, prm, st, grid);
    case 8: return launch_tc_inst<KH, 8, PREC>(plan, prm, st, grid);
    default: return fail(FCC_ERR_UNSUPPORTED, "the tensor-core path needs 128 <= N <= 1024");
    }
}

template <int PREC>
fcc_status_t launch_tc_prec(const fcc_plan *plan, const TcParams &prm, cudaStream_t st, int grid)
{
    switch (plan->kh) {
    case 2: return launch_tc_kh<2, PREC>(plan, prm, st, grid);
    case 4: return launch_tc_kh<4, PREC>(plan, prm, st, grid);
    case 6: return launch_tc_kh<6, PREC>(plan, prm, st, grid);
    case 8: return launch_tc_kh<8, PREC>(plan, prm, st, grid);
    default: return fail(FCC_ERR_UNSUPPORTED, "more than 8 bases of one parity");
    }
}

}  // namespace

// Host side: check the tensor-core path applies and size its shared memory;
// pack the basis tiles (K-major core matrices, rows (c', n), columns (k, c)).
fcc_status_t prepare_tc(fcc_plan *plan)
{
    const fcc_plan_info_t &in = plan->info;
    if (in.Q % kChunkRec != 0 || in.Q > 256)
        return fail(FCC_ERR_UNSUPPORTED, "the tensor-core path needs 128 <= N <= 1024");
    if (plan->n_slots > 32) return fail(FCC_ERR_UNSUPPORTED, "the tensor-core path needs M <= 16");
    if (!plan->kh) return fail(FCC_ERR_UNSUPPORTED, "more than 8 bases of one parity");
    const int frame_bytes = in.M * in.B * 8;
    if (frame_bytes % 16) return fail(FCC_ERR_UNSUPPORTED, "the tensor-core path needs an even number of mics");
    int smem_max = 0;
    FCC_CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, plan->device));
    smem_max = std::min(smem_max, 232448);
    // the reconstruction on the tensor cores for long lag grids (center >= 32: the
    // 16-mic grid's 97 lag steps take 14.5 instead of 17.8 ms; the 8-mic circle's 21
    // steps are 1 % faster on the CUDA cores) whose S and D fit the tensor memory
    // beside the accumulators; else the CUDA-core scan
    int npad = in.center >= 32 ? ((in.center + 1) + 15) & ~15 : 0;
    if (npad > kMaxNpad) npad = 0;
    int F = std::max(1, 32 / plan->n_slots);
    TcLayout L{};
    for (; F >= 1; --F) {
        L = tc_layout(plan->n_slots, in.Q, plan->kh, in.center, F * in.M, F, frame_bytes, npad);
        if (L.total <= (size_t)smem_max) break;
    }
    if (F < 1) return fail(FCC_ERR_UNSUPPORTED, "frame too large for the tensor-core path");
    plan->tc_F = F;
    plan->tc_smem = L.total;
    plan->tc_npad = npad;
    if (npad) {
        const std::vector<uint16_t> rt = recon_tables_f16(plan, npad, 0, 0, 2);
        FCC_CUDA_TRY(cudaMalloc(&plan->d_tc_rbases, rt.size() * sizeof(uint16_t)));
        FCC_CUDA_TRY(cudaMemcpy(plan->d_tc_rbases, rt.data(), rt.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    }
    // basis tiles, BF16 or FP16
    const int Q = in.Q, KB = 2 * Q;  // columns (k, c), k < Q
    std::vector<uint16_t> tiles((size_t)2 * kNTile * KB, 0);
    auto put = [&](int part, int n, int kc, double v) {
        const size_t off = (size_t)part * kNTile * KB +
                           (((size_t)(n / 8) * (KB / 8) + kc / 8) * 64 + (n % 8) * 8 + (kc % 8));
        if (in.prec == FCC_PREC_BF16) {
            __nv_bfloat16 h = __float2bfloat16_rn((float)v);
            tiles[off] = *reinterpret_cast<uint16_t *>(&h);
        } else {
            __half h = __float2half_rn((float)v);
            tiles[off] = *reinterpret_cast<uint16_t *>(&h);
        }
    };
    for (int c = 0; c < 2; ++c)
        for (int nb = 0; nb < 8; ++nb)
            for (int k = 0; k < Q; ++k) {
                const int n = c * 8 + nb, kc = 2 * k + c;
                put(0, n, kc, nb < in.K_even ? plan->Pe[(size_t)nb * (Q + 1) + k] : 0.0);
                put(1, n, kc, nb < in.K_odd ? plan->Po[(size_t)nb * Q + k] : 0.0);
            }
    std::vector<float> peq(8, 0.f);
    for (int nb = 0; nb < in.K_even && nb < 8; ++nb) peq[nb] = (float)plan->Pe[(size_t)nb * (Q + 1) + Q];
    FCC_CUDA_TRY(cudaMalloc(&plan->d_tc_bases, tiles.size() * sizeof(uint16_t)));
    FCC_CUDA_TRY(cudaMemcpy(plan->d_tc_bases, tiles.data(), tiles.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    FCC_CUDA_TRY(cudaMalloc(&plan->d_tc_peq, 8 * sizeof(float)));
    FCC_CUDA_TRY(cudaMemcpy(plan->d_tc_peq, peq.data(), 8 * sizeof(float), cudaMemcpyHostToDevice));
    return FCC_OK;
}

fcc_status_t launch_tc(const fcc_plan *plan, const float2 *spectra, long long T, int *idx, float *peak, float *tau,
                       float *coef, float *corr, cudaStream_t st)
{
    const fcc_plan_info_t &in = plan->info;
    if (!plan->tc_smem) return fail(FCC_ERR_UNSUPPORTED, "the tensor-core path is not available for this plan");
    if (reinterpret_cast<uintptr_t>(spectra) & 15) return fail(FCC_ERR_INVALID_ARG, "spectra not 16-byte aligned");
    TcParams prm{};
    prm.spectra = spectra;
    prm.T = T;
    prm.M = in.M;
    prm.B = in.B;
    prm.Q = in.Q;
    prm.P = in.P;
    prm.n_slots = plan->n_slots;
    prm.F = plan->tc_F;
    const long long n_tiles = (T + prm.F - 1) / prm.F;
    if (n_tiles > 0x7fffffffLL) return fail(FCC_ERR_UNSUPPORTED, "too many frames for one call");
    prm.n_tiles = (int)n_tiles;
    prm.center = in.center;
    prm.I = in.I;
    prm.KE = in.K_even;
    prm.KO = in.K_odd;
    prm.delta = (float)in.delta;
    prm.bases = plan->d_tc_bases;
    prm.peq = plan->d_tc_peq;
    prm.rbases = plan->d_tc_rbases;
    prm.npad = plan->tc_npad;
    prm.recon = plan->d_recon;
    prm.slots = plan->d_slots;
    prm.out_idx = idx;
    prm.out_peak = peak;
    prm.out_tau = tau;
    prm.out_coef = coef;
    prm.out_corr = corr;
    prm.err = plan->d_err;
    const int grid = (int)std::min<long long>(n_tiles, (long long)plan->num_sms);
    if (in.prec == FCC_PREC_BF16) return launch_tc_prec<FCC_PREC_BF16>(plan, prm, st, grid);
    return launch_tc_prec<FCC_PREC_FP16>(plan, prm, st, grid);
}

}  // namespace fcc
