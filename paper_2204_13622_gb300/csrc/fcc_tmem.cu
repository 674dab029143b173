// fcc_tmem.cu -- the FCC hot path with the Eq. 9 projection on the tcgen05
// tensor cores and its A operand written straight into tensor memory.
//
// For a microphone pair and a bin pair (f, N/2 - f), with a = R(f) and
// b = R(N/2 - f) (R = u_i u_j^*, u = X / |X|, Sec. 2 with alpha = 1), Eq. 8
// folds x_s = a + b and x_d = a - b, and Eq. 9 projects them on the cropped
// even and odd bases.  Written as one contraction over the folded bins,
//   zE.re = sum_f pe(f) (Re a + Re b),     zO.re = sum_f po(f) (Re a - Re b),
//   zE.im = sum_f pe(f) (Im a + Im b),     zO.im = sum_f po(f) (Im a - Im b),
// the fold itself goes into the B operand: the K rows (f, a) and (f, b) of B
// carry (pe, po) and (pe, -po).  The same B serves the real and the imaginary
// parts; they accumulate into two column ranges of D.  Bin N/4 is the record
// f = Q with b = 0 and no odd weight (Eq. 8; its x_d is zero).
//
// A tile is 128 TMEM lanes = 32 slots x 4 pairs; a slot is a 2x2 block of the
// pair triangle (mics {i1, i2} x {j1, j2}), the same slots as the CUDA-core
// kernel, and a tile holds F = 32 / slots-per-frame whole frames.  The four
// threads of a lane group (tcgen05.st shape 16x256b: thread t writes lanes t/4
// and t/4 + 8 of a 16-lane half, columns 2 (t % 4) + {0, 1} of every 8-column
// group) take the records f = 4h + (t % 4) of quad h; one thread holds the four
// pairs of its slot (four 16-byte loads per record for four pairs).
//
// Precision:
//   FP32: kind::tf32 with a two-term split of both operands.  The tensor core
//         reads the top 19 bits of an FP32 operand (truncation), so the raw
//         value is the high term and x - trunc(x) (exact in FP32) the low
//         term; both go into their own K groups against B = [B_hi | B_lo] in
//         N.  The result keeps about 21 bits; the split costs one bitwise AND
//         and half a packed subtraction per value.
//   BF16 / FP16: kind::f16, the cross spectra rounded once to the operand
//         type (both bins of a record packed by one conversion), FP32
//         accumulation; PHAT and cross spectra stay FP32.
//
// Roles (512 threads, persistent over tiles):
//   * warps 0-7  producers, two per TMEM lane quadrant: PHAT of the staged
//     raw frames (FP32) into folded unit-phase records in shared memory, then
//     per chunk of CH record quads the slot's cross spectra, tcgen05.st into
//     the chunk's A buffer (NBA buffers in a ring);
//   * warp 8     copy warp: one cp.async.bulk per tile into a ring of S stages;
//   * warps 9 .. 9 + NI - 1  MMA warps: chunk c of a tile goes to MMA warp
//     c % NI, which accumulates it into its own copy of D (one thread issues
//     tcgen05.mma serially; several issuing warps overlap), so the sum is
//     deterministic;
//   * warps 12-15 epilogue, one per lane quadrant, a tile behind the MMAs (two
//     D buffers): tcgen05.ld of the NI copies of their lane (one pair-frame per
//     thread), the reconstruction on the lag grid, argmax, refinement and
//     outputs as the CUDA-core kernel.
// Every wait is bounded; on expiry the kernel latches FCC_ERR_TIMEOUT, waits
// (with the full bound) for its own copies and MMAs in flight, frees its tensor
// memory and returns.
#include <algorithm>
#include <cfloat>
#include <cstdlib>
#include <cstring>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fcc_device.cuh"
#include "fcc_internal.h"

namespace fcc {
namespace {

constexpr int kTmProd = 8;        // producer warps (two per TMEM lane quadrant)
constexpr int kTmCopy = 8;        // copy warp
constexpr int kTmIss0 = 9;        // first MMA warp
constexpr int kTmMaxIss = 3;      // MMA warps at most
constexpr int kTmEpi0 = 12;       // first epilogue warp (12 % 4 == 0)
constexpr int kTmEpi = 4;         // epilogue warps
constexpr int kTmThreads = 512;
constexpr int kTmCols = 512;      // tensor memory columns allocated

// Barrier indices.
enum {
    kTbRawFull = 0,             // [kTmMaxStages]
    kTbRawEmpty = 4,            // [kTmMaxStages]
    kTbAFull = 8,               // [kTmMaxA]
    kTbAEmpty = 16,             // [kTmMaxA]
    kTbDFull = 24,              // [2]: D buffer (tile parity) complete
    kTbDEmpty = 26,             // [2]: D buffer read by the epilogue
    kTbUFree = 28,
    kTbUReady = 29,
    kTbIssDone = 30,            // [kTmMaxIss]
    kTbCount = 34
};
constexpr int kTmMaxStages = 4;
constexpr int kTmMaxA = 8;

struct TmLayout {
    size_t bar, slot, recon, btab, ubuf, raw, raw_stage, total;
};

__host__ __device__ inline TmLayout tm_layout(const TmParams &p)
{
    TmLayout L;
    size_t o = 0;
    L.bar = o;
    o += kTbCount * 8 + 16;
    o = (o + 15) & ~(size_t)15;
    L.slot = o;
    o += (size_t)p.n_slots * sizeof(Slot);
    o = (o + 15) & ~(size_t)15;
    L.recon = o;
    o += (size_t)(p.center + 1) * 4 * p.kh * sizeof(float);
    o = (o + 127) & ~(size_t)127;
    L.btab = o;
    o += (size_t)p.nq * p.bq;
    o = (o + 127) & ~(size_t)127;
    L.ubuf = o;
    o += (size_t)p.F * p.M * p.us;
    o = (o + 127) & ~(size_t)127;
    L.raw = o;
    L.raw_stage = (((size_t)p.F * p.M * p.B * 8) + 127) & ~(size_t)127;
    o += (size_t)p.S * L.raw_stage;
    L.total = o;
    return L;
}

// Records of a microphone row are stored at position f ^ 4 for microphones
// 2, 3 (mod 4), so the two slots of a quarter-warp, whose 16-byte loads cover
// records 4h .. 4h+3 of two rows, usually fall into opposite halves of the 128
// bank bytes.
__host__ __device__ __forceinline__ int tm_swz(int mic) { return (mic & 2) ? 4 : 0; }

// f32x2 -> its low TF32 term: v - trunc19(v) per element (exact in FP32).
__device__ __forceinline__ f2 tf32_lo(f2 v)
{
    float a, b;
    upk(v, a, b);
    const float ha = __uint_as_float(__float_as_uint(a) & 0xffffe000u);
    const float hb = __uint_as_float(__float_as_uint(b) & 0xffffe000u);
    return sub2(v, pk(ha, hb));
}

__device__ __forceinline__ uint32_t f2lo(f2 v) { return (uint32_t)(v & 0xffffffffull); }
__device__ __forceinline__ uint32_t f2hi(f2 v) { return (uint32_t)(v >> 32); }

// Two FP32 values (element 0 = lo, element 1 = hi) rounded to one packed 16-bit pair.
template <int PREC>
__device__ __forceinline__ uint32_t tm_pack16(f2 v)
{
    float a, b;
    upk(v, a, b);
    uint32_t r;
    if constexpr (PREC == FCC_PREC_BF16)
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
    else
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
    return r;
}

__device__ __forceinline__ void tm_st_x4(uint32_t taddr, const uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.16x256b.x4.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]));
}
__device__ __forceinline__ void tm_st_x1(uint32_t taddr, uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3)
{
    asm volatile("tcgen05.st.sync.aligned.16x256b.x1.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "r"(r0), "r"(r1),
                 "r"(r2), "r"(r3));
}

template <int KIND>  // 0: kind::tf32, 1: kind::f16
__device__ __forceinline__ void tm_mma(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, bool acc)
{
    if constexpr (KIND == 0)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
            "r"(a), "l"(bdesc), "r"(idesc), "r"((uint32_t)acc));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
            "r"(a), "l"(bdesc), "r"(idesc), "r"((uint32_t)acc));
}

__device__ __forceinline__ void tm_ld32(uint32_t taddr, float *v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tm_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// mbarrier try_wait that may suspend the thread (up to hint_ns) until the
// phase completes, so waiting warps take no issue slots.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, unsigned parity, unsigned hint_ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}
// Bounded wait on an mbarrier phase (false when `limit` cycles pass first).
__device__ bool tm_wait(uint64_t *bar, unsigned parity, long long limit)
{
    if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
        if (clock64() - t0 > limit) return false;
    }
}
// A bounded wait whose outcome is the same in every lane of the warp.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, unsigned parity, long long limit)
{
    return __all_sync(0xffffffffu, tm_wait(bar, parity, limit));
}

template <int KH, int PREC>
__global__ void __launch_bounds__(kTmThreads, 1) fcc_tm_kernel(const __grid_constant__ TmParams p)
{
    constexpr bool F32 = PREC == FCC_PREC_FP32;
    constexpr int KT = KH <= 4 ? 4 : 8;       // bases per parity in the MMA layout
    constexpr int NN = 4 * KT;                // MMA N (one D region for FP32, both for f16)
    constexpr int DW = F32 ? 8 * KT : 4 * KT; // D columns per MMA warp
    constexpr int CW = F32 ? 32 : 8;          // A columns per record quad
    extern __shared__ __align__(1024) unsigned char smem[];
    const TmLayout lay = tm_layout(p);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + lay.bar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + lay.bar + kTbCount * 8);
    Slot *slots = reinterpret_cast<Slot *>(smem + lay.slot);
    float *recon = reinterpret_cast<float *>(smem + lay.recon);
    unsigned char *ubuf = smem + lay.ubuf;
    unsigned char *raw = smem + lay.raw;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Q = p.Q, B = p.B, M = p.M;
    const int frame_bytes = M * B * 8;
    const int n_local = (p.n_tiles > (int)blockIdx.x)
                            ? (p.n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x
                            : 0;
    const int n_ch = (p.nq + p.CH - 1) / p.CH;
    const unsigned FULLM = 0xffffffffu;

    if (threadIdx.x == 0) {
        for (int s = 0; s < p.S; ++s) {
            mbar_init(&bar[kTbRawFull + s], 1);
            mbar_init(&bar[kTbRawEmpty + s], kTmProd);
        }
        for (int b = 0; b < p.NBA; ++b) {
            mbar_init(&bar[kTbAFull + b], kTmProd);
            mbar_init(&bar[kTbAEmpty + b], 1);
        }
        for (int d = 0; d < 2; ++d) {
            mbar_init(&bar[kTbDFull + d], (unsigned)p.NI);
            mbar_init(&bar[kTbDEmpty + d], kTmEpi);
        }
        mbar_init(&bar[kTbUFree], kTmProd);
        mbar_init(&bar[kTbUReady], kTmProd);
        for (int i = 0; i < kTmMaxIss; ++i) mbar_init(&bar[kTbIssDone + i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int e = threadIdx.x; e < p.n_slots; e += blockDim.x) slots[e] = p.slots[e];
    for (int e = threadIdx.x; e < (p.center + 1) * 4 * KH; e += blockDim.x) recon[e] = p.recon[e];
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(p.btab);
        uint4 *dst = reinterpret_cast<uint4 *>(smem + lay.btab);
        for (int e = threadIdx.x; e < p.nq * p.bq / 16; e += blockDim.x) dst[e] = src[e];
        uint4 *u = reinterpret_cast<uint4 *>(ubuf);  // padding records stay zero
        for (int e = threadIdx.x; e < p.F * M * p.us / 16; e += blockDim.x) u[e] = make_uint4(0, 0, 0, 0);
    }
    fence_proxy_async();
    if (warp == kTmCopy) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "n"(kTmCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t a0col = (uint32_t)(2 * p.NI * DW);  // A ring after two buffers of NI copies of D

    auto tile_frames = [&](int j, int &nf) {
        const long long f0 = ((long long)blockIdx.x + (long long)j * gridDim.x) * p.F;
        nf = (int)min((long long)p.F, p.T - f0);
        return f0;
    };

    if (warp == kTmCopy) {
        // ================= copy warp =================
        if (lane == 0) {
            int issued = 0;
            for (int j = 0; j < n_local; ++j) {
                const int s = j % p.S;
                if (!tm_wait(&bar[kTbRawEmpty + s], ((unsigned)(j / p.S) & 1u) ^ 1u, p.wait_cycles)) {
                    atomicOr(p.err, kErrTimeout);
                    break;
                }
                int nf;
                const long long f0 = tile_frames(j, nf);
                const unsigned bytes = (unsigned)nf * (unsigned)frame_bytes;
                if (p.inject && blockIdx.x == 0 && j == 0) continue;  // test hook: withhold the first copy
                mbar_arrive_expect_tx(&bar[kTbRawFull + s], bytes);
                bulk_g2s(raw + (size_t)s * lay.raw_stage,
                         reinterpret_cast<const unsigned char *>(p.spectra) + (size_t)f0 * frame_bytes, bytes,
                         &bar[kTbRawFull + s]);
                issued = j + 1;
            }
            // never retire with a copy in flight: wait (full bound) for the last copy of every stage
            for (int j = max(0, issued - p.S); j < issued; ++j) {
                if (p.inject && blockIdx.x == 0 && j == 0) continue;
                if (!tm_wait(&bar[kTbRawFull + j % p.S], (unsigned)(j / p.S) & 1u, kWaitCycles))
                    atomicOr(p.err, kErrTimeout);
            }
        }
    } else if (warp >= kTmIss0 && warp < kTmIss0 + p.NI) {
        // ================= MMA warps =================
        if (lane == 0) {
            const int iw = warp - kTmIss0;
            constexpr uint32_t fmt = F32 ? ((2u << 7) | (2u << 10))
                                         : (PREC == FCC_PREC_BF16 ? ((1u << 7) | (1u << 10)) : 0u);
            constexpr uint32_t idesc = (1u << 4) | fmt | ((uint32_t)(NN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
            const uint32_t btab = smem_u32(smem + lay.btab);
            // A buffer of the current chunk and the parity of its fill, advanced per
            // chunk.  Chunks go to the MMA warps round-robin over the whole sequence
            // of chunks (not per tile), so a warp's consecutive chunks are exactly NI
            // <= NBA apart: when it waits for fill k of a buffer, fill k - 1 has
            // landed and the parity of the wait is unambiguous.
            int b = 0;
            unsigned fpar = 0;
            int cw = 0;  // (global chunk index) % NI
            bool ok = true, any = false;
            for (int j = 0; j < n_local && ok; ++j) {
                bool first = true;
                const int db = j & 1;  // D buffer of this tile: the epilogue runs a tile behind
                const uint32_t d_re = tmem + (uint32_t)((db * p.NI + iw) * DW), d_im = d_re + 4 * KT;
                for (int c = 0; c < n_ch; ++c) {
                    const int bc = b;
                    const unsigned pc = fpar;
                    if (++b == p.NBA) {
                        b = 0;
                        fpar ^= 1u;
                    }
                    const bool mine = cw == iw;
                    if (++cw == p.NI) cw = 0;
                    if (!mine) continue;
                    if (first && !tm_wait(&bar[kTbDEmpty + db], ((unsigned)(j >> 1) & 1u) ^ 1u, p.wait_cycles)) {
                        ok = false;
                        break;
                    }
                    if (!tm_wait(&bar[kTbAFull + bc], pc, p.wait_cycles)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int nqc = min(p.CH, p.nq - c * p.CH);
                    for (int qq = 0; qq < nqc; ++qq) {
                        const int h = c * p.CH + qq;
                        const uint32_t acol = tmem + a0col + (uint32_t)((bc * p.CH + qq) * CW);
                        const uint64_t bd = umma_desc(btab + (uint32_t)(h * p.bq), 128, 256);
                        const bool acc = !(first && qq == 0);
                        if constexpr (F32) {
                            tm_mma<0>(d_re, acol, bd, idesc, acc);
                            tm_mma<0>(d_im, acol + 8, bd, idesc, acc);
                            tm_mma<0>(d_re, acol + 16, bd, idesc, true);
                            tm_mma<0>(d_im, acol + 24, bd, idesc, true);
                        } else {
                            tm_mma<1>(d_re, acol, bd, idesc, acc);
                        }
                    }
                    umma_commit(&bar[kTbAEmpty + bc]);
                    first = false;
                    any = true;
                }
                if (!ok) break;
                umma_commit(&bar[kTbDFull + db]);
            }
            if (!ok) atomicOr(p.err, kErrTimeout);
            // retire only when every MMA this warp issued has completed
            umma_commit(&bar[kTbIssDone + iw]);
            if (!tm_wait(&bar[kTbIssDone + iw], 0u, kWaitCycles)) atomicOr(p.err, kErrTimeout);
            (void)any;
        }
    } else if (warp < kTmProd) {
        // ================= producer warps =================
        const int q = warp & 3, hh = warp >> 2;
        const int rg = lane >> 2, tt = lane & 3;
        const int sidx = 8 * q + rg;                  // slot of this lane group in the tile
        const int TS = p.F * p.n_slots;
        const int fl = sidx < TS ? sidx / p.n_slots : 0;
        Slot sl{};
        if (sidx < TS) sl = slots[sidx - fl * p.n_slots];
        const int RS = Q / 32;                        // records per lane in the PHAT
        int b = 0;          // A buffer of the next chunk
        unsigned fpar = 0;  // parity of that buffer's next fill
        bool ok = true;
        for (int j = 0; j < n_local && ok; ++j) {
            int nf;
            const long long f0 = tile_frames(j, nf);
            const int s = j % p.S;
            // the unit-phase records of the previous tile are no longer read
            if (j > 0 && !warp_wait(&bar[kTbUFree], (unsigned)(j - 1) & 1u, p.wait_cycles)) {
                ok = false;
                break;
            }
            if (!warp_wait(&bar[kTbRawFull + s], (unsigned)(j / p.S) & 1u, p.wait_cycles)) {
                ok = false;
                break;
            }
            // ---- PHAT (FP32) into folded records (re f, re f', im f, im f'), f' = N/2 - f
            {
                const unsigned char *st = raw + (size_t)s * lay.raw_stage;
                bool bad = false;
                for (int R = warp; R < nf * M; R += kTmProd) {
                    const float2 *xr = reinterpret_cast<const float2 *>(st + (size_t)R * B * 8);
                    float4 *rec = reinterpret_cast<float4 *>(ubuf + (size_t)R * p.us);
                    const int sw = tm_swz(R % M);
                    // the fast form for the whole row first (independent records, so
                    // their loads overlap), then one vote: a row with a zero, tiny,
                    // huge or non-finite bin is redone in the careful form
                    bool rok = true;
#pragma unroll 4
                    for (int jj = 0; jj < RS; ++jj) {
                        const int fp = lane + 32 * jj;
                        bool o1, o2;
                        const float2 a = unit_phase_fast(xr[fp], o1);
                        const float2 b = unit_phase_fast(xr[2 * Q - fp], o2);
                        rok = rok && o1 && o2;
                        rec[fp ^ sw] = make_float4(a.x, b.x, a.y, b.y);
                    }
                    if (lane == 0) {
                        bool o;
                        const float2 c = unit_phase_fast(xr[Q], o);
                        rok = rok && o;
                        rec[Q ^ sw] = make_float4(c.x, 0.f, c.y, 0.f);
                    }
                    if (!__all_sync(FULLM, rok)) {
                        for (int jj = 0; jj < RS; ++jj) {
                            const int fp = lane + 32 * jj;
                            const float2 a = unit_phase_slow(xr[fp], bad);
                            const float2 b = unit_phase_slow(xr[2 * Q - fp], bad);
                            rec[fp ^ sw] = make_float4(a.x, b.x, a.y, b.y);
                        }
                        if (lane == 0) {
                            const float2 c = unit_phase_slow(xr[Q], bad);
                            rec[Q ^ sw] = make_float4(c.x, 0.f, c.y, 0.f);
                        }
                    }
                }
                if (__any_sync(FULLM, bad) && lane == 0) atomicOr(p.err, kErrNonFinite);
            }
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&bar[kTbRawEmpty + s]);  // the raw stage may be refilled
                mbar_arrive(&bar[kTbUReady]);
            }
            if (!warp_wait(&bar[kTbUReady], (unsigned)j & 1u, p.wait_cycles)) {
                ok = false;
                break;
            }
            // ---- this lane group's slot.  Record f = 4h + tt of a row sits at position
            // f ^ sw = 4 (h ^ (sw / 4)) + tt; chunks hold an even number of quads, so
            // the quads h of this warp all have the parity hh and each row's record
            // address is a fixed base + 64 h.
            const bool act = sidx < TS && fl < nf;
            const unsigned char *ub[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int mic = act ? sl.mic[r] : 0;
                const int s4 = tm_swz(mic) >> 2;
                ub[r] = ubuf + (size_t)(fl * M + mic) * p.us + 16 * tt + (s4 ? (hh ? -64 : 64) : 0);
            }
            // cross spectra of one record for the slot's four pairs, packed over the two
            // bins: re[q] = (Re a, Re b), im[q] = (Im a, Im b)
            auto record = [&](int h, f2 (&re)[4], f2 (&im)[4]) {
                float4 X[2], Y[2];
                if (act) {
                    X[0] = *reinterpret_cast<const float4 *>(ub[0] + 64 * h);
                    X[1] = *reinterpret_cast<const float4 *>(ub[1] + 64 * h);
                    Y[0] = *reinterpret_cast<const float4 *>(ub[2] + 64 * h);
                    Y[1] = *reinterpret_cast<const float4 *>(ub[3] + 64 * h);
                } else {
                    X[0] = X[1] = Y[0] = Y[1] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                f2 xr[2], xi[2], nxr[2], yr[2], yi[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    xr[u] = pk(X[u].x, X[u].y);
                    xi[u] = pk(X[u].z, X[u].w);
                    nxr[u] = pk(-X[u].x, -X[u].y);
                    yr[u] = pk(Y[u].x, Y[u].y);
                    yi[u] = pk(Y[u].z, Y[u].w);
                }
                // pair (ix, iy): (Re a, Re b) = xr yr + xi yi, (Im a, Im b) = xi yr - xr yi
#pragma unroll
                for (int pq = 0; pq < 4; ++pq) {
                    const int ix = pq >> 1, iy = pq & 1;
                    re[pq] = fma2(xi[ix], yi[iy], mul2(xr[ix], yr[iy]));
                    im[pq] = fma2(nxr[ix], yi[iy], mul2(xi[ix], yr[iy]));
                }
            };
            // ---- A chunks.  Per chunk a thread forms all of its records first (loads and
            // arithmetic of up to RMAX records in flight), then stores them: tcgen05.st
            // reads its source registers asynchronously, so no register it reads is
            // rewritten before the chunk's wait::st.
            constexpr int RMAX = F32 ? (KH > 4 ? 1 : 2) : 4;  // records per thread per chunk (CH <= 2 RMAX)
            constexpr int VR = F32 ? 32 : 8;       // 32-bit values per record
            for (int c = 0; c < n_ch; ++c) {
                if (!warp_wait(&bar[kTbAEmpty + b], fpar ^ 1u, p.wait_cycles)) {
                    ok = false;
                    break;
                }
                const int nqc = min(p.CH, p.nq - c * p.CH);
                uint32_t v[RMAX][VR];
#pragma unroll
                for (int r = 0; r < RMAX; ++r) {
                    const int qq = hh + 2 * r;
                    if (qq < nqc) {
                        f2 re[4], im[4];
                        record(c * p.CH + qq, re, im);
                        if constexpr (F32) {
                            // per 16-lane half hb: pairs 2 hb and 2 hb + 1; groups (Re hi, Im hi, Re lo, Im lo)
#pragma unroll
                            for (int hb = 0; hb < 2; ++hb) {
                                const int p0 = 2 * hb, p1 = 2 * hb + 1;
                                const f2 rl0 = tf32_lo(re[p0]), il0 = tf32_lo(im[p0]);
                                const f2 rl1 = tf32_lo(re[p1]), il1 = tf32_lo(im[p1]);
                                uint32_t *o = v[r] + 16 * hb;
                                o[0] = f2lo(re[p0]), o[1] = f2hi(re[p0]), o[2] = f2lo(re[p1]), o[3] = f2hi(re[p1]);
                                o[4] = f2lo(im[p0]), o[5] = f2hi(im[p0]), o[6] = f2lo(im[p1]), o[7] = f2hi(im[p1]);
                                o[8] = f2lo(rl0), o[9] = f2hi(rl0), o[10] = f2lo(rl1), o[11] = f2hi(rl1);
                                o[12] = f2lo(il0), o[13] = f2hi(il0), o[14] = f2lo(il1), o[15] = f2hi(il1);
                            }
                        } else {
#pragma unroll
                            for (int pq = 0; pq < 4; ++pq) {
                                v[r][2 * pq] = tm_pack16<PREC>(re[pq]);
                                v[r][2 * pq + 1] = tm_pack16<PREC>(im[pq]);
                            }
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < RMAX; ++r) {
                    const int qq = hh + 2 * r;
                    if (qq < nqc) {
                        const uint32_t col = tmem + a0col + (uint32_t)((b * p.CH + qq) * CW);
#pragma unroll
                        for (int hb = 0; hb < 2; ++hb) {
                            const uint32_t taddr = col + ((uint32_t)(32 * q + 16 * hb) << 16);
                            if constexpr (F32) {
                                const uint32_t *o = v[r] + 16 * hb;
                                const uint32_t rr[16] = {o[0], o[1], o[2],  o[3],  o[4],  o[5],  o[6],  o[7],
                                                         o[8], o[9], o[10], o[11], o[12], o[13], o[14], o[15]};
                                tm_st_x4(taddr, rr);
                            } else {
                                const uint32_t *o = v[r] + 4 * hb;
                                tm_st_x1(taddr, o[0], o[1], o[2], o[3]);
                            }
                        }
                    }
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar[kTbAFull + b]);
                if (++b == p.NBA) {
                    b = 0;
                    fpar ^= 1u;
                }
            }
            if (!ok) break;
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[kTbUFree]);
        }
        if (!ok && lane == 0) atomicOr(p.err, kErrTimeout);
    } else if (warp >= kTmEpi0) {
        // ================= epilogue warps =================
        const int q = warp & 3;
        const int hb = lane >> 4, i2 = (lane >> 3) & 1, rg = lane & 7;
        const int sidx = 8 * q + rg, pidx = 2 * hb + i2;
        const int TS = p.F * p.n_slots;
        const int fl = sidx < TS ? sidx / p.n_slots : 0;
        int pq = -1;
        if (sidx < TS) {
            const Slot sl = slots[sidx - fl * p.n_slots];
            pq = pidx == 0 ? sl.pair[0] : pidx == 1 ? sl.pair[1] : pidx == 2 ? sl.pair[2] : sl.pair[3];
        }
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        bool ok = true;
        for (int j = 0; j < n_local; ++j) {
            int nf;
            const long long f0 = tile_frames(j, nf);
            const int db = j & 1;
            if (!warp_wait(&bar[kTbDFull + db], (unsigned)(j >> 1) & 1u, p.wait_cycles)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float acc[DW];
#pragma unroll
            for (int e = 0; e < DW; ++e) acc[e] = 0.f;
            for (int iw = 0; iw < p.NI; ++iw) {
                float v[32];
#pragma unroll
                for (int part = 0; part < DW / 32 + (DW % 32 ? 1 : 0); ++part) {
                    const uint32_t taddr = tmem + lane_base + (uint32_t)((db * p.NI + iw) * DW + 32 * part);
                    if constexpr (DW % 32 == 0) {
                        tm_ld32(taddr, v);
#pragma unroll
                        for (int e = 0; e < 32; ++e) acc[32 * part + e] += v[e];
                    } else {
                        tm_ld16(taddr, v);
#pragma unroll
                        for (int e = 0; e < 16; ++e) acc[e] += v[e];
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[kTbDEmpty + db]);
            // coefficients in the packing of the CUDA-core kernel: zE = (sum pe Re x_s, sum pe Im x_s),
            // zO = (sum po Re x_d, sum po Im x_d)
            f2 zE[KH], zO[KH];
#pragma unroll
            for (int v = 0; v < KH; ++v) {
                if constexpr (F32) {
                    zE[v] = pk(acc[v] + acc[2 * KT + v], acc[4 * KT + v] + acc[6 * KT + v]);
                    zO[v] = pk(acc[KT + v] + acc[3 * KT + v], acc[5 * KT + v] + acc[7 * KT + v]);
                } else {
                    zE[v] = pk(acc[v], acc[2 * KT + v]);
                    zO[v] = pk(acc[KT + v], acc[3 * KT + v]);
                }
            }
            if (!(pq >= 0 && fl < nf)) continue;
            const size_t o = (size_t)(f0 + fl) * p.P + pq;
            float *corr = p.out_corr ? p.out_corr + o * p.I : nullptr;
            // the lag scan two steps at a time, each step's S and D over two
            // partial sums (four independent FMA chains of KH instead of one of
            // 2 KH); the steps are compared in increasing m as in eval_SD's scan
            float best, S, D;
            {
                f2 e = 0ull, o = 0ull;
                const float4 *g = reinterpret_cast<const float4 *>(recon);
#pragma unroll
                for (int k = 0; k < KH; ++k) {
                    const float4 w = g[k];
                    e = fma2(pk(w.x, w.y), zE[k], e);
                    o = fma2(pk(w.z, w.w), zO[k], o);
                }
                upk(add2(e, o), S, D);
            }
            best = S - D;
            int bi = p.center;
            if (corr) corr[p.center] = best;
            auto take = [&](int m, float Sm, float Dm) {
                const float ym = Sm + Dm, yp = Sm - Dm;  // y(center - m), y(center + m)
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
            int m = 1;
            for (; m + 1 <= p.center; m += 2) {
                const float4 *g0 = reinterpret_cast<const float4 *>(recon + (size_t)m * 4 * KH);
                const float4 *g1 = g0 + KH;
                f2 e0 = 0ull, o0 = 0ull, e1 = 0ull, o1 = 0ull;
#pragma unroll
                for (int k = 0; k < KH; ++k) {
                    const float4 w0 = g0[k], w1 = g1[k];
                    e0 = fma2(pk(w0.x, w0.y), zE[k], e0);
                    o0 = fma2(pk(w0.z, w0.w), zO[k], o0);
                    e1 = fma2(pk(w1.x, w1.y), zE[k], e1);
                    o1 = fma2(pk(w1.z, w1.w), zO[k], o1);
                }
                float S0, D0, S1, D1;
                upk(add2(e0, o0), S0, D0);
                upk(add2(e1, o1), S1, D1);
                take(m, S0, D0);
                take(m + 1, S1, D1);
            }
            if (m <= p.center) {
                eval_SD<KH>(recon, m, zE, zO, S, D);
                take(m, S, D);
            }
            p.out_idx[o] = bi;
            p.out_peak[o] = best;
            if (p.out_tau) {
                float off = 0.f;
                if (bi > 0 && bi < p.I - 1) {
                    // three-point parabola; the differences are exact in FP64
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
        if (!ok && lane == 0) atomicOr(p.err, kErrTimeout);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == kTmCopy)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTmCols));
}

template <int KH, int PREC>
fcc_status_t launch_tm_inst(const fcc_plan *plan, const TmParams &prm, cudaStream_t st, int grid)
{
    static bool attr_set[64] = {};
    const int dev = plan->device;
    if (!attr_set[dev & 63]) {
        cudaError_t e = cudaFuncSetAttribute(fcc_tm_kernel<KH, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             232448);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(fcc_tm_kernel)");
        attr_set[dev & 63] = true;
    }
    fcc_tm_kernel<KH, PREC><<<grid, kTmThreads, plan->tm.smem, st>>>(prm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fcc_tm_kernel launch");
    return FCC_OK;
}

template <int PREC>
fcc_status_t launch_tm_prec(const fcc_plan *plan, const TmParams &prm, cudaStream_t st, int grid)
{
    switch (plan->kh) {
    case 2: return launch_tm_inst<2, PREC>(plan, prm, st, grid);
    case 4: return launch_tm_inst<4, PREC>(plan, prm, st, grid);
    case 6: return launch_tm_inst<6, PREC>(plan, prm, st, grid);
    case 8: return launch_tm_inst<8, PREC>(plan, prm, st, grid);
    default: return fail(FCC_ERR_UNSUPPORTED, "more than 8 bases of one parity");
    }
}

TmParams tm_params_geometry(const fcc_plan *plan)
{
    const fcc_plan_info_t &in = plan->info;
    TmParams p{};
    p.M = in.M;
    p.B = in.B;
    p.Q = in.Q;
    p.P = in.P;
    p.n_slots = plan->n_slots;
    p.center = in.center;
    p.kh = plan->kh;
    p.nq = in.Q / 4 + 1;
    const int KT = plan->kh <= 4 ? 4 : 8;
    p.bq = 4 * KT * 32;
    p.us = ((in.Q + 4 + 7) / 8) * 8 * 16;
    p.F = plan->tm.F;
    p.S = plan->tm.S;
    p.NI = plan->tm.NI;
    p.NBA = plan->tm.NBA;
    p.CH = plan->tm.CH;
    return p;
}

}  // namespace

// Host side: whether the tensor-memory path applies, its geometry and its B
// table (K-major core matrices, one block of 8 K rows x 4 KT columns per record
// quad; K row (t, c) of quad h is record f = 4h + t, c = a / b for FP32, and
// (Re a, Re b, Im a, Im b) for the 16-bit forms).
fcc_status_t prepare_tm(fcc_plan *plan)
{
    const fcc_plan_info_t &in = plan->info;
    plan->tm = TmGeometry{};
    if (in.form != FCC_FORM_FOLDED) return fail(FCC_ERR_UNSUPPORTED, "the tensor-memory path takes folded plans");
    if (in.Q < 32 || in.Q > 256) return fail(FCC_ERR_UNSUPPORTED, "the tensor-memory path needs 128 <= N <= 1024");
    if (plan->n_slots > 32) return fail(FCC_ERR_UNSUPPORTED, "the tensor-memory path needs M <= 16");
    if (!plan->kh) return fail(FCC_ERR_UNSUPPORTED, "more than 8 bases of one parity");
    if ((in.M * in.B * 8) % 16) return fail(FCC_ERR_UNSUPPORTED, "the tensor-memory path needs an even number of mics");
    const bool f32 = in.prec == FCC_PREC_FP32;
    const int KT = plan->kh <= 4 ? 4 : 8;
    const int DW = f32 ? 8 * KT : 4 * KT, CW = f32 ? 32 : 8;
    const int nq = in.Q / 4 + 1;
    int smem_max = 0;
    FCC_CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, plan->device));
    smem_max = std::min(smem_max, 232448);
    // tensor memory: NI copies of D and a ring of NBA buffers of CH quads
    TmGeometry g{};
    bool found = false;
    const char *ei = getenv("FCC_TM_ISSUERS");
    const int want_ni = ei ? atoi(ei) : 0;
    const char *eb = getenv("FCC_TM_NBA"), *ec = getenv("FCC_TM_CH");
    const int want_nba = eb ? atoi(eb) : 0, want_ch = ec ? atoi(ec) : 0;
    for (int NI = kTmMaxIss; NI >= 1 && !found; --NI) {
        if (want_ni && NI != want_ni) continue;
        const int avail = kTmCols - 2 * NI * DW;
        // NBA >= NI: the MMA warp of chunk g waits for fill g / NBA of its buffer only
        // after finishing chunk g - NI, so fill g / NBA - 1 has completed and the
        // parity of the wait is unambiguous
        for (int NBA = std::min(kTmMaxA, NI + 1); NBA >= std::max(2, NI) && !found; --NBA) {
            if (want_nba && NBA != want_nba) continue;
            // an even number of quads per chunk: the two producer warps of a lane
            // quadrant take the even and the odd quads
            int CH = std::min(avail / (NBA * CW), f32 ? (plan->kh > 4 ? 2 : 4) : 8) & ~1;
            if (want_ch) {
                if (want_ch > CH || (want_ch & 1)) continue;
                CH = want_ch;
            }
            if (CH < 2) continue;
            if ((nq + CH - 1) / CH < NI) continue;
            g.NI = NI;
            g.NBA = NBA;
            g.CH = CH;
            found = true;
        }
    }
    if (!found) return fail(FCC_ERR_UNSUPPORTED, "tensor memory too small for this plan");
    // shared memory: F frames per tile (F * slots <= 32), S raw stages
    TmParams p{};
    p.M = in.M;
    p.B = in.B;
    p.Q = in.Q;
    p.n_slots = plan->n_slots;
    p.center = in.center;
    p.kh = plan->kh;
    p.nq = nq;
    p.bq = 4 * KT * 32;
    p.us = ((in.Q + 4 + 7) / 8) * 8 * 16;
    bool fit = false;
    for (int F = std::max(1, 32 / plan->n_slots); F >= 1 && !fit; --F) {
        for (int S = 2; S >= 1 && !fit; --S) {
            p.F = F;
            p.S = S;
            const TmLayout L = tm_layout(p);
            if (L.total <= (size_t)smem_max) {
                g.F = F;
                g.S = S;
                g.smem = L.total;
                fit = true;
            }
        }
    }
    if (!fit) return fail(FCC_ERR_UNSUPPORTED, "frame too large for the tensor-memory path");
    // B table
    const int Q = in.Q, KE = in.K_even, KO = in.K_odd, NN = 4 * KT;
    std::vector<unsigned char> tab((size_t)nq * p.bq, 0);
    auto pe = [&](int v, int f, int c) -> double {
        if (v >= KE || f > Q || (f == Q && c == 1)) return 0.0;
        return plan->Pe[(size_t)v * (Q + 1) + f];
    };
    auto po = [&](int v, int f, int c) -> double {
        if (v >= KO || f >= Q) return 0.0;
        const double w = plan->Po[(size_t)v * Q + f];
        return c == 1 ? -w : w;
    };
    for (int h = 0; h < nq; ++h)
        for (int k = 0; k < (f32 ? 8 : 16); ++k)
            for (int n = 0; n < NN; ++n) {
                const int nc = n / 8, r = n % 8;
                unsigned char *blk = tab.data() + (size_t)h * p.bq + nc * 256 + r * 16;
                if (f32) {
                    const int t = k / 2, c = k % 2, f = 4 * h + t;
                    const int part = n / KT, v = n % KT;
                    const double w = (part & 1) ? po(v, f, c) : pe(v, f, c);
                    float hi = (float)w;
                    uint32_t hb;
                    std::memcpy(&hb, &hi, 4);
                    hb &= 0xffffe000u;
                    std::memcpy(&hi, &hb, 4);
                    const float lo = (float)(w - (double)hi);
                    const float val = part < 2 ? hi : lo;
                    std::memcpy(blk + (k / 4) * 128 + (k % 4) * 4, &val, 4);
                } else {
                    const int t = k / 4, c4 = k % 4, f = 4 * h + t;
                    const int region = n / (2 * KT), part = (n / KT) & 1, v = n % KT;
                    double w = 0.0;
                    if (region == (c4 >> 1)) w = part ? po(v, f, c4 & 1) : pe(v, f, c4 & 1);
                    uint16_t bits;
                    if (in.prec == FCC_PREC_BF16) {
                        __nv_bfloat16 x = __float2bfloat16_rn((float)w);
                        std::memcpy(&bits, &x, 2);
                    } else {
                        __half x = __float2half_rn((float)w);
                        std::memcpy(&bits, &x, 2);
                    }
                    std::memcpy(blk + (k / 8) * 128 + (k % 8) * 2, &bits, 2);
                }
            }
    void *d = nullptr;
    cudaError_t e = dev_alloc(&d, tab.size());
    if (e == cudaSuccess) e = cudaMemcpy(d, tab.data(), tab.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "tensor-memory path tables");
    }
    cudaFree(plan->d_tm_btab);
    plan->d_tm_btab = d;
    plan->tm = g;
    if (debug_enabled())
        fprintf(stderr, "[fcc] tmem path: F=%d S=%d NI=%d NBA=%d CH=%d smem=%zu\n", g.F, g.S, g.NI, g.NBA, g.CH,
                g.smem);
    return FCC_OK;
}

fcc_status_t launch_tm(const fcc_plan *plan, const float2 *spectra, long long T, int *idx, float *peak, float *tau,
                       float *coef, float *corr, cudaStream_t st)
{
    const fcc_plan_info_t &in = plan->info;
    if (!plan->tm.smem) return fail(FCC_ERR_UNSUPPORTED, "the tensor-memory path is not available for this plan");
    if (reinterpret_cast<uintptr_t>(spectra) & 15) return fail(FCC_ERR_INVALID_ARG, "spectra not 16-byte aligned");
    TmParams prm = tm_params_geometry(plan);
    prm.spectra = spectra;
    prm.T = T;
    const long long n_tiles = (T + prm.F - 1) / prm.F;
    if (n_tiles > 0x7fffffffLL) return fail(FCC_ERR_UNSUPPORTED, "too many frames for one call");
    prm.n_tiles = (int)n_tiles;
    prm.I = in.I;
    prm.KE = in.K_even;
    prm.KO = in.K_odd;
    prm.delta = (float)in.delta;
    prm.btab = plan->d_tm_btab;
    prm.recon = plan->d_recon;
    prm.slots = plan->d_slots;
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
    if (T == 0) return FCC_OK;
    const int grid = (int)std::min<long long>(n_tiles, (long long)plan->num_sms);
    switch (in.prec) {
    case FCC_PREC_FP32: return launch_tm_prec<FCC_PREC_FP32>(plan, prm, st, grid);
    case FCC_PREC_BF16: return launch_tm_prec<FCC_PREC_BF16>(plan, prm, st, grid);
    default: return launch_tm_prec<FCC_PREC_FP16>(plan, prm, st, grid);
    }
}

}  // namespace fcc
