// fcc_device.cuh -- device helpers shared by the FCC kernels (one copy per
// translation unit): packed FP32 pairs, mbarrier / bulk-copy primitives with
// bounded waits, the phase transform, the bank swizzle of the folded records
// and the lag-grid reconstruction.
#pragma once

#include <cfloat>
#include <cstdint>
#include <cuda_fp16.h>

namespace fcc {
namespace {

constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz


// ---- packed FP32 pairs (f32x2 register pairs)
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ---- mbarrier / bulk copy
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
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
// try_wait that may suspend the thread until the phase completes or about
// hint_ns pass, so a waiting warp takes no issue slots meanwhile.
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t *bar, unsigned parity, unsigned hint_ns)
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
// Bounded wait on an mbarrier phase; false if it did not complete in time.
__device__ bool mbar_wait(uint64_t *bar, unsigned parity, long long limit = kWaitCycles)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try_wait_hint(bar, parity, 2000u)) return true;
        if (clock64() - t0 > limit) return false;
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
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// u = x / |x|.  Fast path for |x|^2 in the normal FP32 range; `ok` reports
// whether it applied (callers take unit_phase_slow, warp-uniformly, otherwise).
__device__ __forceinline__ float2 unit_phase_fast(float2 x, bool &ok)
{
    const float s = fmaf(x.x, x.x, x.y * x.y);
    ok = (s >= FLT_MIN) && (s <= FLT_MAX);
    const float r = rsqrtf(s);
    float a, b;
    upk(mul2(pk(x.x, x.y), pk(r, r)), a, b);
    return make_float2(a, b);
}
// u = x / |x| with u = 0 for x = 0; rescaled for |x|^2 outside the normal FP32
// range; flags NaN / Inf (u = 0).
__device__ __noinline__ float2 unit_phase_slow(float2 x, bool &bad)
{
    const float s = fmaf(x.x, x.x, x.y * x.y);
    if (s >= FLT_MIN && s <= FLT_MAX) {
        const float r = rsqrtf(s);
        return make_float2(x.x * r, x.y * r);
    }
    if (!(fabsf(x.x) <= FLT_MAX) || !(fabsf(x.y) <= FLT_MAX)) {
        bad = true;
        return make_float2(0.f, 0.f);
    }
    const float m = fmaxf(fabsf(x.x), fabsf(x.y));
    if (m == 0.f) return make_float2(0.f, 0.f);
    const float a = x.x / m, b = x.y / m;
    const float r = rsqrtf(fmaf(a, a, b * b));
    return make_float2(a * r, b * r);
}

// Records of rows R = 2, 4, 6 (mod 8) are stored with bit 2 of their index
// flipped.  Row R's record 0 sits in 16-byte bank group ceil(R/2) mod 8; with the
// flip, the 8 rows of a frame at one bin pair fall into 8 different bank groups,
// so a quarter-warp reading one bin pair of several rows is conflict-free.
__device__ __forceinline__ int rec_swz(int R, int Q) { return (Q >= 8 && !(R & 1) && (R & 7)) ? 4 : 0; }

// S(m) and D(m) for tau = m / den >= 0 from the packed coefficients:
// y(center + m) = S - D, y(center - m) = S + D.  Table row m holds, per k,
// (gSe, gDe, gSo, gDo), matching the packs zE[k] = (Re z_e, Im z_e) and
// zO[k] = (Re z_o, Im z_o).
template <int KH>
__device__ __forceinline__ void eval_SD(const float *recon, int m, const f2 *zE, const f2 *zO, float &S, float &D)
{
    const float4 *g = reinterpret_cast<const float4 *>(recon + (size_t)m * 4 * KH);
    f2 sd = 0ull;
#pragma unroll
    for (int k = 0; k < KH; ++k) {
        const float4 v = g[k];
        sd = fma2(pk(v.x, v.y), zE[k], sd);
        sd = fma2(pk(v.z, v.w), zO[k], sd);
    }
    upk(sd, S, D);
}

template <int KH>
__device__ __forceinline__ float y_at(const float *recon, int center, int i, const f2 *zE, const f2 *zO)
{
    const int m = i >= center ? i - center : center - i;
    float S, D;
    eval_SD<KH>(recon, m, zE, zO, S, D);
    return i >= center ? S - D : S + D;
}

// ---- tcgen05 (5th-generation tensor cores, tensor memory)
// Shared-memory matrix descriptor: K-major, no swizzle, 8-row x 16-byte core
// matrices; lbo = byte stride between core matrices along K, sbo = along M/N.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t idesc, bool acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(da), "l"(db), "r"(idesc), "r"((uint32_t)acc));
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
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

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
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

// tcgen05.ld without its wait: the values may be used only after tmem_wait_ld.
__device__ __forceinline__ void tmem_ld16_nw(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Four 32-bit columns of this thread's tensor-memory lane, without the wait.
__device__ __forceinline__ void tmem_ld4_nw(uint32_t taddr, float (&v)[4])
{
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = __uint_as_float(r[j]);
}

// tmem_wait_ld for two four-column loads.
__device__ __forceinline__ void tmem_wait_ld4(float (&a)[4], float (&b)[4])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(a[0]), "+f"(a[1]), "+f"(a[2]), "+f"(a[3]), "+f"(b[0]), "+f"(b[1]), "+f"(b[2]), "+f"(b[3])
                 :
                 : "memory");
}

// Waits for this thread's tcgen05.ld; the loaded arrays pass through the wait so
// that no use of them is scheduled before it.
__device__ __forceinline__ void tmem_wait_ld(float (&a)[16], float (&b)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(a[0]), "+f"(a[1]), "+f"(a[2]), "+f"(a[3]), "+f"(a[4]), "+f"(a[5]), "+f"(a[6]), "+f"(a[7]),
                   "+f"(a[8]), "+f"(a[9]), "+f"(a[10]), "+f"(a[11]), "+f"(a[12]), "+f"(a[13]), "+f"(a[14]), "+f"(a[15]),
                   "+f"(b[0]), "+f"(b[1]), "+f"(b[2]), "+f"(b[3]), "+f"(b[4]), "+f"(b[5]), "+f"(b[6]), "+f"(b[7]),
                   "+f"(b[8]), "+f"(b[9]), "+f"(b[10]), "+f"(b[11]), "+f"(b[12]), "+f"(b[13]), "+f"(b[14]), "+f"(b[15])
                 :
                 : "memory");
}

// Two FP32 values rounded to one packed FP16 pair (element 0 in the low half).
__device__ __forceinline__ uint32_t f16x2(float e0, float e1)
{
    uint32_t r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(e1), "f"(e0));
    return r;
}
__device__ __forceinline__ float lo16(uint32_t v) { return __half2float(__ushort_as_half((unsigned short)(v & 0xffffu))); }
__device__ __forceinline__ float hi16(uint32_t v) { return __half2float(__ushort_as_half((unsigned short)(v >> 16))); }

// Eight 32-bit columns of this thread's tensor-memory lane.
__device__ __forceinline__ void st8(uint32_t taddr, const uint32_t *r)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
                 "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

// D (tensor memory) += A (tensor memory, FP16) x B (shared-memory descriptor, FP16).
__device__ __forceinline__ void mma_f16_ta(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, bool acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
        "r"(a), "l"(bdesc), "r"(idesc), "r"((uint32_t)acc));
}

}  // namespace
}  // namespace fcc
