// fcc_device.cuh -- device helpers shared by the FCC kernels (one copy per
// translation unit): packed FP32 pairs, mbarrier / bulk-copy primitives with
// bounded waits, the phase transform, the bank swizzle of the folded records
// and the lag-grid reconstruction.
#pragma once

#include <cfloat>
#include <cstdint>

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
// Bounded wait on an mbarrier phase; false if it did not complete in time.
__device__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
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
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// u = x / |x|.  Fast path for |x|^2 in the normal FP32 range; `ok` reports
// whether it applied (callers take unit_phase_slow, warp-uniformly, otherwise).
__device__ __forceinline__ float2 unit_phase_fast(float2 x, bool &ok)
{
    const float s = fmaf(x.x, x.x, x.y * x.y);
    ok = (s >= FLT_MIN) && (s <= FLT_MAX);
    const float r = rsqrtf(s);
    return make_float2(x.x * r, x.y * r);
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

}  // namespace
}  // namespace fcc
