// fcc_fp32.cu -- the FP32 FCC hot path for sm_103a.
//
// One persistent kernel.  A CTA holds G groups of GW warps; every group owns S/G
// stages of a shared-memory ring and streams its own frame tiles through them
// (tile k of the CTA belongs to group k % G and lives in stage k % S):
//   1. stage    : one cp.async.bulk per tile (F whole frames, contiguous
//                 [F][M][B] complex64), completed on the stage's mbarrier.  The
//                 group issues the copy of its next tile into a stage as soon as
//                 its own main loop has left it, so the copy overlaps the
//                 group's reduction and reconstruction.  All waits are bounded.
//   2. PHAT +   : each microphone row is normalised, u = X / |X| (0 for X = 0)
//      re-lay     (Sec. 2, eq. 1 with alpha = 1: X_i X_j^* / |X_i X_j^*| =
//                 u_i u_j^*, so M instead of P reciprocal square roots per bin),
//                 and rewritten in place in "folded" order: the 16-byte record fp
//                 holds (u(fp), u(N/2 - fp)) for fp < N/4 -- the two bins that
//                 Eq. 8 adds and subtracts -- and the lone bin N/4 sits at one
//                 end of the row.  Rows at odd positions are shifted by 8 bytes
//                 so that every record is 16-byte aligned while each row stays
//                 inside its own bytes (N/2 + 1 is odd).
//   3. fold +   : a lane owns a 2x2 block of the pair triangle (mics {i1,i2} x
//      project    {j1,j2}: 4 pairs from 4 rows) and one chunk of the bin-pair
//                 axis.  Per record it forms the 4 x 2 cross spectra in
//                 registers, folds them into x_s / x_d (Eq. 8) with packed FP32
//                 adds, and accumulates (Re, Im) x_s against the even cropped
//                 bases and (Re, Im) x_d against the odd ones (Eqs. 7, 9) with
//                 packed FFMA2.  No pair spectrum leaves registers.
//   4. reduce   : the C chunk lanes of a slot reduce-scatter their partial
//                 projections with warp shuffles; lane q keeps pair q.
//   5. output   : y(tau) on the lag grid from the 2K coefficients -- the grid is
//                 symmetric, so one pass over tau >= 0 gives y(tau) and y(-tau)
//                 -- argmax (lowest index wins ties), peak, and the three-point
//                 quadratic refinement (differences formed exactly in FP64).
// HBM traffic is the spectra read once plus the per-pair results.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "fcc_device.cuh"
#include "fcc_internal.h"

#include "fcc_fp32_tiles.cuh"

namespace fcc {
namespace {

template <int KH, int RS>
__global__ void __launch_bounds__(max_compute_warps(KH) * 32, 1) fcc_fp32_kernel(const __grid_constant__ Fp32Params p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int n_local = (p.n_tiles > (int)blockIdx.x)
                            ? (p.n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x
                            : 0;
    fp32_tiles<KH, RS, false, true>(p, smem, blockIdx.x, gridDim.x, n_local);
}

// Batched form: many plans of one (KH, RS) class in one persistent launch.  A
// CTA takes jobs (one plan, a run of its tiles) from a shared counter in the
// host's order (largest first); per job it copies the plan's parameters into a
// shared-memory header, runs the same tile pipeline, then invalidates the
// job's barriers so the next job can lay out its own ring.
template <int KH, int RS>
__global__ void __launch_bounds__(max_compute_warps(KH) * 32, 1) fcc_fp32_batch_kernel(const __grid_constant__ BatchParams bp)
{
    extern __shared__ __align__(128) unsigned char smem[];
    Fp32Params *hdr = reinterpret_cast<Fp32Params *>(smem);
    int *s_job = reinterpret_cast<int *>(smem + kBatchHeaderBytes - 8);
    unsigned char *body = smem + kBatchHeaderBytes;
    for (;;) {
        if (threadIdx.x == 0) *s_job = atomicAdd(bp.counter, 1);
        __syncthreads();
        const int j = *s_job;
        if (j >= bp.n_jobs) break;
        const BatchJob job = bp.jobs[j];
        {
            const int *src = reinterpret_cast<const int *>(bp.arrays + job.array);
            int *dst = reinterpret_cast<int *>(hdr);
            for (int e = threadIdx.x; e < (int)(sizeof(Fp32Params) / sizeof(int)); e += blockDim.x) dst[e] = src[e];
        }
        __syncthreads();
        fp32_tiles<KH, RS, false>(*hdr, body, job.tile0, 1, job.n_tiles);
        __syncthreads();
        if (threadIdx.x == 0) {
            uint64_t *bars = reinterpret_cast<uint64_t *>(body);
            for (int s = 0; s < 3 * hdr->S; ++s) mbar_inval(&bars[s]);
        }
    }
}

template <int KH, int RS>
fcc_status_t launch_inst(const fcc_plan *plan, const Fp32Params &prm, cudaStream_t st, int grid, size_t smem)
{
    static bool attr_set[64] = {};
    const int dev = plan->device;
    if (!attr_set[dev & 63]) {
        cudaError_t e = cudaFuncSetAttribute(fcc_fp32_kernel<KH, RS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             232448);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(fcc_fp32_kernel)");
        attr_set[dev & 63] = true;
    }
    fcc_fp32_kernel<KH, RS><<<grid, prm.G * prm.GW * 32, smem, st>>>(prm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fcc_fp32_kernel launch");
    return FCC_OK;
}

template <int KH>
fcc_status_t launch_kh(const fcc_plan *plan, const Fp32Params &prm, cudaStream_t st, int grid, size_t smem)
{
    const int rs = prm.Q <= 32 ? 1 : prm.Q / 32;
    switch (rs) {
    case 1: return launch_inst<KH, 1>(plan, prm, st, grid, smem);
    case 2: return launch_inst<KH, 2>(plan, prm, st, grid, smem);
    case 4: return launch_inst<KH, 4>(plan, prm, st, grid, smem);
    case 8: return launch_inst<KH, 8>(plan, prm, st, grid, smem);
    default: return fail(FCC_ERR_UNSUPPORTED, "the FP32 kernel needs N <= 1024");
    }
}

}  // namespace

// Every geometry that fits: chunks per slot (C), warps per group (GW), groups
// (G), frames per stage (F) and the ring depth (S = G * stages per group), best
// heuristic score first.  Each stage is only ever filled for, and released by,
// one group, so every group sees a plain single-consumer ring and a phase parity
// can never be stale.  The shared-memory budget leaves room for the batched
// kernel's header, so one geometry serves both launch forms.
fcc_status_t fp32_candidates(const fcc_plan *plan, std::vector<Fp32Geometry> &out, int max_warps)
{
    out.clear();
    const fcc_plan_info_t &in = plan->info;
    const int kh = plan->kh;
    const int n_slots = plan->n_slots;
    const int frame_bytes = in.M * in.B * 8;
    if (in.Q > 32 * kMaxRowSlots || kh == 0) return FCC_OK;  // N > 1024: the FP32 kernel is not used
    int smem_max = 0;
    FCC_CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, plan->device));
    smem_max = std::min(smem_max, 232448) - kBatchHeaderBytes;
    // basis row, padded to an odd number of 16-byte units: KH even then KH odd
    // weights (folded), or 2 KH float4 of cosine / sine weights (split form)
    const int BS = in.form == FCC_FORM_REIM_SPLIT ? 4 * (2 * kh + 1) : ((2 * kh / 4) % 2 == 0) ? 2 * kh + 4 : 2 * kh;
    const int maxw = max_warps > 0 ? std::min(max_warps, max_compute_warps(kh)) : max_compute_warps(kh);
    std::vector<std::pair<double, Fp32Geometry>> scored;
    for (int C = 4; C <= 32 && C <= in.Q; C <<= 1) {
        const int SB = 32 / C;
        const int nb = (n_slots + SB - 1) / SB;
        const double util = (double)n_slots / (nb * SB);
        for (int F = 1; nb * F <= maxw; ++F) {
            const int GW = nb * F;
            for (int G = maxw / GW; G >= 1; --G) {
                for (int Sg = 2; Sg >= 1; --Sg) {
                    const int S = G * Sg;
                    const SmemLayout L = smem_layout(S, n_slots, in.Q, kh, C, BS, in.center, F, frame_bytes);
                    if (L.total > (size_t)smem_max) continue;
                    // resident warps first (measured on the 8-mic circle: 12 warps of
                    // one frame each beat 6 pairs of warps with double-buffered
                    // stages by 1.4x); fewer chunks mean a shorter shuffle
                    // reduction; a second stage per group only breaks ties
                    const double score =
                        util * (G * GW) * (1.0 - 0.1 * std::log2((double)C / 4.0)) + (Sg >= 2 ? 0.01 : 0.0);
                    scored.push_back({score, Fp32Geometry{C, SB, nb * 32, GW, G, F, S, BS, L.total}});
                }
            }
        }
    }
    std::stable_sort(scored.begin(), scored.end(),
                     [](const auto &a, const auto &b) { return a.first > b.first; });
    for (auto &e : scored) out.push_back(e.second);
    return FCC_OK;
}

// The heuristic choice (first candidate); FCC_FP32_GROUPS /
// FCC_FP32_STAGES_PER_GROUP pin G and S/G (tuning only).
fcc_status_t choose_fp32_geometry(fcc_plan *plan)
{
    std::vector<Fp32Geometry> cand;
    fcc_status_t st = fp32_candidates(plan, cand);
    if (st != FCC_OK) return st;
    const fcc_plan_info_t &in = plan->info;
    if (in.Q > 32 * kMaxRowSlots || plan->kh == 0) return FCC_OK;
    const char *eg = getenv("FCC_FP32_GROUPS");
    const char *es = getenv("FCC_FP32_STAGES_PER_GROUP");
    const int want_g = eg ? atoi(eg) : 0, want_sg = es ? atoi(es) : 0;
    for (const Fp32Geometry &g : cand) {
        if (want_g && g.G != want_g) continue;
        if (want_sg && g.S / g.G != want_sg) continue;
        plan->geo = g;
        return FCC_OK;
    }
    return fail(FCC_ERR_UNSUPPORTED, "frame too large for the shared-memory ring");
}

// Kernel parameters of one call of the plan (geometry and tables from the plan).
Fp32Params make_fp32_params(const fcc_plan *plan, const float2 *spectra, long long T, int *idx, float *peak,
                            float *tau, float *coef, float *corr, unsigned *err)
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
    prm.SB = g.SB;
    prm.BS = g.BS;
    prm.lanes_frame = g.lanes_frame;
    prm.GW = g.GW;
    prm.G = g.G;
    prm.F = g.F;
    prm.S = g.S;
    prm.n_tiles = (int)std::min<long long>((T + g.F - 1) / g.F, 0x7fffffffLL);
    prm.frame_floats = in.M * in.B * 2;
    const size_t frame_bytes = (size_t)in.M * in.B * 8;
    prm.bulk = (frame_bytes % 16 == 0) && ((reinterpret_cast<uintptr_t>(spectra) & 15) == 0);
    prm.center = in.center;
    prm.I = in.I;
    prm.KE = in.K_even;
    prm.KO = in.K_odd;
    prm.delta = (float)in.delta;
    prm.basis = plan->d_basis;
    prm.recon = plan->d_recon;
    prm.slots = plan->d_slots;
    prm.out_idx = idx;
    prm.out_peak = peak;
    prm.out_tau = tau;
    prm.out_coef = coef;
    prm.out_corr = corr;
    prm.err = err;
    DebugHooks &dh = debug_hooks();
    prm.wait_cycles = dh.wait_cycles;
    prm.inject = 0;
    if (dh.withhold_copies > 0) {
        --dh.withhold_copies;
        prm.inject = 1;
    }
    return prm;
}

// Tensor-core lag grid of the FP32 kernel (fcc_fp32_tiles.cuh): the weights of
// lag steps m = 1 .. center, rounded up to a multiple of 32 rows, as three-term
// FP16 split tables, scaled by a power of two that puts the largest |weight| in
// [2^14, 2^15).  Built for folded plans with 6 or 8 bases per parity (the kernel
// instances that carry the tensor-core code) and at least 32 lag steps each way;
// FCC_FP32_MMA_RECON=0 leaves them out (the CUDA-core scan throughout).
fcc_status_t prepare_fp32_mma(fcc_plan *plan)
{
    const fcc_plan_info_t &in = plan->info;
    const char *env = getenv("FCC_FP32_MMA_RECON");
    if (env && atoi(env) == 0) return FCC_OK;
    if (in.form != FCC_FORM_FOLDED || plan->kh < 6 || in.center < 32) return FCC_OK;
    const int npad = (in.center + 31) / 32 * 32;
    if (npad > 256) return FCC_OK;
    double wmax = 0.0;
    for (int m = 1; m <= in.center; ++m) {
        const int i = in.center + m;
        const double ang = M_PI * 0.5 * (double)m / (double)in.den;
        const double a = std::fabs(std::cos(ang)), b = std::fabs(std::sin(ang));
        const double ab = 2.0 * std::max(a, b);
        for (int k = 0; k < in.K_even; ++k) wmax = std::max(wmax, ab * std::fabs(plan->Ue[(size_t)i * in.K_even + k]));
        for (int k = 0; k < in.K_odd; ++k) wmax = std::max(wmax, ab * std::fabs(plan->Uo[(size_t)i * in.K_odd + k]));
    }
    if (!(wmax > 0.0)) return FCC_OK;
    int ex = 0;
    std::frexp(wmax, &ex);  // wmax in [2^(ex-1), 2^ex)
    const int shift = 15 - ex;
    if (shift < -20 || shift > 20) return FCC_OK;
    const std::vector<uint16_t> rt = recon_tables_f16(plan, npad, 1, shift, kMmaParts);
    FCC_CUDA_TRY(dev_alloc(&plan->d_fp32_rbases, rt.size() * sizeof(uint16_t)));
    FCC_CUDA_TRY(cudaMemcpy(plan->d_fp32_rbases, rt.data(), rt.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    plan->fp32_npad = npad;
    plan->fp32_rshift = shift;
    return FCC_OK;
}

fcc_status_t launch_fp32(const fcc_plan *plan, const float2 *spectra, long long T, int *idx, float *peak,
                         float *tau, float *coef, float *corr, cudaStream_t st)
{
    const Fp32Geometry &g = plan->geo;
    if (g.G == 0) return fail(FCC_ERR_UNSUPPORTED, "the FP32 kernel needs N <= 1024");
    const long long n_tiles = (T + g.F - 1) / g.F;
    if (n_tiles > 0x7fffffffLL) return fail(FCC_ERR_UNSUPPORTED, "too many frames for one call");
    if (plan->info.form == FCC_FORM_REIM_SPLIT && coef)
        return fail(FCC_ERR_UNSUPPORTED, "the split form has no coefficient output");
    Fp32Params prm = make_fp32_params(plan, spectra, T, idx, peak, tau, coef, corr, plan->d_err);
    const int grid = (int)std::min<long long>(n_tiles, (long long)plan->num_sms);
    if (plan->info.form == FCC_FORM_REIM_SPLIT) return launch_fp32_reim(plan, prm, st, grid);
    // the tensor-core lag grid wants one pair per lane (C = 4), groups of at most
    // four warps (distinct tensor-memory row quadrants), every group's A (48),
    // S and D columns inside 512 (64 + 2 npad each), and its tables and barriers
    // behind the ring
    size_t smem = g.smem_bytes;
    const int npad = plan->fp32_npad;
    const size_t extra = (size_t)kMmaHeader + (size_t)2 * kMmaParts * npad * 32;
    if (plan->d_fp32_rbases && g.C == 4 && g.GW <= 4 && g.G * (64 + 2 * npad) <= 512 &&
        g.smem_bytes + extra <= 232448) {
        prm.rbases = plan->d_fp32_rbases;
        prm.npad = npad;
        prm.rshift = plan->fp32_rshift;
        smem += extra;
    }
    switch (plan->kh) {
    case 2: return launch_kh<2>(plan, prm, st, grid, smem);
    case 4: return launch_kh<4>(plan, prm, st, grid, smem);
    case 6: return launch_kh<6>(plan, prm, st, grid, smem);
    case 8: return launch_kh<8>(plan, prm, st, grid, smem);
    default: return fail(FCC_ERR_UNSUPPORTED, "more than 8 bases of one parity");
    }
}

int fp32_threads(int kh) { return max_compute_warps(kh) * 32; }

namespace {
template <int KH, int RS>
fcc_status_t launch_batch_inst(const BatchParams &bp, int grid, size_t smem, cudaStream_t st)
{
    if (grid == 0) {  // prepare only: raise the shared-memory limit (not capturable)
        cudaError_t e = cudaFuncSetAttribute(fcc_fp32_batch_kernel<KH, RS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
        return e == cudaSuccess ? FCC_OK : cuda_fail(e, "cudaFuncSetAttribute(fcc_fp32_batch_kernel)");
    }
    fcc_fp32_batch_kernel<KH, RS><<<grid, max_compute_warps(KH) * 32, smem, st>>>(bp);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FCC_OK : cuda_fail(e, "fcc_fp32_batch_kernel launch");
}

template <int KH>
fcc_status_t launch_batch_kh(int rs, const BatchParams &bp, int grid, size_t smem, cudaStream_t st)
{
    switch (rs) {
    case 1: return launch_batch_inst<KH, 1>(bp, grid, smem, st);
    case 2: return launch_batch_inst<KH, 2>(bp, grid, smem, st);
    case 4: return launch_batch_inst<KH, 4>(bp, grid, smem, st);
    case 8: return launch_batch_inst<KH, 8>(bp, grid, smem, st);
    default: return fail(FCC_ERR_UNSUPPORTED, "the FP32 kernel needs N <= 1024");
    }
}
}  // namespace

// One persistent launch of the batched kernel for the (kh, rs) class.  `smem` =
// kBatchHeaderBytes + the largest layout of the class's plans.  grid = 0 only
// prepares the kernel (call once per device before capturing a launch).
fcc_status_t launch_fp32_batch(int kh, int rs, const BatchParams &bp, int grid, size_t smem, cudaStream_t st)
{
    switch (kh) {
    case 2: return launch_batch_kh<2>(rs, bp, grid, smem, st);
    case 4: return launch_batch_kh<4>(rs, bp, grid, smem, st);
    case 6: return launch_batch_kh<6>(rs, bp, grid, smem, st);
    case 8: return launch_batch_kh<8>(rs, bp, grid, smem, st);
    default: return fail(FCC_ERR_UNSUPPORTED, "more than 8 bases of one parity");
    }
}

int fp32_row_slots(int Q) { return Q <= 32 ? 1 : Q / 32; }

}  // namespace fcc
