// fcc_api.cu -- the extern "C" entry points declared in include/fcc.h.
#include <algorithm>
#include <cuda_fp16.h>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "fcc_debug.h"
#include "fcc_internal.h"

namespace fcc {

static thread_local std::string g_last_error;

fcc_status_t fail(fcc_status_t st, const std::string &msg)
{
    g_last_error = msg;
    return st;
}

fcc_status_t cuda_fail(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? FCC_ERR_OOM : FCC_ERR_CUDA;
}

DebugHooks &debug_hooks()
{
    static DebugHooks h{2000000000LL, 0, 0};
    return h;
}

cudaError_t dev_alloc(void **p, size_t bytes)
{
    DebugHooks &h = debug_hooks();
    if (h.fail_allocs > 0) {
        --h.fail_allocs;
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

namespace {

int pair_index(int M, int i, int j) { return i * M - i * (i + 1) / 2 + (j - i - 1); }

// Tile the pair triangle into 2x2 blocks of microphone groups {2a, 2a+1}:
// off-diagonal blocks carry up to 4 pairs; the one pair inside each group is
// collected two groups at a time.
std::vector<Slot> make_slots(int M)
{
    std::vector<Slot> out;
    const int G = (M + 1) / 2;
    auto mic = [&](int g, int r) { return 2 * g + r < M ? 2 * g + r : -1; };
    for (int a = 0; a < G; ++a)
        for (int b = a + 1; b < G; ++b) {
            int m[4] = {mic(a, 0), mic(a, 1), mic(b, 0), mic(b, 1)};
            Slot s;
            for (int q = 0; q < 4; ++q) {
                int i = m[q >> 1], j = m[2 + (q & 1)];
                s.pair[q] = (i >= 0 && j >= 0) ? pair_index(M, i, j) : -1;
            }
            for (int r = 0; r < 4; ++r) s.mic[r] = m[r] >= 0 ? m[r] : m[r & 2];
            out.push_back(s);
        }
    std::vector<int> diag;
    for (int a = 0; a < G; ++a)
        if (mic(a, 1) >= 0) diag.push_back(a);
    for (size_t k = 0; k < diag.size(); k += 2) {
        int a = diag[k], b = (k + 1 < diag.size()) ? diag[k + 1] : -1;
        Slot s;
        s.mic[0] = 2 * a;
        s.mic[2] = 2 * a + 1;
        s.mic[1] = b >= 0 ? 2 * b : 2 * a;
        s.mic[3] = b >= 0 ? 2 * b + 1 : 2 * a + 1;
        s.pair[0] = pair_index(M, 2 * a, 2 * a + 1);
        s.pair[1] = -1;
        s.pair[2] = -1;
        s.pair[3] = b >= 0 ? pair_index(M, 2 * b, 2 * b + 1) : -1;
        out.push_back(s);
    }
    return out;
}

// FP32 tables for the kernel (kh = bases per parity, padded with zeros):
//   basis: rows of BS floats, (pe_0 .. pe_{kh-1}, po_0 .. po_{kh-1}, pad); chunk c of
//     the bin-pair axis (QC = Q / C rows) starts at row c (QC + 1) -- one zero row
//     between chunks staggers their shared-memory banks -- and bin N/4 (no odd
//     part) is row C (QC + 1);
//   recon [center+1][4 kh]: row m (tau = m/den >= 0), per k the four weights
//     (gSe, gDe, gSo, gDo) = (2a Ue, 2b Ue, -2b Uo, 2a Uo) at tau, with
//     a = cos(pi tau / 2), b = sin(pi tau / 2); then y(+tau) = S - D and
//     y(-tau) = S + D where S = gSe.Re z_e + gSo.Re z_o and D = gDe.Im z_e + gDo.Im z_o
//     (Ue is even and Uo odd in tau).
// Split form (FCC_FORM_REIM_SPLIT), same row order: per coefficient v < 2 kh the
// float4 (C_v(f), S_v(f), C_v(N/2 - f), S_v(N/2 - f)) of the cosine / sine
// projections (sigma v of C = Re W and of S = Im W, zero past K_c / K_s), and
// (C_v(N/4), S_v(N/4), 0, 0) in the bin N/4 row; recon row m holds per k
// (2 U_c[k], 2 U_s[k], 2 U_c[kh + k], 2 U_s[kh + k]) at tau = m / den, so that
// S = 2 U_c . c, D = 2 U_s . s and y(+/-tau) = S -/+ D (U_c even, U_s odd in tau).
void pack_tables(const fcc_plan *plan, std::vector<float> &basis, std::vector<float> &recon)
{
    const fcc_plan_info_t &in = plan->info;
    const int kh = plan->kh, Q = in.Q, KE = in.K_even, KO = in.K_odd;
    const int C = plan->geo.C, BS = plan->geo.BS, QC = Q / C;
    basis.assign((size_t)(Q + C + 1) * BS, 0.f);
    if (in.form == FCC_FORM_REIM_SPLIT) {
        const int B = in.B;
        auto cw = [&](int v, int f) { return v < KE ? (float)plan->Pe[(size_t)v * B + f] : 0.f; };
        auto sw = [&](int v, int f) { return v < KO ? (float)plan->Po[(size_t)v * B + f] : 0.f; };
        for (int f = 0; f <= Q; ++f) {
            const int row = f < Q ? (f / QC) * (QC + 1) + f % QC : C * (QC + 1);
            float *r = &basis[(size_t)row * BS];
            for (int v = 0; v < 2 * kh; ++v) {
                r[4 * v] = cw(v, f);
                r[4 * v + 1] = sw(v, f);
                if (f < Q) {
                    r[4 * v + 2] = cw(v, 2 * Q - f);
                    r[4 * v + 3] = sw(v, 2 * Q - f);
                }
            }
        }
        recon.assign((size_t)(in.center + 1) * 4 * kh, 0.f);
        auto uc = [&](int i, int k) { return k < KE ? plan->Ue[(size_t)i * KE + k] : 0.0; };
        auto us = [&](int i, int k) { return k < KO ? plan->Uo[(size_t)i * KO + k] : 0.0; };
        for (int m = 0; m <= in.center; ++m)
            for (int k = 0; k < kh; ++k) {
                float *g = &recon[((size_t)m * kh + k) * 4];
                g[0] = (float)(2.0 * uc(in.center + m, k));
                g[1] = (float)(2.0 * us(in.center + m, k));
                g[2] = (float)(2.0 * uc(in.center + m, kh + k));
                g[3] = (float)(2.0 * us(in.center + m, kh + k));
            }
        return;
    }
    for (int f = 0; f <= Q; ++f) {
        const int row = f < Q ? (f / QC) * (QC + 1) + f % QC : C * (QC + 1);
        float *r = &basis[(size_t)row * BS];
        for (int k = 0; k < KE; ++k) r[k] = (float)plan->Pe[(size_t)k * (Q + 1) + f];
        if (f < Q)
            for (int k = 0; k < KO; ++k) r[kh + k] = (float)plan->Po[(size_t)k * Q + f];
    }
    recon.assign((size_t)(in.center + 1) * 4 * kh, 0.f);
    for (int m = 0; m <= in.center; ++m) {
        const int i = in.center + m;
        const double ang = M_PI * 0.5 * (double)m / (double)in.den;
        const double a = std::cos(ang), b = std::sin(ang);
        float *g = &recon[(size_t)m * 4 * kh];
        for (int k = 0; k < KE; ++k) {
            const double u = plan->Ue[(size_t)i * KE + k];
            g[4 * k] = (float)(2.0 * a * u);
            g[4 * k + 1] = (float)(2.0 * b * u);
        }
        for (int k = 0; k < KO; ++k) {
            const double u = plan->Uo[(size_t)i * KO + k];
            g[4 * k + 2] = (float)(-2.0 * b * u);
            g[4 * k + 3] = (float)(2.0 * a * u);
        }
    }
}

}  // namespace

// FP16 weight tables of the lag-grid reconstruction on the tensor cores,
// [S part 0 .. parts-1, D part 0 .. parts-1][npad][16] in K-major 8 x 8 core
// matrices: row n holds the weights of lag step m = m0 + n on (Re zE[0..7],
// Re zO[0..7]) for S and on the imaginary parts for D (S = sum 2a Ue Re zE -
// 2b Uo Re zO, D = sum 2b Ue Im zE + 2a Uo Im zO at tau = m / den, a =
// cos(pi tau / 2), b = sin(pi tau / 2)), so that y(center -/+ m) = S +/- D.
// Each weight, scaled by 2^shift, is split into `parts` FP16 terms (part 0 =
// fp16(w), each next part the FP16 rounding of what is left).  Rows past the
// grid's last lag step are zero.
std::vector<uint16_t> recon_tables_f16(const fcc_plan *plan, int npad, int m0, int shift, int parts)
{
    const fcc_plan_info_t &in = plan->info;
    const int KE = in.K_even, KO = in.K_odd;
    std::vector<uint16_t> rt((size_t)2 * parts * npad * 16, 0);
    const double sc = std::ldexp(1.0, shift);
    auto put = [&](int t, int n, int k, double w) {
        double v = w * sc;
        const size_t off = (((size_t)(n / 8) * 2 + k / 8) * 64 + (n % 8) * 8 + (k % 8));
        for (int q = 0; q < parts; ++q) {
            const __half h = __float2half_rn((float)v);
            rt[(size_t)(t * parts + q) * npad * 16 + off] = *reinterpret_cast<const uint16_t *>(&h);
            v -= (double)__half2float(h);
        }
    };
    for (int n = 0; n < npad && m0 + n <= in.center; ++n) {
        const int m = m0 + n, i = in.center + m;
        const double ang = M_PI * 0.5 * (double)m / (double)in.den;
        const double a = std::cos(ang), b = std::sin(ang);
        for (int k = 0; k < KE && k < 8; ++k) {
            const double u = plan->Ue[(size_t)i * KE + k];
            put(0, n, k, 2.0 * a * u);
            put(1, n, k, 2.0 * b * u);
        }
        for (int k = 0; k < KO && k < 8; ++k) {
            const double u = plan->Uo[(size_t)i * KO + k];
            put(0, n, 8 + k, -2.0 * b * u);
            put(1, n, 8 + k, 2.0 * a * u);
        }
    }
    return rt;
}

fcc_status_t set_fp32_geometry(fcc_plan *plan, const Fp32Geometry &g)
{
    plan->geo = g;
    std::vector<float> basis, recon;
    if (g.C) pack_tables(plan, basis, recon);
    else basis.assign(4, 0.f), recon.assign(4, 0.f);  // N > 1024: no FP32 kernel
    float *nb = nullptr, *nr = nullptr;
    cudaError_t e = dev_alloc(reinterpret_cast<void **>(&nb), basis.size() * sizeof(float));
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&nr), recon.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(nb, basis.data(), basis.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(nr, recon.data(), recon.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(nb);
        cudaFree(nr);
        return cuda_fail(e, "plan tables");
    }
    if (plan->d_basis || plan->d_recon) cudaDeviceSynchronize();  // no launch may still read the old tables
    cudaFree(plan->d_basis);
    cudaFree(plan->d_recon);
    plan->d_basis = nb;
    plan->d_recon = nr;
    return FCC_OK;
}

namespace {

// The host-streaming staging ring (fcc_tdoa_host), back to "not created".
void free_staging(fcc_plan *p)
{
    for (int b = 0; b < 2; ++b) {
        cudaFree(p->d_stage[b]);
        cudaFree(p->d_stage_idx[b]);
        cudaFree(p->d_stage_peak[b]);
        cudaFree(p->d_stage_tau[b]);
        p->d_stage[b] = nullptr;
        p->d_stage_idx[b] = nullptr;
        p->d_stage_peak[b] = nullptr;
        p->d_stage_tau[b] = nullptr;
    }
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    p->copy_stream = nullptr;
    for (auto &e : p->ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    p->stage_frames = 0;
}

void free_plan(fcc_plan *p)
{
    if (!p) return;
    cudaFree(p->d_basis);
    cudaFree(p->d_recon);
    cudaFree(p->d_slots);
    cudaFree(p->d_err);
    cudaFree(p->d_tc_bases);
    cudaFree(p->d_tc_peq);
    cudaFree(p->d_tc_rbases);
    cudaFree(p->d_fp32_rbases);
    cudaFree(p->d_tm_btab);
    cudaFree(p->d_smooth_basis);
    cudaFree(p->d_stft_tab);
    pcm_destroy(p);
    free_staging(p);
    gcc_destroy(p);
    delete p;
}

}  // namespace
}  // namespace fcc

// Validate a plan description and derive the plan's sizes (host only).
fcc_status_t fcc::plan_info_from_desc(const fcc_plan_desc_t *d, fcc_plan_info_t &in, int &dev)
{
    if (!d) return fail(FCC_ERR_INVALID_ARG, "null desc");
    if (d->n_mics < 2) return fail(FCC_ERR_INVALID_ARG, "n_mics < 2");
    if (d->n_mics > 16) return fail(FCC_ERR_UNSUPPORTED, "n_mics > 16");
    if (!(d->fs > 0)) return fail(FCC_ERR_INVALID_ARG, "fs <= 0");
    if (d->N < 16 || d->N > 4096 || (d->N & (d->N - 1)))
        return fail(FCC_ERR_INVALID_ARG, "N must be a power of two in [16, 4096]");
    if (d->lag_den < 1 || d->lag_den > 64) return fail(FCC_ERR_INVALID_ARG, "lag_den out of [1, 64]");
    if (d->prec < FCC_PREC_FP32 || d->prec > FCC_PREC_FP16) return fail(FCC_ERR_INVALID_ARG, "prec");
    if (d->form != FCC_FORM_FOLDED && d->form != FCC_FORM_REIM_SPLIT) return fail(FCC_ERR_INVALID_ARG, "form");
    if (d->form == FCC_FORM_REIM_SPLIT && d->prec != FCC_PREC_FP32)
        return fail(FCC_ERR_UNSUPPORTED, "the split form is FP32 only");
    if (d->K < 0) return fail(FCC_ERR_INVALID_ARG, "K < 0");
    const double c = d->c > 0 ? d->c : 343.0;
    int L;
    if (d->tau_max > 0) {
        L = (int)std::ceil(d->tau_max - 1e-9);
    } else {
        if (!d->mic_xyz) return fail(FCC_ERR_INVALID_ARG, "tau_max <= 0 needs mic_xyz");
        double dmax = 0;
        for (int i = 0; i < d->n_mics; ++i)
            for (int j = i + 1; j < d->n_mics; ++j) {
                double s = 0;
                for (int k = 0; k < 3; ++k) {
                    double t = d->mic_xyz[3 * i + k] - d->mic_xyz[3 * j + k];
                    s += t * t;
                }
                dmax = std::max(dmax, std::sqrt(s));
            }
        L = (int)std::ceil(dmax * d->fs / c - 1e-9);
    }
    if (L < 1) return fail(FCC_ERR_INVALID_ARG, "lag half-range must be at least one sample");
    const int I = 2 * L * d->lag_den + 1;
    if (I > 1025) return fail(FCC_ERR_UNSUPPORTED, "more than 1025 lag candidates");
    if (L * 2 > d->N / 2) return fail(FCC_ERR_INVALID_ARG, "lag range too large for N");

    dev = d->device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return fail(FCC_ERR_CUDA, "no CUDA device");
    in = fcc_plan_info_t{};
    in.M = d->n_mics;
    in.P = in.M * (in.M - 1) / 2;
    in.N = d->N;
    in.B = d->N / 2 + 1;
    in.Q = d->N / 4;
    in.L = L;
    in.den = d->lag_den;
    in.I = I;
    in.center = L * d->lag_den;
    in.prec = d->prec;
    in.form = d->form;
    in.delta = 1.0 / d->lag_den;
    in.fs = d->fs;
    in.c = c;
    return FCC_OK;
}

using namespace fcc;

int fcc::resolved_engine(const fcc_plan *plan)
{
    switch (plan->engine) {
    case FCC_ENGINE_CUDA_CORES: return FCC_ENGINE_CUDA_CORES;
    case FCC_ENGINE_TENSOR_TMEM: return FCC_ENGINE_TENSOR_TMEM;
    case FCC_ENGINE_TENSOR_SMEM: return FCC_ENGINE_TENSOR_SMEM;
    default:
        if (plan->info.prec == FCC_PREC_FP32) return FCC_ENGINE_CUDA_CORES;
        return FCC_ENGINE_TENSOR_SMEM;
    }
}

extern "C" {

const char *fcc_status_string(fcc_status_t s)
{
    switch (s) {
    case FCC_OK: return "ok";
    case FCC_ERR_INVALID_ARG: return "invalid argument";
    case FCC_ERR_UNSUPPORTED: return "unsupported";
    case FCC_ERR_OOM: return "out of memory";
    case FCC_ERR_CUDA: return "CUDA error";
    case FCC_ERR_TIMEOUT: return "device wait timed out";
    case FCC_ERR_NONFINITE: return "non-finite input";
    case FCC_ERR_NOT_CONVERGED: return "SVD did not converge";
    }
    return "unknown status";
}

const char *fcc_last_error(void) { return g_last_error.c_str(); }

fcc_status_t fcc_debug_set(int hook, long long value)
{
    DebugHooks &h = debug_hooks();
    switch (hook) {
    case FCC_DEBUG_WAIT_CYCLES:
        if (value != 0 && value < 1000) return fail(FCC_ERR_INVALID_ARG, "wait bound below 1000 cycles");
        h.wait_cycles = value ? value : 2000000000LL;
        return FCC_OK;
    case FCC_DEBUG_WITHHOLD_COPY:
        if (value < 0 || value > (1 << 30)) return fail(FCC_ERR_INVALID_ARG, "count out of range");
        h.withhold_copies = (int)value;
        return FCC_OK;
    case FCC_DEBUG_FAIL_ALLOC:
        if (value < 0 || value > (1 << 30)) return fail(FCC_ERR_INVALID_ARG, "count out of range");
        h.fail_allocs = (int)value;
        return FCC_OK;
    }
    return fail(FCC_ERR_INVALID_ARG, "unknown debug hook");
}

fcc_status_t fcc_plan_create(const fcc_plan_desc_t *d, fcc_plan_t **out)
{
    g_last_error.clear();
    if (!d || !out) return fail(FCC_ERR_INVALID_ARG, "null desc or out");
    *out = nullptr;
    fcc_plan_info_t info0;
    int dev = 0;
    fcc_status_t st0 = plan_info_from_desc(d, info0, dev);
    if (st0 != FCC_OK) return st0;
    DeviceScope scope(dev);
    if (!scope.ok) return fail(FCC_ERR_CUDA, "cudaSetDevice failed");
    fcc_plan *p = new (std::nothrow) fcc_plan();
    if (!p) return fail(FCC_ERR_OOM, "host allocation");
    p->device = dev;
    p->info = info0;
    fcc_plan_info_t &in = p->info;
    p->taus.resize(in.I);
    for (int i = 0; i < in.I; ++i) p->taus[i] = (double)(i - in.center) / (double)in.den;
    cudaError_t e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        free_plan(p);
        return cuda_fail(e, "cudaDeviceGetAttribute");
    }
    fcc_status_t st = build_plan_bases(p, d->K, d->energy > 0 ? d->energy : 0.999);
    if (st != FCC_OK) {
        free_plan(p);
        return st;
    }
    const int kmax = std::max(in.K_even, in.K_odd);
    if (in.form == FCC_FORM_REIM_SPLIT) {
        // KB = max(K_c, K_s) packed coefficient pairs (c_k, s_k), rounded up to a
        // multiple of 4; the per-pair kernel's template counts KB / 2 of them
        const int kb = (kmax + 3) / 4 * 4;
        p->kh = kb <= 16 ? kb / 2 : 0;
    } else {
        p->kh = kmax <= 2 ? 2 : kmax <= 4 ? 4 : kmax <= 6 ? 6 : kmax <= 8 ? 8 : 0;
    }
    std::vector<Slot> slots = make_slots(in.M);
    p->n_slots = (int)slots.size();
    if (p->kh) {
        // the FP32 kernel's tables (folded or split form); the split form also
        // gets the per-pair kernel's weights (Eq. 1 smoothing)
        st = choose_fp32_geometry(p);
        if (st == FCC_OK) st = set_fp32_geometry(p, p->geo);
        if (st == FCC_OK && in.form == FCC_FORM_REIM_SPLIT) st = prepare_reim(p);
        if (st != FCC_OK) {
            free_plan(p);
            return st;
        }
    } else if (in.form == FCC_FORM_REIM_SPLIT) {
        st = set_fp32_geometry(p, Fp32Geometry{});  // placeholder tables: more bases than any kernel takes
        if (st != FCC_OK) {
            free_plan(p);
            return st;
        }
    }
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&p->d_slots), slots.size() * sizeof(Slot));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_slots, slots.data(), slots.size() * sizeof(Slot), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&p->d_err), sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(unsigned));
    if (e != cudaSuccess) {
        free_plan(p);
        return cuda_fail(e, "plan tables");
    }
    if (in.form == FCC_FORM_FOLDED && in.prec == FCC_PREC_FP32 && p->kh) st = prepare_per_pair(p);
    if (st == FCC_OK && in.form == FCC_FORM_FOLDED && p->kh >= 6) st = prepare_fp32_mma(p);
    if (st == FCC_OK) st = prepare_stft(p);
    if (st != FCC_OK) {
        free_plan(p);
        return st;
    }
    if (in.prec != FCC_PREC_FP32) {
        st = prepare_tc(p);
        if (st != FCC_OK) {
            free_plan(p);
            return st;
        }
    }
    if (in.form == FCC_FORM_FOLDED) {
        // the tensor-memory path where it applies; a plan it does not apply to
        // keeps the other engines (the reason stays in fcc_last_error)
        st = prepare_tm(p);
        if (st == FCC_ERR_OOM || st == FCC_ERR_CUDA) {
            free_plan(p);
            return st;
        }
    }
    if (debug_enabled())
        fprintf(stderr, "[fcc] plan M=%d N=%d I=%d K=%d (%d+%d) kh=%d slots=%d fp32: C=%d SB=%d GW=%d G=%d F=%d S=%d smem=%zu\n",
                in.M, in.N, in.I, in.K, in.K_even, in.K_odd, p->kh, p->n_slots, p->geo.C, p->geo.SB, p->geo.GW,
                p->geo.G, p->geo.F, p->geo.S, p->geo.smem_bytes);
    *out = p;
    return FCC_OK;
}

void fcc_plan_destroy(fcc_plan_t *plan)
{
    if (!plan) return;
    DeviceScope scope(plan->device);
    cudaDeviceSynchronize();
    free_plan(plan);
}

fcc_status_t fcc_plan_set_engine(fcc_plan_t *plan, int engine)
{
    if (!plan) return fail(FCC_ERR_INVALID_ARG, "null plan");
    if (engine < FCC_ENGINE_AUTO || engine > FCC_ENGINE_TENSOR_SMEM) return fail(FCC_ERR_INVALID_ARG, "engine");
    const bool fp32 = plan->info.prec == FCC_PREC_FP32;
    if (engine == FCC_ENGINE_CUDA_CORES && (!fp32 || plan->geo.G == 0))
        return fail(FCC_ERR_UNSUPPORTED, "the CUDA-core kernel runs FP32 plans with N <= 1024");
    if (engine == FCC_ENGINE_TENSOR_TMEM && !plan->tm.smem)
        return fail(FCC_ERR_UNSUPPORTED, "the tensor-memory kernel does not apply to this plan");
    if (engine == FCC_ENGINE_TENSOR_SMEM && (fp32 || !plan->tc_smem))
        return fail(FCC_ERR_UNSUPPORTED, "the shared-memory tensor-core kernel runs BF16 / FP16 plans");
    plan->engine = engine;
    return FCC_OK;
}

fcc_status_t fcc_plan_get_engine(const fcc_plan_t *plan, int *engine)
{
    if (!plan || !engine) return fail(FCC_ERR_INVALID_ARG, "null plan or engine");
    *engine = resolved_engine(plan);
    return FCC_OK;
}

fcc_status_t fcc_plan_info(const fcc_plan_t *plan, fcc_plan_info_t *info)
{
    if (!plan || !info) return fail(FCC_ERR_INVALID_ARG, "null argument");
    *info = plan->info;
    return FCC_OK;
}

fcc_status_t fcc_plan_taus(const fcc_plan_t *plan, double *taus)
{
    if (!plan || !taus) return fail(FCC_ERR_INVALID_ARG, "null argument");
    std::copy(plan->taus.begin(), plan->taus.end(), taus);
    return FCC_OK;
}

fcc_status_t fcc_plan_singular_values(const fcc_plan_t *plan, double *s_even, int *n_even, double *s_odd,
                                      int *n_odd)
{
    if (!plan) return fail(FCC_ERR_INVALID_ARG, "null plan");
    if (n_even) *n_even = (int)plan->s_even.size();
    if (n_odd) *n_odd = (int)plan->s_odd.size();
    if (s_even) std::copy(plan->s_even.begin(), plan->s_even.end(), s_even);
    if (s_odd) std::copy(plan->s_odd.begin(), plan->s_odd.end(), s_odd);
    return FCC_OK;
}

fcc_status_t fcc_plan_bases(const fcc_plan_t *plan, double *Pe, double *Po, double *Ue, double *Uo)
{
    if (!plan) return fail(FCC_ERR_INVALID_ARG, "null plan");
    if (Pe) std::copy(plan->Pe.begin(), plan->Pe.end(), Pe);
    if (Po) std::copy(plan->Po.begin(), plan->Po.end(), Po);
    if (Ue) std::copy(plan->Ue.begin(), plan->Ue.end(), Ue);
    if (Uo) std::copy(plan->Uo.begin(), plan->Uo.end(), Uo);
    return FCC_OK;
}

fcc_status_t fcc_tdoa(fcc_plan_t *plan, const void *d_spectra, long long T, int *d_lag_idx, float *d_peak,
                      float *d_tau_hat, float *d_coeffs, float *d_corr, void *stream)
{
    if (!plan) return fail(FCC_ERR_INVALID_ARG, "null plan");
    if (T < 0) return fail(FCC_ERR_INVALID_ARG, "T < 0");
    if (T == 0) return FCC_OK;
    if (!d_spectra || !d_lag_idx || !d_peak) return fail(FCC_ERR_INVALID_ARG, "null spectra/lag_idx/peak");
    if (reinterpret_cast<uintptr_t>(d_spectra) & 15) return fail(FCC_ERR_INVALID_ARG, "spectra not 16-byte aligned");
    if ((reinterpret_cast<uintptr_t>(d_lag_idx) | reinterpret_cast<uintptr_t>(d_peak) |
         reinterpret_cast<uintptr_t>(d_tau_hat) | reinterpret_cast<uintptr_t>(d_coeffs) |
         reinterpret_cast<uintptr_t>(d_corr)) & 3)
        return fail(FCC_ERR_INVALID_ARG, "output not 4-byte aligned");
    if (!plan->kh) return fail(FCC_ERR_UNSUPPORTED, "more than 8 bases of one parity");
    DeviceScope scope(plan->device);
    if (!scope.ok) return fail(FCC_ERR_CUDA, "cudaSetDevice failed");
    return launch_tdoa(plan, static_cast<const float2 *>(d_spectra), T, d_lag_idx, d_peak, d_tau_hat, d_coeffs,
                       d_corr, static_cast<cudaStream_t>(stream));
}

fcc_status_t fcc_plan_sync(fcc_plan_t *plan, void *stream)
{
    if (!plan) return fail(FCC_ERR_INVALID_ARG, "null plan");
    DeviceScope scope(plan->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    FCC_CUDA_TRY(cudaStreamSynchronize(st));
    unsigned err = 0;
    FCC_CUDA_TRY(cudaMemcpyAsync(&err, plan->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    FCC_CUDA_TRY(cudaMemsetAsync(plan->d_err, 0, sizeof(unsigned), st));
    FCC_CUDA_TRY(cudaStreamSynchronize(st));
    if (err & kErrTimeout) return fail(FCC_ERR_TIMEOUT, "a device-side wait expired");
    if (err & kErrNonFinite) return fail(FCC_ERR_NONFINITE, "NaN or Inf in the spectra");
    return FCC_OK;
}

fcc_status_t fcc_tdoa_host(fcc_plan_t *plan, const void *h_spectra, long long T, int *h_lag_idx,
                           float *h_peak, float *h_tau_hat, void *stream)
{
    if (!plan) return fail(FCC_ERR_INVALID_ARG, "null plan");
    if (T < 0) return fail(FCC_ERR_INVALID_ARG, "T < 0");
    if (T == 0) return FCC_OK;
    if (!h_spectra || !h_lag_idx || !h_peak) return fail(FCC_ERR_INVALID_ARG, "null host buffer");
    if (!plan->kh) return fail(FCC_ERR_UNSUPPORTED, "more than 8 bases of one parity");
    DeviceScope scope(plan->device);
    if (!scope.ok) return fail(FCC_ERR_CUDA, "cudaSetDevice failed");
    const fcc_plan_info_t &in = plan->info;
    const size_t frame_bytes = (size_t)in.M * in.B * 8;
    if (!plan->stage_frames) {
        // the staging ring, created on first use; stage_frames is set only once
        // every part exists, and a failed creation frees the parts it made
        const long long chunk = std::max<long long>(1, (256LL << 20) / (long long)frame_bytes);
        cudaError_t e = cudaSuccess;
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = dev_alloc(&plan->d_stage[b], chunk * frame_bytes);
            if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&plan->d_stage_idx[b]), chunk * in.P * sizeof(int));
            if (e == cudaSuccess)
                e = dev_alloc(reinterpret_cast<void **>(&plan->d_stage_peak[b]), chunk * in.P * sizeof(float));
            if (e == cudaSuccess)
                e = dev_alloc(reinterpret_cast<void **>(&plan->d_stage_tau[b]), chunk * in.P * sizeof(float));
        }
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&plan->copy_stream, cudaStreamNonBlocking);
        for (auto &ev : plan->ev)
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            free_staging(plan);
            return e == cudaErrorMemoryAllocation ? fail(FCC_ERR_OOM, "fcc_tdoa_host staging")
                                                  : cuda_fail(e, "fcc_tdoa_host staging");
        }
        plan->stage_frames = chunk;
    }
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaStream_t hs = plan->copy_stream;
    // ev[b]: H2D of buffer b done; ev[2+b]: buffer b free again (kernel and D2H done)
    FCC_CUDA_TRY(cudaEventRecord(plan->ev[4], cs));
    FCC_CUDA_TRY(cudaStreamWaitEvent(hs, plan->ev[4], 0));
    const char *src = static_cast<const char *>(h_spectra);
    long long chunk_id = 0;
    for (long long t0 = 0; t0 < T; t0 += plan->stage_frames, ++chunk_id) {
        const int b = (int)(chunk_id & 1);
        const long long n = std::min(plan->stage_frames, T - t0);
        if (chunk_id >= 2) FCC_CUDA_TRY(cudaStreamWaitEvent(hs, plan->ev[2 + b], 0));
        FCC_CUDA_TRY(cudaMemcpyAsync(plan->d_stage[b], src + (size_t)t0 * frame_bytes, (size_t)n * frame_bytes,
                                     cudaMemcpyHostToDevice, hs));
        FCC_CUDA_TRY(cudaEventRecord(plan->ev[b], hs));
        FCC_CUDA_TRY(cudaStreamWaitEvent(cs, plan->ev[b], 0));
        fcc_status_t st = launch_tdoa(plan, static_cast<const float2 *>(plan->d_stage[b]), n, plan->d_stage_idx[b],
                                      plan->d_stage_peak[b], h_tau_hat ? plan->d_stage_tau[b] : nullptr, nullptr,
                                      nullptr, cs);
        if (st != FCC_OK) return st;
        const size_t o = (size_t)t0 * in.P, cnt = (size_t)n * in.P;
        FCC_CUDA_TRY(cudaMemcpyAsync(h_lag_idx + o, plan->d_stage_idx[b], cnt * sizeof(int), cudaMemcpyDeviceToHost, cs));
        FCC_CUDA_TRY(cudaMemcpyAsync(h_peak + o, plan->d_stage_peak[b], cnt * sizeof(float), cudaMemcpyDeviceToHost, cs));
        if (h_tau_hat)
            FCC_CUDA_TRY(cudaMemcpyAsync(h_tau_hat + o, plan->d_stage_tau[b], cnt * sizeof(float),
                                         cudaMemcpyDeviceToHost, cs));
        FCC_CUDA_TRY(cudaEventRecord(plan->ev[2 + b], cs));
    }
    return fcc_plan_sync(plan, stream);
}

fcc_status_t fcc_gcc_tdoa(fcc_plan_t *plan, const void *d_spectra, long long T, int *d_lag_idx, float *d_peak,
                          float *d_corr, void *stream)
{
    if (!plan) return fail(FCC_ERR_INVALID_ARG, "null plan");
    if (T < 0) return fail(FCC_ERR_INVALID_ARG, "T < 0");
    if (T == 0) return FCC_OK;
    if (!d_spectra || !d_lag_idx || !d_peak) return fail(FCC_ERR_INVALID_ARG, "null spectra/lag_idx/peak");
    if (reinterpret_cast<uintptr_t>(d_spectra) & 15) return fail(FCC_ERR_INVALID_ARG, "spectra not 16-byte aligned");
    DeviceScope scope(plan->device);
    if (!scope.ok) return fail(FCC_ERR_CUDA, "cudaSetDevice failed");
    return gcc_run(plan, static_cast<const float2 *>(d_spectra), T, d_lag_idx, d_peak, d_corr,
                   static_cast<cudaStream_t>(stream));
}

}  // extern "C"
