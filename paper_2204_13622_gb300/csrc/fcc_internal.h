// fcc_internal.h -- shared declarations of the CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdlib>
#include <string>
#include <vector>

#include "fcc.h"

namespace fcc {

// Device error word bits (latched by kernels, read by fcc_plan_sync).
enum : unsigned {
    kErrNonFinite = 1u,
    kErrTimeout = 2u,
};

// Records a detail message for fcc_last_error() and returns `st`.
fcc_status_t fail(fcc_status_t st, const std::string &msg);
fcc_status_t cuda_fail(cudaError_t e, const char *what);

// Test hooks (include/fcc_debug.h), process-wide.
struct DebugHooks {
    long long wait_cycles;  // device wait bound for FP32 launches
    int withhold_copies;    // FP32 launches left that withhold one bulk copy
    int fail_allocs;        // plan allocations left that fail
};
DebugHooks &debug_hooks();
// cudaMalloc through the allocation-failure hook.
cudaError_t dev_alloc(void **p, size_t bytes);

// FCC_DEBUG set to anything but "" or "0": print plan geometry and tuning steps.
inline bool debug_enabled()
{
    const char *d = std::getenv("FCC_DEBUG");
    return d && *d && !(d[0] == '0' && d[1] == 0);
}

// Makes `dev` current for the scope of one entry point and restores the
// caller's device afterwards.
struct DeviceScope {
    int prev = -1;
    bool ok = true;
    explicit DeviceScope(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceScope()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

#define FCC_CUDA_TRY(call)                                          \
    do {                                                            \
        cudaError_t e__ = (call);                                   \
        if (e__ != cudaSuccess) return ::fcc::cuda_fail(e__, #call); \
    } while (0)

// One work slot of the FP32 kernel: a 2x2 block of the pair triangle,
// mics {i1, i2} x {j1, j2}; pair[q] is the output pair index of
// (i1,j1), (i1,j2), (i2,j1), (i2,j2) or -1 when that product is not a pair.
struct Slot {
    int mic[4];   // i1, i2, j1, j2
    int pair[4];
};

// Launch geometry of the FP32 kernel, chosen on the host per plan.
struct Fp32Geometry {
    int C;            // frequency chunks per slot (lanes that share one slot)
    int SB;           // slots per warp (32 / C); a warp's lanes are chunk-major
    int lanes_frame;  // lanes per frame: whole warps, ceil(n_slots / SB) * 32
    int GW;           // warps per group
    int G;            // groups per CTA
    int F;            // frames per stage (tile)
    int S;            // stages in the shared-memory ring (a multiple of G)
    int BS;           // basis row stride in floats (an odd number of 16-byte units)
    size_t smem_bytes;
};

inline bool same_geometry(const Fp32Geometry &a, const Fp32Geometry &b)
{
    return a.C == b.C && a.GW == b.GW && a.G == b.G && a.F == b.F && a.S == b.S;
}

// Kernel parameters of the FP32 path (passed by value).
struct Fp32Params {
    const float2 *spectra;  // [T][M][B]
    long long T;
    int M, B, Q, N, P;
    int n_slots, C, SB, lanes_frame, GW, G, F, S, BS;
    int n_tiles;
    int frame_floats;       // M * B * 2
    int bulk;               // 1: cp.async.bulk staging, 0: plain-load staging
    int center, I, KE, KO;  // KE/KO: actual basis counts (<= KH)
    float delta;
    const float *basis;     // [Q+C+1][BS]: per chunk QC rows + one zero row, then bin N/4
    const float *recon;     // [center+1][KH][4]: (gSe, gDe, gSo, gDo) per k
    const Slot *slots;      // [n_slots]
    int *out_idx;
    float *out_peak;
    float *out_tau;         // nullable
    float *out_coef;        // nullable, [T][P][2K]
    float *out_corr;        // nullable, [T][P][I]
    unsigned *err;
    long long wait_cycles;  // bound of every device-side wait (clock cycles)
    int inject;             // test hook: 1 = the copy of the plan's first tile is withheld
    // lag grid on the tensor cores (single-plan folded launches; npad = 0: CUDA cores)
    const void *rbases;     // FP16 [S 3 parts, D 3 parts][npad][16], lag steps m = 1 .. npad
    int npad;               // a multiple of 32, >= center
    int rshift;             // the weights are scaled by 2^rshift
};

// Batched FP32 form: one job = a run of consecutive tiles of one plan.
struct BatchJob {
    int array;    // index into BatchParams::arrays
    int tile0;    // first tile (F frames each, F from the array's geometry)
    int n_tiles;
    int code;     // kernel instance of the array: 4 (KH / 2 - 1) + log2(RS)
};

struct BatchParams {
    const Fp32Params *arrays;  // [n_arrays], device
    const BatchJob *jobs;      // [n_jobs], device, in the order CTAs take them
    int n_jobs;
    int *counter;              // next job; zeroed before every launch
};

// Shared-memory header of the batched kernel (the job's Fp32Params and the job
// index) in front of the plan's own layout.
constexpr int kBatchHeaderBytes = 256;
static_assert(sizeof(Fp32Params) + 8 <= kBatchHeaderBytes, "batch header");

// Kernel parameters of the tensor-core (BF16 / FP16) path.
struct TcParams {
    const float2 *spectra;  // [T][M][B]
    long long T;
    int M, B, Q, P, n_slots, F, n_tiles;
    int center, I, KE, KO;
    float delta;
    const void *bases;      // 2 parts x [16][2Q] 16-bit, K-major core matrices
    const float *peq;       // [8]: even bases at bin N/4
    const void *rbases;     // lag-grid tables for the reconstruction on the tensor cores:
                            // [S hi, S lo, D hi, D lo][npad][16] FP16, K-major core matrices
    int npad;               // lag steps 0..center rounded up to 16; 0: the CUDA-core scan
    const float *recon;     // as in Fp32Params
    const Slot *slots;
    int *out_idx;
    float *out_peak;
    float *out_tau;
    float *out_coef;
    float *out_corr;
    unsigned *err;
};

// Geometry of the tensor-memory path (fcc_tmem.cu), chosen on the host per plan.
struct TmGeometry {
    int F = 0;    // frames per tile (F * slots <= 32: 128 TMEM lanes)
    int S = 0;    // raw frame stages
    int NI = 0;   // MMA-issuing warps (each with its own copy of D)
    int NBA = 0;  // A buffers in the tensor-memory ring
    int CH = 0;   // record quads per A buffer (chunk)
    size_t smem = 0;
};

// Kernel parameters of the tensor-memory path (passed by value).
struct TmParams {
    const float2 *spectra;  // [T][M][B]
    long long T;
    int M, B, Q, P, n_slots, F, S, n_tiles;
    int center, I, KE, KO, kh;
    int nq;                 // record quads: Q / 4 + 1 (records 0..Q, then zeros)
    int bq;                 // bytes of one quad's B block
    int us;                 // bytes per unit-phase row (a multiple of 128)
    int NI, NBA, CH;
    float delta;
    const void *btab;       // [nq][bq] B blocks (K-major core matrices)
    const float *recon;     // as in Fp32Params
    const Slot *slots;
    int *out_idx;
    float *out_peak;
    float *out_tau;
    float *out_coef;
    float *out_corr;
    unsigned *err;
    long long wait_cycles;
    int inject;             // test hook: CTA 0 withholds the copy of its first tile
};

}  // namespace fcc

// The plan object behind the opaque ABI handle.
struct fcc_plan {
    fcc_plan_info_t info{};
    int device = 0;
    int kh = 0;                    // padded basis count per parity (template instance)
    std::vector<double> taus;      // [I]
    std::vector<double> s_even, s_odd;
    std::vector<double> Pe, Po, Ue, Uo;  // FP64 bases as used (see fcc_plan_bases)
    // device
    float *d_basis = nullptr;
    float *d_recon = nullptr;
    fcc::Slot *d_slots = nullptr;
    unsigned *d_err = nullptr;
    int n_slots = 0;
    fcc::Fp32Geometry geo{};
    int num_sms = 0;
    // host-streaming staging (fcc_tdoa_host), created lazily
    void *d_stage[2] = {nullptr, nullptr};
    int *d_stage_idx[2] = {nullptr, nullptr};
    float *d_stage_peak[2] = {nullptr, nullptr};
    float *d_stage_tau[2] = {nullptr, nullptr};
    long long stage_frames = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev[6] = {};
    // GCC baseline workspace, created lazily
    void *gcc_state = nullptr;
    // tensor-core (BF16 / FP16) path
    float *d_smooth_basis = nullptr;   // smoothed path: [2 kh][QP], created on first use
    float *d_stft_tab = nullptr;       // STFT front-end: twiddles and window, created on first use
    void *pcm_state = nullptr;         // fcc_tdoa_pcm_host staging, created on first use
    void *d_tc_bases = nullptr;
    float *d_tc_peq = nullptr;
    void *d_tc_rbases = nullptr;       // reconstruction tables of the tensor-core path (or null)
    void *d_fp32_rbases = nullptr;     // FP32 kernel: lag-grid tables for the tensor cores (or null)
    int fp32_npad = 0, fp32_rshift = 0;
    int tc_npad = 0;
    int tc_F = 0;
    size_t tc_smem = 0;
    // tensor-memory path (fcc_tmem.cu)
    void *d_tm_btab = nullptr;
    fcc::TmGeometry tm{};
    int engine = 0;                    // fcc_engine_t requested (FCC_ENGINE_AUTO = 0)
};

namespace fcc {
fcc_status_t plan_info_from_desc(const fcc_plan_desc_t *d, fcc_plan_info_t &in, int &dev);
fcc_status_t build_plan_bases(fcc_plan *plan, int K_req, double energy);
fcc_status_t finish_plan_bases(fcc_plan *plan, const std::vector<double> &Xe, const std::vector<double> &Xo,
                               const std::vector<double> &Je, const std::vector<double> &Jo, int K_req,
                               double energy);
fcc_status_t choose_fp32_geometry(fcc_plan *plan);
// max_warps > 0 keeps only geometries of at most that many compute warps.
fcc_status_t fp32_candidates(const fcc_plan *plan, std::vector<Fp32Geometry> &out, int max_warps = 0);
// Set the plan's FP32 geometry and rebuild its device tables for it.
// FP16 split weight tables (`parts` terms) of the tensor-core lag grids (fcc_api.cu).
std::vector<uint16_t> recon_tables_f16(const fcc_plan *plan, int npad, int m0, int shift, int parts);
// FP32 kernel: builds the tensor-core lag-grid tables when the plan's grid is long
// enough for them to pay (fcc_fp32.cu).
fcc_status_t prepare_fp32_mma(fcc_plan *plan);
fcc_status_t set_fp32_geometry(fcc_plan *plan, const Fp32Geometry &g);
Fp32Params make_fp32_params(const fcc_plan *plan, const float2 *spectra, long long T, int *idx, float *peak,
                            float *tau, float *coef, float *corr, unsigned *err);
fcc_status_t launch_fp32_batch(int kh, int rs, const BatchParams &bp, int grid, size_t smem, cudaStream_t st);
// The single persistent launch of the batched form: every array of every kernel
// class in one grid of kBatchAllWarps-warp CTAs (grid = 0 only prepares).
constexpr int kBatchAllWarps = 8;
fcc_status_t launch_fp32_batch_all(const BatchParams &bp, int grid, size_t smem, cudaStream_t st);
int fp32_threads(int kh);
int fp32_row_slots(int Q);
fcc_status_t launch_fp32(const fcc_plan *plan, const float2 *spectra, long long T, int *idx,
                         float *peak, float *tau, float *coef, float *corr, cudaStream_t st);
fcc_status_t prepare_tc(fcc_plan *plan);
fcc_status_t launch_tc(const fcc_plan *plan, const float2 *spectra, long long T, int *idx, float *peak,
                       float *tau, float *coef, float *corr, cudaStream_t st);
// Split-form (FCC_FORM_REIM_SPLIT) weights of the per-pair kernel (Eq. 1
// smoothing), and the split-form FP32 kernel's launch (alpha = 1).
fcc_status_t prepare_reim(fcc_plan *plan);
fcc_status_t launch_fp32_reim(const fcc_plan *plan, const Fp32Params &prm, cudaStream_t st, int grid);
fcc_status_t prepare_tm(fcc_plan *plan);
fcc_status_t launch_tm(const fcc_plan *plan, const float2 *spectra, long long T, int *idx, float *peak,
                       float *tau, float *coef, float *corr, cudaStream_t st);
// The engine a plan runs fcc_tdoa on (fcc_engine_t, never AUTO).
int resolved_engine(const fcc_plan *plan);
// By the plan's engine: the CUDA-core kernel (FP32, folded or split form), the
// tensor-memory kernel, or the shared-memory tensor-core kernel (16-bit forms).
inline fcc_status_t launch_tdoa(const fcc_plan *plan, const float2 *spectra, long long T, int *idx, float *peak,
                                float *tau, float *coef, float *corr, cudaStream_t st)
{
    switch (resolved_engine(plan)) {
    case FCC_ENGINE_TENSOR_TMEM: return launch_tm(plan, spectra, T, idx, peak, tau, coef, corr, st);
    case FCC_ENGINE_TENSOR_SMEM: return launch_tc(plan, spectra, T, idx, peak, tau, coef, corr, st);
    default: return launch_fp32(plan, spectra, T, idx, peak, tau, coef, corr, st);
    }
}
void pcm_destroy(fcc_plan *plan);
// Plan-time tables of the per-pair kernel (folded form) and of the STFT front-end.
fcc_status_t prepare_per_pair(fcc_plan *plan);
fcc_status_t prepare_stft(fcc_plan *plan);
fcc_status_t gcc_run(fcc_plan *plan, const float2 *spectra, long long T, int *idx, float *peak,
                     float *corr, cudaStream_t st);
void gcc_destroy(fcc_plan *plan);
}  // namespace fcc
