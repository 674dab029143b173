// fcc_fp32_reim.cu -- the split form (FCC_FORM_REIM_SPLIT) for alpha = 1 on the
// FP32 tile pipeline of fcc_fp32_tiles.cuh.
//
// The split form truncates C = Re W and S = Im W (Eq. 3) separately, so
// y = 2 (C_K Re x - S_K Im x) with C_K = U_c (sigma v^T)_c and S_K likewise.
// cos(2 pi (N/2 - f) tau / N) is not +/- cos(2 pi f tau / N) unless tau is an
// integer, so the Eq. 8 fold does not apply: each 16-byte record
// (u(f), u(N/2 - f)) of the per-microphone PHAT gives the two cross spectra
// a = x(f) y(f)^* and b = x(N/2 - f) y(N/2 - f)^* of a pair, and per coefficient
// v two packed FMAs add (C_v, S_v) * (Re, Im) at both bins into (c_v, s_v).
// Staging, PHAT, reduce-scatter, reconstruction, argmax and refinement are the
// folded kernel's.
#include <algorithm>

#include "fcc_fp32_tiles.cuh"

namespace fcc {
namespace {

template <int KH, int RS>
__global__ void __launch_bounds__(max_compute_warps(KH) * 32, 1)
    fcc_fp32_reim_kernel(const __grid_constant__ Fp32Params p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int n_local = (p.n_tiles > (int)blockIdx.x)
                            ? (p.n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x
                            : 0;
    fp32_tiles<KH, RS, true>(p, smem, blockIdx.x, gridDim.x, n_local);
}

template <int KH, int RS>
fcc_status_t launch_reim_inst(const fcc_plan *plan, const Fp32Params &prm, cudaStream_t st, int grid)
{
    static bool attr_set[64] = {};
    const int dev = plan->device;
    if (!attr_set[dev & 63]) {
        cudaError_t e = cudaFuncSetAttribute(fcc_fp32_reim_kernel<KH, RS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(fcc_fp32_reim_kernel)");
        attr_set[dev & 63] = true;
    }
    fcc_fp32_reim_kernel<KH, RS><<<grid, prm.G * prm.GW * 32, plan->geo.smem_bytes, st>>>(prm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fcc_fp32_reim_kernel launch");
    return FCC_OK;
}

template <int KH>
fcc_status_t launch_reim_kh(const fcc_plan *plan, const Fp32Params &prm, cudaStream_t st, int grid)
{
    switch (prm.Q <= 32 ? 1 : prm.Q / 32) {
    case 1: return launch_reim_inst<KH, 1>(plan, prm, st, grid);
    case 2: return launch_reim_inst<KH, 2>(plan, prm, st, grid);
    case 4: return launch_reim_inst<KH, 4>(plan, prm, st, grid);
    case 8: return launch_reim_inst<KH, 8>(plan, prm, st, grid);
    default: return fail(FCC_ERR_UNSUPPORTED, "the FP32 kernel needs N <= 1024");
    }
}

}  // namespace

// kh = half the coefficient pairs (c_v, s_v) per pair: max(K_c, K_s) rounded up
// to a multiple of 4, halved.
fcc_status_t launch_fp32_reim(const fcc_plan *plan, const Fp32Params &prm, cudaStream_t st, int grid)
{
    switch (plan->kh) {
    case 2: return launch_reim_kh<2>(plan, prm, st, grid);
    case 4: return launch_reim_kh<4>(plan, prm, st, grid);
    case 6: return launch_reim_kh<6>(plan, prm, st, grid);
    case 8: return launch_reim_kh<8>(plan, prm, st, grid);
    default: return fail(FCC_ERR_UNSUPPORTED, "more than 16 coefficient pairs");
    }
}

}  // namespace fcc
