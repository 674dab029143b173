// fcc_batch_all.cu -- the batched form's single persistent launch.
//
// One grid of kBatchAllWarps-warp CTAs runs every array of the batch, whatever
// its kernel class (bases per parity KH, fold records per lane RS): the CTAs
// take jobs -- one array, a run of its frame tiles -- from one queue ordered
// largest first, copy the array's kernel parameters into a shared-memory
// header, and run the tile pipeline of that array's class (the same per-frame
// arithmetic as fcc_tdoa with the same geometry).  The kernel's register budget
// is the largest class's (eight warps of up to 255 registers), so every array's
// geometry is limited to eight compute warps.
#include <algorithm>
#include <cfloat>

#include "fcc_device.cuh"
#include "fcc_internal.h"

#include "fcc_fp32_tiles.cuh"

namespace fcc {
namespace {

__global__ void __launch_bounds__(kBatchAllWarps * 32, 1) fcc_fp32_batch_all_kernel(const __grid_constant__ BatchParams bp)
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
        switch (job.code) {  // 4 (KH / 2 - 1) + log2(RS), uniform over the CTA
        case 0: fp32_tiles<2, 1, false>(*hdr, body, job.tile0, 1, job.n_tiles); break;
        case 1: fp32_tiles<2, 2, false>(*hdr, body, job.tile0, 1, job.n_tiles); break;
        case 2: fp32_tiles<2, 4, false>(*hdr, body, job.tile0, 1, job.n_tiles); break;
        case 3: fp32_tiles<2, 8, false>(*hdr, body, job.tile0, 1, job.n_tiles); break;
        case 4: fp32_tiles<4, 1, false>(*hdr, body, job.tile0, 1, job.n_tiles); break;
        case 5: fp32_tiles<4, 2, false>(*hdr, body, job.tile0, 1, job.n_tiles); break;
        case 6: fp32_tiles<4, 4, false>(*hdr, body, job.tile0, 1, job.n_tiles); break;
        case 7: fp32_tiles<4, 8, false>(*hdr, body, job.tile0, 1, job.n_tiles); break;
        case 8: fp32_tiles<6, 1, false>(*hdr, body, job.tile0, 1, job.n_tiles); break;
        case 9: fp32_tiles<6, 2, false>(*hdr, body, job.tile0, 1, job.n_tiles); break;
        case 10: fp32_tiles<6, 4, false>(*hdr, body, job.tile0, 1, job.n_tiles); break;
        case 11: fp32_tiles<6, 8, false>(*hdr, body, job.tile0, 1, job.n_tiles); break;
        case 12: fp32_tiles<8, 1, false>(*hdr, body, job.tile0, 1, job.n_tiles); break;
        case 13: fp32_tiles<8, 2, false>(*hdr, body, job.tile0, 1, job.n_tiles); break;
        case 14: fp32_tiles<8, 4, false>(*hdr, body, job.tile0, 1, job.n_tiles); break;
        default: fp32_tiles<8, 8, false>(*hdr, body, job.tile0, 1, job.n_tiles); break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint64_t *bars = reinterpret_cast<uint64_t *>(body);
            for (int s = 0; s < 3 * hdr->S; ++s) mbar_inval(&bars[s]);
        }
    }
}

}  // namespace

fcc_status_t launch_fp32_batch_all(const BatchParams &bp, int grid, size_t smem, cudaStream_t st)
{
    if (grid == 0) {  // prepare only: raise the shared-memory limit (not capturable)
        cudaError_t e = cudaFuncSetAttribute(fcc_fp32_batch_all_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             232448);
        return e == cudaSuccess ? FCC_OK : cuda_fail(e, "cudaFuncSetAttribute(fcc_fp32_batch_all_kernel)");
    }
    fcc_fp32_batch_all_kernel<<<grid, kBatchAllWarps * 32, smem, st>>>(bp);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FCC_OK : cuda_fail(e, "fcc_fp32_batch_all_kernel launch");
}

}  // namespace fcc
