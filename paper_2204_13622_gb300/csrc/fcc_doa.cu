// fcc_doa.cu -- DoA search over candidate directions from the pairs' FCC
// correlations on the lag grid (the next step named in the paper's
// conclusion): score(u) = sum over pairs of y_ij at tau_ij(u), linearly
// interpolated on the grid, and the best candidate per frame.
//
// srp_kernel<F>: persistent CTAs over tiles of F frames.  A tile's
// correlations are staged in shared memory as (y_k, y_{k+1} - y_k) pairs, so
// one 8-byte load and one FMA read an interpolated value.  Thread = candidate
// (groups of blockDim.x candidates): per pair it loads the candidate's grid
// position (k, w) once (L2-resident table [P][D]) and accumulates all F frames'
// scores; then each thread keeps its best candidate per frame, and the CTA
// reduces the per-frame maxima (lowest caller index on ties).  The candidates
// are searched in an order that makes every 32 consecutive ones a compact
// patch of directions (recursive median splits), so a warp's 32 reads of one
// pair's row land on a few neighbouring lags: broadcasts and distinct banks
// instead of bank conflicts.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cstring>
#include <cmath>
#include <vector>

#include "fcc_doa.h"
#include "fcc_internal.h"

struct fcc_doa {
    fcc_plan *plan = nullptr;
    int device = 0;         // the plan's device, kept so that destroy never reads the plan
    int D = 0, P = 0, I = 0;
    int F = 1, per_sm = 1;  // frames per search tile, resident search CTAs per SM
    int2 *d_tab = nullptr;  // [P][D] in search order: (k, bits of w), position k + w on the lag grid
    int *d_orig = nullptr;  // [D]: the caller's index of each candidate in search order
};

namespace fcc {
namespace {

constexpr int kSrpThreads = 256;
constexpr int kQB = 8;  // pairs per batch of table loads
constexpr size_t kSrpSmemBudget = 100 * 1024;  // two or more CTAs per SM
constexpr size_t kDoaChunkBytes = 256u << 20;  // correlations of one chunk of fcc_tdoa_doa

struct SrpParams {
    const float *corr;  // [T][P][I]
    long long T;
    int P, I, D;
    const int2 *tab;    // [P][D]
    const int *orig;    // [D]
    int *out_idx;
    float *out_score;
    unsigned *err;
};

template <int F>
__global__ void __launch_bounds__(kSrpThreads) srp_kernel(const __grid_constant__ SrpParams p)
{
    extern __shared__ __align__(16) float2 tile[];  // [F][P][I]: (y_k, y_{k+1} - y_k)
    __shared__ float red_s[kSrpThreads / 32][F];
    __shared__ int red_i[kSrpThreads / 32][F];
    const int PI = p.P * p.I;
    const long long n_tiles = (p.T + F - 1) / F;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    bool bad = false;
    for (long long tl = blockIdx.x; tl < n_tiles; tl += gridDim.x) {
        const long long t0 = tl * F;
        const int nf = (int)min((long long)F, p.T - t0);
        __syncthreads();  // the previous tile's reads are done
        const float *src = p.corr + (size_t)t0 * PI;
        // k = e mod I, stepped without a division (blockDim.x mod I < I: one wrap at most)
        const int step_k = (int)blockDim.x % p.I, lim = nf * PI;
        int k = (int)threadIdx.x % p.I;
        for (int e = threadIdx.x; e < F * PI; e += blockDim.x) {
            float y = 0.f, dy = 0.f;
            if (e < lim) {
                y = __ldg(src + e);
                dy = k + 1 < p.I ? __ldg(src + e + 1) - y : 0.f;
            }
            tile[e] = make_float2(y, dy);
            k += step_k;
            if (k >= p.I) k -= p.I;
        }
        __syncthreads();
        float best[F];
        int bidx[F];
#pragma unroll
        for (int f = 0; f < F; ++f) {
            best[f] = -FLT_MAX;
            bidx[f] = INT_MAX;
        }
        for (int d0 = 0; d0 < p.D; d0 += blockDim.x) {
            const int d = d0 + threadIdx.x;
            if (d < p.D) {
                float acc[F];
#pragma unroll
                for (int f = 0; f < F; ++f) acc[f] = 0.f;
                const int o = __ldg(p.orig + d);
                const int2 *tb = p.tab + d;
                // the grid positions come from L2: the next kQB pairs' entries are in
                // flight while the current kQB pairs are summed
                int2 cur[kQB];
#pragma unroll
                for (int u = 0; u < kQB; ++u) cur[u] = u < p.P ? __ldg(tb + (size_t)u * p.D) : make_int2(0, 0);
                for (int q0 = 0; q0 < p.P; q0 += kQB) {
                    int2 nxt[kQB];
#pragma unroll
                    for (int u = 0; u < kQB; ++u)
                        nxt[u] = q0 + kQB + u < p.P ? __ldg(tb + (size_t)(q0 + kQB + u) * p.D) : make_int2(0, 0);
#pragma unroll
                    for (int u = 0; u < kQB; ++u) {
                        if (q0 + u < p.P) {
                            const float w = __int_as_float(cur[u].y);
                            const float2 *col = tile + (q0 + u) * p.I + cur[u].x;
#pragma unroll
                            for (int f = 0; f < F; ++f) {
                                const float2 v = col[f * PI];
                                acc[f] += fmaf(w, v.y, v.x);
                            }
                        }
                        cur[u] = nxt[u];
                    }
                }
#pragma unroll
                for (int f = 0; f < F; ++f) {
                    bad = bad || !(fabsf(acc[f]) <= FLT_MAX);
                    if (acc[f] > best[f] || (acc[f] == best[f] && o < bidx[f])) {
                        best[f] = acc[f];
                        bidx[f] = o;
                    }
                }
            }
        }
        // per frame: the CTA's maximum, lowest index on ties
#pragma unroll
        for (int f = 0; f < F; ++f) {
            float s = best[f];
            int i = bidx[f];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float os = __shfl_xor_sync(0xffffffffu, s, off);
                const int oi = __shfl_xor_sync(0xffffffffu, i, off);
                if (os > s || (os == s && oi < i)) {
                    s = os;
                    i = oi;
                }
            }
            if (lane == 0) {
                red_s[warp][f] = s;
                red_i[warp][f] = i;
            }
        }
        __syncthreads();
        if (threadIdx.x < nf) {
            const int f = threadIdx.x;
            float s = red_s[0][f];
            int i = red_i[0][f];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (red_s[w][f] > s || (red_s[w][f] == s && red_i[w][f] < i)) {
                    s = red_s[w][f];
                    i = red_i[w][f];
                }
            p.out_idx[t0 + f] = i == INT_MAX ? -1 : i;
            p.out_score[t0 + f] = s;
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(p.err, kErrNonFinite);
}

int srp_frames(int P, int I)
{
    const size_t per = (size_t)P * I * sizeof(float2);
    int F = 16;
    while (F > 1 && (size_t)F * per > kSrpSmemBudget) F >>= 1;
    return F;
}

template <int F>
fcc_status_t launch_srp_f(const SrpParams &prm, int num_sms, cudaStream_t st)
{
    const size_t smem = (size_t)F * prm.P * prm.I * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(srp_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(srp_kernel)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, srp_kernel<F>, kSrpThreads, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm < 1) return fail(FCC_ERR_UNSUPPORTED, "the lag grid of one frame does not fit in shared memory");
    const long long tiles = (prm.T + F - 1) / F;
    const int grid = (int)std::min<long long>(tiles, (long long)num_sms * per_sm);
    srp_kernel<F><<<grid, kSrpThreads, smem, st>>>(prm);
    e = cudaGetLastError();
    return e == cudaSuccess ? FCC_OK : cuda_fail(e, "srp_kernel launch");
}

fcc_status_t launch_srp(const fcc_doa *doa, const float *corr, long long T, int *idx, float *score, cudaStream_t st)
{
    SrpParams prm{};
    prm.corr = corr;
    prm.T = T;
    prm.P = doa->P;
    prm.I = doa->I;
    prm.D = doa->D;
    prm.tab = doa->d_tab;
    prm.orig = doa->d_orig;
    prm.out_idx = idx;
    prm.out_score = score;
    prm.err = doa->plan->d_err;
    switch (srp_frames(doa->P, doa->I)) {
    case 16: return launch_srp_f<16>(prm, doa->plan->num_sms, st);
    case 8: return launch_srp_f<8>(prm, doa->plan->num_sms, st);
    case 4: return launch_srp_f<4>(prm, doa->plan->num_sms, st);
    case 2: return launch_srp_f<2>(prm, doa->plan->num_sms, st);
    default: return launch_srp_f<1>(prm, doa->plan->num_sms, st);
    }
}

// Frames per chunk of fcc_tdoa_doa: whole waves of the search grid (every
// resident search CTA takes the same number of tiles) within the byte budget.
long long doa_chunk_frames(const fcc_doa *doa)
{
    const long long per = (long long)doa->P * doa->I * 4;
    const long long wave = (long long)doa->plan->num_sms * doa->per_sm * doa->F;
    return std::max<long long>(1, (long long)kDoaChunkBytes / per / wave) * wave;
}

// Order candidates so that consecutive runs of 32 are compact patches: split
// the set at the median of its widest coordinate, recursively, cutting at
// multiples of 32.
void patch_order(const double *dirs, std::vector<int> &idx, int lo, int hi)
{
    if (hi - lo <= 32) return;
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int e = lo; e < hi; ++e)
        for (int a = 0; a < 3; ++a) {
            mn[a] = std::min(mn[a], dirs[3 * (size_t)idx[e] + a]);
            mx[a] = std::max(mx[a], dirs[3 * (size_t)idx[e] + a]);
        }
    int ax = 0;
    for (int a = 1; a < 3; ++a)
        if (mx[a] - mn[a] > mx[ax] - mn[ax]) ax = a;
    const int n = hi - lo, groups = (n + 31) / 32;
    const int mid = lo + std::min(n, (groups / 2) * 32);
    std::nth_element(idx.begin() + lo, idx.begin() + mid, idx.begin() + hi, [&](int a, int b) {
        const double va = dirs[3 * (size_t)a + ax], vb = dirs[3 * (size_t)b + ax];
        return va < vb || (va == vb && a < b);
    });
    patch_order(dirs, idx, lo, mid);
    patch_order(dirs, idx, mid, hi);
}

template <int F>
int srp_per_sm(const fcc_doa *doa)
{
    const size_t smem = (size_t)F * doa->P * doa->I * sizeof(float2);
    if (cudaFuncSetAttribute(srp_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, srp_kernel<F>, kSrpThreads, smem) != cudaSuccess)
        return 0;
    return per_sm;
}

int srp_occupancy(const fcc_doa *doa)
{
    switch (doa->F) {
    case 16: return srp_per_sm<16>(doa);
    case 8: return srp_per_sm<8>(doa);
    case 4: return srp_per_sm<4>(doa);
    case 2: return srp_per_sm<2>(doa);
    default: return srp_per_sm<1>(doa);
    }
}

}  // namespace
}  // namespace fcc

using namespace fcc;

extern "C" {

fcc_status_t fcc_doa_create(fcc_plan_t *plan, const double *mic_xyz, const double *dirs, int n_dirs, fcc_doa_t **out)
{
    if (!out) return fail(FCC_ERR_INVALID_ARG, "null output");
    *out = nullptr;
    if (!plan || !mic_xyz || !dirs) return fail(FCC_ERR_INVALID_ARG, "null plan/mic_xyz/dirs");
    if (n_dirs < 1) return fail(FCC_ERR_INVALID_ARG, "n_dirs < 1");
    const fcc_plan_info_t &in = plan->info;
    const int M = in.M, P = in.P, I = in.I, D = n_dirs;
    if (I < 2) return fail(FCC_ERR_UNSUPPORTED, "a lag grid of one point");
    for (int e = 0; e < 3 * M; ++e)
        if (!std::isfinite(mic_xyz[e])) return fail(FCC_ERR_INVALID_ARG, "non-finite mic_xyz");
    for (long long e = 0; e < 3LL * D; ++e)
        if (!std::isfinite(dirs[e])) return fail(FCC_ERR_INVALID_ARG, "non-finite direction");
    std::vector<int> order(D);
    for (int d = 0; d < D; ++d) order[d] = d;
    patch_order(dirs, order, 0, D);
    // grid position of tau_ij(u) = -(fs / c) (r_i - r_j) . u, clamped to the grid,
    // for the candidates in search order
    std::vector<int2> tab((size_t)P * D);
    const double scale = in.fs / in.c;
    for (int d = 0; d < D; ++d) {
        const double *u = dirs + 3 * (size_t)order[d];
        int q = 0;
        for (int i = 0; i < M; ++i)
            for (int j = i + 1; j < M; ++j, ++q) {
                const double *ri = mic_xyz + 3 * i, *rj = mic_xyz + 3 * j;
                const double tau = -scale * ((ri[0] - rj[0]) * u[0] + (ri[1] - rj[1]) * u[1] + (ri[2] - rj[2]) * u[2]);
                const double pos = std::min((double)(I - 1), std::max(0.0, (tau + in.L) * in.den));
                const int k = std::min(I - 2, (int)std::floor(pos));
                const float w = (float)(pos - k);
                int wb;
                std::memcpy(&wb, &w, 4);
                tab[(size_t)q * D + d] = make_int2(k, wb);
            }
    }
    DeviceScope scope(plan->device);
    if (!scope.ok) return fail(FCC_ERR_CUDA, "cudaSetDevice failed");
    fcc_doa *doa = new (std::nothrow) fcc_doa;
    if (!doa) return fail(FCC_ERR_OOM, "host allocation");
    doa->plan = plan;
    doa->device = plan->device;
    doa->D = D;
    doa->P = P;
    doa->I = I;
    doa->F = srp_frames(P, I);
    doa->per_sm = srp_occupancy(doa);
    if (doa->per_sm < 1) {
        delete doa;
        return fail(FCC_ERR_UNSUPPORTED, "the lag grid of one frame does not fit in shared memory");
    }
    cudaError_t e = cudaMalloc(&doa->d_tab, tab.size() * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc(&doa->d_orig, (size_t)D * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(doa->d_tab, tab.data(), tab.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(doa->d_orig, order.data(), (size_t)D * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(doa->d_tab);
        cudaFree(doa->d_orig);
        delete doa;
        return e == cudaErrorMemoryAllocation ? fail(FCC_ERR_OOM, "cudaMalloc(doa tables)") : cuda_fail(e, "doa tables");
    }
    *out = doa;
    return FCC_OK;
}

void fcc_doa_destroy(fcc_doa_t *doa)
{
    if (!doa) return;
    DeviceScope scope(doa->device);
    cudaFree(doa->d_tab);
    cudaFree(doa->d_orig);
    delete doa;
}

fcc_status_t fcc_doa_search(fcc_doa_t *doa, const float *d_corr, long long T, int *d_dir_idx, float *d_score,
                            void *stream)
{
    if (!doa) return fail(FCC_ERR_INVALID_ARG, "null search object");
    if (T < 0) return fail(FCC_ERR_INVALID_ARG, "T < 0");
    if (T == 0) return FCC_OK;
    if (!d_corr || !d_dir_idx || !d_score) return fail(FCC_ERR_INVALID_ARG, "null corr/dir_idx/score");
    if ((reinterpret_cast<uintptr_t>(d_corr) & 15) ||
        ((reinterpret_cast<uintptr_t>(d_dir_idx) | reinterpret_cast<uintptr_t>(d_score)) & 3))
        return fail(FCC_ERR_INVALID_ARG, "misaligned buffer");
    DeviceScope scope(doa->plan->device);
    if (!scope.ok) return fail(FCC_ERR_CUDA, "cudaSetDevice failed");
    return launch_srp(doa, d_corr, T, d_dir_idx, d_score, static_cast<cudaStream_t>(stream));
}

fcc_status_t fcc_doa_workspace(const fcc_doa_t *doa, long long T, long long *bytes)
{
    if (!doa || !bytes) return fail(FCC_ERR_INVALID_ARG, "null argument");
    if (T < 0) return fail(FCC_ERR_INVALID_ARG, "T < 0");
    const long long ch = std::min<long long>(doa_chunk_frames(doa), std::max<long long>(T, 1));
    // correlations, then per-pair lag index and peak (16-byte aligned pieces)
    const long long corr = (ch * doa->P * doa->I * 4 + 15) / 16 * 16;
    const long long pp = (ch * doa->P * 4 + 15) / 16 * 16;
    *bytes = T == 0 ? 0 : corr + 2 * pp;
    return FCC_OK;
}

fcc_status_t fcc_tdoa_doa(fcc_doa_t *doa, const void *d_spectra, long long T, int *d_dir_idx, float *d_score,
                          int *d_lag_idx, float *d_peak, void *d_work, long long work_bytes, void *stream)
{
    if (!doa) return fail(FCC_ERR_INVALID_ARG, "null search object");
    if (T < 0) return fail(FCC_ERR_INVALID_ARG, "T < 0");
    if (T == 0) return FCC_OK;
    if (!d_spectra || !d_dir_idx || !d_score || !d_work) return fail(FCC_ERR_INVALID_ARG, "null argument");
    if ((reinterpret_cast<uintptr_t>(d_spectra) | reinterpret_cast<uintptr_t>(d_work)) & 15)
        return fail(FCC_ERR_INVALID_ARG, "spectra / workspace not 16-byte aligned");
    if ((reinterpret_cast<uintptr_t>(d_dir_idx) | reinterpret_cast<uintptr_t>(d_score) |
         reinterpret_cast<uintptr_t>(d_lag_idx) | reinterpret_cast<uintptr_t>(d_peak)) & 3)
        return fail(FCC_ERR_INVALID_ARG, "output not 4-byte aligned");
    long long need = 0;
    fcc_status_t st = fcc_doa_workspace(doa, T, &need);
    if (st != FCC_OK) return st;
    if (work_bytes < need) return fail(FCC_ERR_INVALID_ARG, "workspace too small");
    fcc_plan *plan = doa->plan;
    if (!plan->kh) return fail(FCC_ERR_UNSUPPORTED, "more than 8 bases of one parity");
    DeviceScope scope(plan->device);
    if (!scope.ok) return fail(FCC_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long ch = std::min(doa_chunk_frames(doa), T);
    const int P = doa->P;
    unsigned char *w = static_cast<unsigned char *>(d_work);
    float *corr = reinterpret_cast<float *>(w);
    const long long corr_b = (ch * P * doa->I * 4 + 15) / 16 * 16, pp = (ch * P * 4 + 15) / 16 * 16;
    int *w_idx = reinterpret_cast<int *>(w + corr_b);
    float *w_peak = reinterpret_cast<float *>(w + corr_b + pp);
    const size_t frame_elems = (size_t)plan->info.M * plan->info.B;
    for (long long t0 = 0; t0 < T; t0 += ch) {
        const long long n = std::min(ch, T - t0);
        const float2 *X = static_cast<const float2 *>(d_spectra) + (size_t)t0 * frame_elems;
        int *li = d_lag_idx ? d_lag_idx + (size_t)t0 * P : w_idx;
        float *pk = d_peak ? d_peak + (size_t)t0 * P : w_peak;
        st = launch_tdoa(plan, X, n, li, pk, nullptr, nullptr, corr, s);
        if (st != FCC_OK) return st;
        st = launch_srp(doa, corr, n, d_dir_idx + t0, d_score + t0, s);
        if (st != FCC_OK) return st;
    }
    return FCC_OK;
}

}  // extern "C"
