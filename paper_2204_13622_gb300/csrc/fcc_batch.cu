// fcc_batch.cu -- batched FCC over many independent arrays (include/fcc_batch.h).
//
// Host runtime: one FP32 plan per array (bases shared through the plan cache),
// optional tile autotuning per distinct (M, N, K, I), jobs cut from each array's
// frame tiles and ordered largest first, and one CUDA graph captured at create:
//   * by default arrays grouped into kernel classes (KH, RS), one persistent
//     launch per class (each with the class's own warp count and register
//     budget), the classes as independent branches of the graph;
//   * with FCC_BATCH_SINGLE_LAUNCH one persistent launch (fcc_batch_all.cu) whose
//     CTAs take every job of every array from one queue; each job names its
//     kernel instance (KH, RS), and the arrays' geometries are limited to that
//     kernel's eight compute warps (one register budget, the largest class's).
// Binding buffers only rewrites the per-array parameter table the kernels read,
// so the graph is captured once.
#include <algorithm>
#include <cstdio>
#include <map>
#include <new>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "fcc_batch.h"
#include "fcc_internal.h"

namespace fcc {
fcc_status_t tune_fp32(fcc_plan *plan, const std::string &path, bool force, int max_cand, double *us_out,
                       int max_warps = 0);
std::string tune_cache_path(const char *p);
}  // namespace fcc

using namespace fcc;

struct fcc_batch {
    struct Class {
        int kh = 0, rs = 0, grid = 0, n_jobs = 0;  // kh = 0: every array, the single launch
        size_t smem = 0;
        std::vector<int> arrays;
        BatchJob *d_jobs = nullptr;
        int *d_counter = nullptr;
        cudaStream_t stream = nullptr;
        cudaEvent_t done = nullptr;
    };
    int device = 0, num_sms = 0;
    std::vector<fcc_plan_t *> plans;
    std::vector<long long> T;
    std::vector<Class> classes;
    Fp32Params *d_arrays = nullptr;
    unsigned *d_err = nullptr;
    cudaStream_t cap = nullptr;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool bound = false;
    bool single = false;  // one persistent launch for every array
    fcc_batch_info_t info{};
};

namespace {

void free_batch(fcc_batch *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto &c : b->classes) {
        cudaFree(c.d_jobs);
        cudaFree(c.d_counter);
        if (c.stream) cudaStreamDestroy(c.stream);
        if (c.done) cudaEventDestroy(c.done);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaFree(b->d_arrays);
    cudaFree(b->d_err);
    for (auto *p : b->plans) fcc_plan_destroy(p);
    delete b;
}

// Cut each array of a class into jobs of whole tiles: about 8 jobs per CTA of
// bytes, at least two tiles per group when the array has them, one array per
// job; the CTAs take them largest first.
std::vector<BatchJob> make_jobs(const fcc_batch *b, const fcc_batch::Class &c, int grid)
{
    double total = 0;
    for (int a : c.arrays) {
        const fcc_plan_info_t &in = b->plans[a]->info;
        total += (double)b->T[a] * in.M * in.B * 8.0;
    }
    const double target = std::max(total / (grid * 8.0), 1.0);
    std::vector<std::pair<double, BatchJob>> jobs;
    for (int a : c.arrays) {
        const fcc_plan *p = b->plans[a];
        const Fp32Geometry &g = p->geo;
        const double tile_bytes = (double)g.F * p->info.M * p->info.B * 8.0;
        const long long n_tiles = (b->T[a] + g.F - 1) / g.F;
        long long per = std::max<long long>((long long)(target / tile_bytes), 2LL * g.G);
        per = std::min(per, n_tiles);
        const long long nj = (n_tiles + per - 1) / per;
        const long long even = (n_tiles + nj - 1) / nj;
        for (long long t0 = 0; t0 < n_tiles; t0 += even) {
            const long long nt = std::min(even, n_tiles - t0);
            const long long frames = std::min<long long>(nt * g.F, b->T[a] - t0 * g.F);
            const int rs = fp32_row_slots(p->info.Q);
            const int code = 4 * (p->kh / 2 - 1) + (rs == 1 ? 0 : rs == 2 ? 1 : rs == 4 ? 2 : 3);
            jobs.push_back({(double)frames * p->info.M * p->info.B * 8.0, BatchJob{a, (int)t0, (int)nt, code}});
        }
    }
    std::stable_sort(jobs.begin(), jobs.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
    std::vector<BatchJob> out;
    for (auto &j : jobs) out.push_back(j.second);
    return out;
}

fcc_status_t capture_graph(fcc_batch *b)
{
    for (auto &c : b->classes) {
        BatchParams bp{};
        fcc_status_t st = c.kh ? launch_fp32_batch(c.kh, c.rs, bp, 0, 0, nullptr)  // prepare
                               : launch_fp32_batch_all(bp, 0, 0, nullptr);
        if (st != FCC_OK) return st;
    }
    FCC_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    fcc_status_t st = FCC_OK;
    cudaError_t e = cudaEventRecord(b->fork, b->cap);
    for (auto &c : b->classes) {
        if (e != cudaSuccess || st != FCC_OK) break;
        e = cudaStreamWaitEvent(c.stream, b->fork, 0);
        if (e == cudaSuccess) e = cudaMemsetAsync(c.d_counter, 0, sizeof(int), c.stream);
        if (e == cudaSuccess) {
            BatchParams bp{b->d_arrays, c.d_jobs, c.n_jobs, c.d_counter};
            st = c.kh ? launch_fp32_batch(c.kh, c.rs, bp, c.grid, c.smem, c.stream)
                      : launch_fp32_batch_all(bp, c.grid, c.smem, c.stream);
        }
        if (e == cudaSuccess && st == FCC_OK) e = cudaEventRecord(c.done, c.stream);
        if (e == cudaSuccess && st == FCC_OK) e = cudaStreamWaitEvent(b->cap, c.done, 0);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    if (st != FCC_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(e != cudaSuccess ? e : e2, "batch graph capture");
    }
    b->graph = g;
    FCC_CUDA_TRY(cudaGraphInstantiate(&b->exec, g, 0));
    return FCC_OK;
}

}  // namespace

extern "C" {

fcc_status_t fcc_batch_create(const fcc_plan_desc_t *descs, const long long *T, int n_arrays, int device, int flags,
                              const char *tune_cache, fcc_batch_t **out)
{
    if (!descs || !T || !out) return fail(FCC_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (n_arrays < 1) return fail(FCC_ERR_INVALID_ARG, "n_arrays < 1");
    int dev = device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return fail(FCC_ERR_CUDA, "no CUDA device");
    DeviceScope scope(dev);
    if (!scope.ok) return fail(FCC_ERR_CUDA, "cudaSetDevice failed");
    for (int a = 0; a < n_arrays; ++a) {
        if (descs[a].prec != FCC_PREC_FP32)
            return fail(FCC_ERR_INVALID_ARG, "array " + std::to_string(a) + ": the batched form is FP32");
        if (descs[a].form != FCC_FORM_FOLDED)
            return fail(FCC_ERR_UNSUPPORTED, "array " + std::to_string(a) + ": the batched form is the folded one");
        if (T[a] < 1) return fail(FCC_ERR_INVALID_ARG, "array " + std::to_string(a) + ": T < 1");
    }
    fcc_batch *b = new (std::nothrow) fcc_batch();
    if (!b) return fail(FCC_ERR_OOM, "host allocation");
    b->device = dev;
    b->single = (flags & FCC_BATCH_SINGLE_LAUNCH) != 0;
    const int cap = b->single ? kBatchAllWarps : 0;  // compute warps an array's geometry may use
    cudaError_t e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e, "cudaDeviceGetAttribute");
    }
    const std::string cache = tune_cache_path(tune_cache);
    std::map<std::string, fcc_plan *> tuned;  // tune key -> representative
    std::set<std::tuple<int, int, int, int, int>> bases;
    for (int a = 0; a < n_arrays; ++a) {
        fcc_plan_desc_t d = descs[a];
        d.device = dev;
        fcc_plan_t *p = nullptr;
        fcc_status_t st = fcc_plan_create(&d, &p);
        if (st != FCC_OK) {
            const std::string msg = "array " + std::to_string(a) + ": " + fcc_last_error();
            free_batch(b);
            return fail(st, msg);
        }
        b->plans.push_back(p);
        b->T.push_back(T[a]);
        if (!p->kh || p->geo.G == 0) {
            free_batch(b);
            return fail(FCC_ERR_UNSUPPORTED, "array " + std::to_string(a) + ": no FP32 kernel (N > 1024 or K > 16)");
        }
        const fcc_plan_info_t &in = p->info;
        bases.insert({in.N, in.I, in.den, in.K_even, in.K_odd});
        if (flags & FCC_BATCH_AUTOTUNE) {
            char key[128];
            std::snprintf(key, sizeof key, "%d|%d|%d|%d|%d", in.M, in.N, in.K_even, in.K_odd, in.I);
            auto it = tuned.find(key);
            if (it == tuned.end()) {
                st = tune_fp32(p, cache, false, 0, nullptr, cap);
                if (st != FCC_OK) {
                    const std::string msg = "array " + std::to_string(a) + ": " + fcc_last_error();
                    free_batch(b);
                    return fail(st, msg);
                }
                tuned[key] = p;
            } else if (!same_geometry(p->geo, it->second->geo)) {
                st = set_fp32_geometry(p, it->second->geo);
                if (st != FCC_OK) {
                    free_batch(b);
                    return st;
                }
            }
        } else if (cap && p->geo.G * p->geo.GW > cap) {
            // the single launch's eight warps: the best heuristic geometry within
            // them, with the same chunk count (so the per-frame arithmetic, and the
            // results, are those of fcc_tdoa with the plan's own geometry)
            std::vector<Fp32Geometry> cand;
            st = fp32_candidates(p, cand, cap);
            const Fp32Geometry *pick = nullptr;
            for (const Fp32Geometry &g : cand)
                if (!pick && g.C == p->geo.C) pick = &g;
            if (!pick && !cand.empty()) pick = &cand[0];
            if (st == FCC_OK && !pick) st = fail(FCC_ERR_UNSUPPORTED, "no geometry within the batched kernel's warps");
            if (st == FCC_OK) st = set_fp32_geometry(p, *pick);
            if (st != FCC_OK) {
                const std::string msg = "array " + std::to_string(a) + ": " + fcc_last_error();
                free_batch(b);
                return fail(st, msg);
            }
        }
    }
    // classes
    std::map<std::pair<int, int>, int> cls;
    for (int a = 0; a < n_arrays; ++a) {
        const fcc_plan *p = b->plans[a];
        const auto key = std::make_pair(p->kh, fp32_row_slots(p->info.Q));
        auto it = cls.find(key);
        if (it == cls.end()) {
            it = cls.emplace(key, (int)b->classes.size()).first;
            b->classes.emplace_back();
            b->classes.back().kh = key.first;
            b->classes.back().rs = key.second;
        }
        b->classes[it->second].arrays.push_back(a);
    }
    fcc_batch_info_t &inf = b->info;
    inf.n_arrays = n_arrays;
    inf.n_classes = (int)b->classes.size();
    inf.n_launches = b->single ? 1 : (int)b->classes.size();
    if (b->single) {
        fcc_batch::Class all;
        for (int a = 0; a < n_arrays; ++a) all.arrays.push_back(a);
        b->classes.clear();
        b->classes.push_back(all);
    }
    inf.n_bases = (int)bases.size();
    for (int a = 0; a < n_arrays; ++a) {
        const fcc_plan_info_t &in = b->plans[a]->info;
        inf.frames += T[a];
        inf.pair_frames += T[a] * in.P;
        inf.spectra_bytes += (double)T[a] * in.M * in.B * 8.0;
        inf.result_bytes += (double)T[a] * in.P * 8.0;
    }
    e = cudaMalloc(&b->d_arrays, sizeof(Fp32Params) * n_arrays);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (auto &c : b->classes) {
        if (e != cudaSuccess) break;
        size_t smem = 0;
        for (int a : c.arrays) smem = std::max(smem, b->plans[a]->geo.smem_bytes);
        c.smem = kBatchHeaderBytes + smem;
        std::vector<BatchJob> jobs = make_jobs(b, c, b->num_sms);
        c.n_jobs = (int)jobs.size();
        c.grid = std::min(b->num_sms, c.n_jobs);
        inf.n_jobs += c.n_jobs;
        e = cudaMalloc(&c.d_jobs, sizeof(BatchJob) * jobs.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(c.d_jobs, jobs.data(), sizeof(BatchJob) * jobs.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&c.d_counter, sizeof(int));
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e, "batch tables");
    }
    fcc_status_t st = capture_graph(b);
    if (st != FCC_OK) {
        free_batch(b);
        return st;
    }
    *out = b;
    return FCC_OK;
}

void fcc_batch_destroy(fcc_batch_t *b)
{
    if (!b) return;
    DeviceScope scope(b->device);
    cudaDeviceSynchronize();
    free_batch(b);
}

fcc_status_t fcc_batch_info(const fcc_batch_t *b, fcc_batch_info_t *info)
{
    if (!b || !info) return fail(FCC_ERR_INVALID_ARG, "null argument");
    *info = b->info;
    return FCC_OK;
}

fcc_status_t fcc_batch_array_info(const fcc_batch_t *b, int a, fcc_plan_info_t *info)
{
    if (!b || !info) return fail(FCC_ERR_INVALID_ARG, "null argument");
    if (a < 0 || a >= (int)b->plans.size()) return fail(FCC_ERR_INVALID_ARG, "array index out of range");
    *info = b->plans[a]->info;
    return FCC_OK;
}

fcc_status_t fcc_batch_bind(fcc_batch_t *b, const void *const *d_spectra, int *const *d_lag_idx,
                            float *const *d_peak, float *const *d_tau_hat)
{
    if (!b || !d_spectra || !d_lag_idx || !d_peak) return fail(FCC_ERR_INVALID_ARG, "null argument");
    DeviceScope scope(b->device);
    if (!scope.ok) return fail(FCC_ERR_CUDA, "cudaSetDevice failed");
    const int n = (int)b->plans.size();
    std::vector<Fp32Params> h(n);
    bool any_tau = false;
    for (int a = 0; a < n; ++a) {
        const std::string where = "array " + std::to_string(a) + ": ";
        if (!d_spectra[a] || !d_lag_idx[a] || !d_peak[a]) return fail(FCC_ERR_INVALID_ARG, where + "null buffer");
        if (reinterpret_cast<uintptr_t>(d_spectra[a]) & 15)
            return fail(FCC_ERR_INVALID_ARG, where + "spectra not 16-byte aligned");
        float *tau = d_tau_hat ? d_tau_hat[a] : nullptr;
        any_tau = any_tau || tau;
        if ((reinterpret_cast<uintptr_t>(d_lag_idx[a]) | reinterpret_cast<uintptr_t>(d_peak[a]) |
             reinterpret_cast<uintptr_t>(tau)) & 3)
            return fail(FCC_ERR_INVALID_ARG, where + "output not 4-byte aligned");
        h[a] = make_fp32_params(b->plans[a], static_cast<const float2 *>(d_spectra[a]), b->T[a], d_lag_idx[a],
                                d_peak[a], tau, nullptr, nullptr, b->d_err);
    }
    FCC_CUDA_TRY(cudaDeviceSynchronize());  // no run may read the table while it changes
    FCC_CUDA_TRY(cudaMemcpy(b->d_arrays, h.data(), sizeof(Fp32Params) * n, cudaMemcpyHostToDevice));
    b->info.result_bytes = 0;
    for (int a = 0; a < n; ++a)
        b->info.result_bytes += (double)b->T[a] * b->plans[a]->info.P * ((d_tau_hat && d_tau_hat[a]) ? 12.0 : 8.0);
    (void)any_tau;
    b->bound = true;
    return FCC_OK;
}

fcc_status_t fcc_batch_run(fcc_batch_t *b, void *stream)
{
    if (!b) return fail(FCC_ERR_INVALID_ARG, "null batch");
    if (!b->bound) return fail(FCC_ERR_INVALID_ARG, "fcc_batch_bind has not been called");
    DeviceScope scope(b->device);
    if (!scope.ok) return fail(FCC_ERR_CUDA, "cudaSetDevice failed");
    FCC_CUDA_TRY(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)));
    return FCC_OK;
}

fcc_status_t fcc_batch_sync(fcc_batch_t *b, void *stream)
{
    if (!b) return fail(FCC_ERR_INVALID_ARG, "null batch");
    DeviceScope scope(b->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    FCC_CUDA_TRY(cudaStreamSynchronize(st));
    unsigned err = 0;
    FCC_CUDA_TRY(cudaMemcpyAsync(&err, b->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    FCC_CUDA_TRY(cudaMemsetAsync(b->d_err, 0, sizeof(unsigned), st));
    FCC_CUDA_TRY(cudaStreamSynchronize(st));
    if (err & kErrTimeout) return fail(FCC_ERR_TIMEOUT, "a device-side wait expired");
    if (err & kErrNonFinite) return fail(FCC_ERR_NONFINITE, "NaN or Inf in the spectra");
    return FCC_OK;
}

}  // extern "C"
