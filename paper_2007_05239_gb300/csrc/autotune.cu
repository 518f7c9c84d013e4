// ml_fastsum_plan_autotune: the spreading tile (bin) edge of a layer's plan
// chosen by timing, with a per-shape cache.
//
// The bin edge B sets the padded shared-memory tile (B + W)^d of the
// spreading and interpolation kernels, hence the CTAs per SM, the number of
// subproblems (CTAs per launch) and the halo overhead of the fold.  The
// automatic rule picks it from a shared-memory budget; the best edge also
// depends on how the points fill the grid, which only a measurement sees.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ml_internal.h"

namespace ml {
namespace {

std::mutex g_tune_mu;
std::map<std::string, int> g_tune_cache;   // layer shape -> chosen bin edge

std::string shape_key(const ml_plan_info &in, int nv)
{
    const int lg = (int)std::floor(std::log2((double)std::max<int64_t>(in.n, 1)));
    return std::to_string(in.d) + "/" + std::to_string(in.prec) + "/" + std::to_string(in.taps) + "/" +
           std::to_string(in.n_os) + "/" + std::to_string(in.N) + "/" + std::to_string(in.L[0]) + "x" +
           std::to_string(in.L[1]) + "x" + std::to_string(in.L[2]) + "/" + std::to_string(nv) + "/" +
           std::to_string(lg);
}

// SplitMix64 of a counter, mapped to [0, 1)
__global__ void k_tune_fill(double *x, int64_t count)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = (uint64_t)(e + 1) * 0x9E3779B97F4A7C15ULL;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z = z ^ (z >> 31);
        x[e] = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    }
}

// average time (ms) of one nv-vector product on this plan (its work counter
// is left as it was)
ml_status time_plan(ml_plan_t plan, const double *X, double *Y, int nv, cudaStream_t st, float *ms)
{
    struct Keep {
        ml_plan_t p;
        int64_t applied;
        ~Keep() { p->applied = applied; }
    } keep{plan, plan->applied};
    ML_TRY(ml_fastsum_apply(&plan, 1, X, nv, Y, ML_RAW_W, st));   // untimed: workspace, caches
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ML_CUDA(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ce, "cudaEventCreate", __FILE__, __LINE__);
    }
    constexpr int kReps = 3;
    ml_status s = ML_OK;
    cudaEventRecord(e0, st);
    for (int r = 0; r < kReps && s == ML_OK; ++r) s = ml_fastsum_apply(&plan, 1, X, nv, Y, ML_RAW_W, st);
    cudaEventRecord(e1, st);
    ce = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != ML_OK) return s;
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaEventElapsedTime", __FILE__, __LINE__);
    *ms = t / kReps;
    return ML_OK;
}

}  // namespace
}  // namespace ml

extern "C" ml_status ml_fastsum_plan_autotune(ml_plan_t *out, const double *points, int64_t n, int d, double sigma,
                                              const ml_plan_params *params, int nv, int *bin_chosen, void *stream)
{
    using namespace ml;
    if (!out) return fail(ML_ERR_ARG, "out is null");
    *out = nullptr;
    if (!params) return fail(ML_ERR_ARG, "params is null");
    if (nv < 1 || nv > kMaxVec) return fail(ML_ERR_ARG, "nv must be in [1, 8]");
    cudaStream_t st = (cudaStream_t)stream;
    ml_plan_params prm = *params;
    prm.bin = 0;
    ml_plan_t base = nullptr;
    ML_TRY(ml_fastsum_plan_ex(&base, points, n, d, sigma, &prm, stream));
    ml_plan_info info;
    ml_plan_get_info(base, &info);
    const std::string key = shape_key(info, nv);
    int cached = 0;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) cached = it->second;
    }
    if (info.nbins == 1 || cached == info.bin) {
        // a single tile (nothing to tune), or the rule's edge already won
        if (bin_chosen) *bin_chosen = info.bin;
        *out = base;
        return ML_OK;
    }
    if (cached > 0) {
        prm.bin = cached;
        ml_plan_t p = nullptr;
        const ml_status s = ml_fastsum_plan_ex(&p, points, n, d, sigma, &prm, stream);
        if (s == ML_OK) {
            ml_plan_destroy(base);
            if (bin_chosen) *bin_chosen = cached;
            *out = p;
            return ML_OK;
        }
    }
    // candidates around the rule's edge (those beyond the shared-memory budget
    // are refused by the plan and skipped)
    const int B0 = info.bin;
    std::vector<int> cand;
    for (int b : {B0 - 2, B0 - 1, B0 + 1, B0 + 2, B0 + 4})
        if (b >= 2 && b != B0) cand.push_back(b);
    DevBuf X, Y;
    ML_TRY(X.ensure((size_t)n * nv * sizeof(double)));
    ML_TRY(Y.ensure((size_t)n * nv * sizeof(double)));
    k_tune_fill<<<(int)std::min<int64_t>((n * nv + 255) / 256, sm_count() * 16), 256, 0, st>>>(X.as<double>(), n * nv);
    ML_CUDA(cudaGetLastError());
    float best_ms = 0.0f;
    ml_status s = time_plan(base, X.as<double>(), Y.as<double>(), nv, st, &best_ms);
    if (s != ML_OK) {
        ml_plan_destroy(base);
        return s;
    }
    ml_plan_t best = base;
    int best_bin = B0;
    for (int b : cand) {
        prm.bin = b;
        ml_plan_t p = nullptr;
        if (ml_fastsum_plan_ex(&p, points, n, d, sigma, &prm, stream) != ML_OK) continue;   // e.g. tile too large
        float ms = 0.0f;
        if (time_plan(p, X.as<double>(), Y.as<double>(), nv, st, &ms) == ML_OK && ms < best_ms) {
            ml_plan_destroy(best);
            best = p;
            best_ms = ms;
            best_bin = b;
        } else {
            ml_plan_destroy(p);
        }
    }
    set_error("");
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best_bin;
    }
    if (bin_chosen) *bin_chosen = best_bin;
    *out = best;
    return ML_OK;
}
