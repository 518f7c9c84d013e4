// ml_fastsum_plan_many: the plans of all layers of a multilayer graph at
// once.  A plan's set-up is a chain of small kernels and host steps with
// synchronisations (bounding box, sort, bin counts, Fourier tables,
// degrees); the layers are independent, so host threads build them
// concurrently, each on its own non-blocking stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "ml_internal.h"

extern "C" ml_status ml_fastsum_plan_many(ml_plan_t *out, const double *const *points, int64_t n, const int *d,
                                          const double *sigma, const ml_plan_params *params, int T, void *stream)
{
    using namespace ml;
    if (!out || !points || !d || !sigma || !params || T < 1) return fail(ML_ERR_ARG, "null argument or T < 1");
    for (int t = 0; t < T; ++t) out[t] = nullptr;
    int dev = 0;
    ML_CUDA(cudaGetDevice(&dev));
    // the points are ready once the caller's stream has reached this point
    cudaEvent_t ready = nullptr;
    ML_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    cudaError_t ce = cudaEventRecord(ready, (cudaStream_t)stream);
    if (ce != cudaSuccess) {
        cudaEventDestroy(ready);
        return cuda_fail(ce, "cudaEventRecord", __FILE__, __LINE__);
    }
    std::vector<ml_status> st(T, ML_OK);
    std::vector<std::string> msg(T);
    std::atomic<int> next{0};
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int workers = std::max(1, std::min<int>(T, (int)std::max(1u, hw / 2)));
    auto work = [&]() {
        cudaSetDevice(dev);
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
        for (int t = next++; t < T; t = next++) {
            if (!s) {
                st[t] = ML_ERR_CUDA;
                msg[t] = "cudaStreamCreate failed";
                continue;
            }
            cudaStreamWaitEvent(s, ready, 0);
            st[t] = ml_fastsum_plan_ex(&out[t], points[t], n, d[t], sigma[t], params, s);
            if (st[t] != ML_OK) msg[t] = ml_last_error();
        }
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    };
    std::vector<std::thread> pool;
    for (int w = 1; w < workers; ++w) pool.emplace_back(work);
    work();
    for (auto &th : pool) th.join();
    cudaEventDestroy(ready);
    for (int t = 0; t < T; ++t)
        if (st[t] != ML_OK) {
            for (int u = 0; u < T; ++u) {
                ml_plan_destroy(out[u]);
                out[u] = nullptr;
            }
            return fail(st[t], "layer " + std::to_string(t) + ": " + msg[t]);
        }
    return ML_OK;
}
