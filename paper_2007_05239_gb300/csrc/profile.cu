// Kernel timing registry: CUDA events around each launch on its stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ml_internal.h"

namespace ml {

namespace {
struct Pending {
    cudaEvent_t a, b;
};
struct Entry {
    int64_t launches = 0;
    double ms = 0.0;
    std::vector<Pending> pending;
};
std::atomic<bool> g_on{false};
std::atomic<long long> g_graph_replays{0};
std::mutex g_mu;
std::map<std::string, Entry> g_tab;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void drain(Entry &en)
{
    for (auto &pd : en.pending) {
        cudaEventSynchronize(pd.b);
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, pd.a, pd.b) == cudaSuccess) en.ms += t;
        g_pool.push_back(pd.a);
        g_pool.push_back(pd.b);
    }
    en.pending.clear();
}
}  // namespace

static thread_local bool t_suppress = false;

bool profiling() { return !t_suppress && g_on.load(std::memory_order_relaxed); }
void count_graph_replay() { g_graph_replays.fetch_add(1, std::memory_order_relaxed); }

NoProfileScope::NoProfileScope() : prev_(t_suppress) { t_suppress = true; }
NoProfileScope::~NoProfileScope() { t_suppress = prev_; }

ProfScope::ProfScope(const char *name, cudaStream_t st) : name_(name), st_(st)
{
    if (!profiling()) return;
    std::lock_guard<std::mutex> lk(g_mu);
    a_ = get_event();
    cudaEventRecord((cudaEvent_t)a_, st_);
    active_ = true;
}

ProfScope::~ProfScope()
{
    if (!active_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t b = get_event();
    cudaEventRecord(b, st_);
    Entry &en = g_tab[name_];
    en.launches += 1;
    en.pending.push_back({(cudaEvent_t)a_, b});
    if (en.pending.size() > 4096) drain(en);
}

}  // namespace ml

extern "C" {

ml_status ml_profile_enable(int on)
{
    ml::g_on.store(on != 0);
    return ML_OK;
}

ml_status ml_profile_reset(void)
{
    std::lock_guard<std::mutex> lk(ml::g_mu);
    for (auto &kv : ml::g_tab) ml::drain(kv.second);
    ml::g_tab.clear();
    return ML_OK;
}

int64_t ml_graph_replays(void) { return (int64_t)ml::g_graph_replays.load(std::memory_order_relaxed); }

ml_status ml_profile_read(int i, const char **name, int64_t *launches, double *ms)
{
    std::lock_guard<std::mutex> lk(ml::g_mu);
    if (i < 0 || i >= (int)ml::g_tab.size()) return ml::fail(ML_ERR_ARG, "profile index out of range");
    auto it = ml::g_tab.begin();
    std::advance(it, i);
    ml::drain(it->second);
    if (name) *name = it->first.c_str();
    if (launches) *launches = it->second.launches;
    if (ms) *ms = it->second.ms;
    return ML_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ peaks
// Throughput micro-kernels for the roofline denominators: independent FMA
// chains on the FP32 or FP64 pipe, and conflict-free 32-bit shared-memory
// atomic adds (lane l of a warp adds to word l of the warp's own 32-word
// row, so every atomic instruction is one wavefront).
namespace ml {
namespace {
constexpr int kPeakChains = 8;
constexpr int kPeakUnroll = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T *sink, int iters, T a, T b)
{
    T x[kPeakChains];
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) x[i] = (T)(threadIdx.x + 1) * (T)(i + 1) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kPeakUnroll; ++k) {
#pragma unroll
            for (int i = 0; i < kPeakChains; ++i) x[i] = fma(x[i], a, b);
        }
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) s += x[i];
    if (s == (T)-1.0) sink[blockIdx.x] = s;   // never true for these inputs; keeps the chains live
}

__global__ void __launch_bounds__(256) k_atomic_peak(int *sink, int iters)
{
    __shared__ int s[256];
    s[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, row = threadIdx.x & ~31;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kPeakUnroll; ++k) atomicAdd(&s[row + ((lane + k) & 31)], it + k);
    }
    __syncthreads();
    if (s[threadIdx.x] == 0x7fffffff) sink[blockIdx.x] = 1;
}
}  // namespace

static ml_status time_peak(int what, double *rate, cudaStream_t st)
{
    const int sms = sm_count();
    const int blocks = sms * 8, threads = 256;
    DevBuf sink;
    ML_TRY(sink.ensure((size_t)blocks * sizeof(double)));
    cudaEvent_t e0, e1;
    ML_CUDA(cudaEventCreate(&e0));
    ML_CUDA(cudaEventCreate(&e1));
    const int iters = what == 0 ? 4096 : (what == 1 ? 96 : 2048);
    double best = 0.0;
    for (int rep = 0; rep < 4; ++rep) {   // first launch untimed (warm-up)
        cudaEventRecord(e0, st);
        if (what == 0)
            k_fma_peak<float><<<blocks, threads, 0, st>>>(sink.as<float>(), iters, 0.9999f, 1e-4f);
        else if (what == 1)
            k_fma_peak<double><<<blocks, threads, 0, st>>>(sink.as<double>(), iters, 0.9999, 1e-4);
        else
            k_atomic_peak<<<blocks, threads, 0, st>>>(sink.as<int>(), iters);
        cudaEventRecord(e1, st);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(e, "peak micro-kernel", __FILE__, __LINE__);
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double ops = (double)blocks * threads * iters * kPeakUnroll * (what == 2 ? 1 : kPeakChains);
        // FMA: 2 flop each, in TFLOP/s; atomics: in 1e12 per second
        const double r = ops * (what == 2 ? 1.0 : 2.0) / (ms * 1e-3) / 1e12;
        if (rep > 0) best = std::max(best, r);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ML_CUDA(cudaGetLastError());
    *rate = best;
    return ML_OK;
}

}  // namespace ml

extern "C" ml_status ml_measure_peak(int what, double *rate, void *stream)
{
    if (what < 0 || what > 2 || !rate) return ml::fail(ML_ERR_ARG, "what must be 0, 1 or 2 and rate non-null");
    ml::NoProfileScope no_events;
    return ml::time_peak(what, rate, (cudaStream_t)stream);
}
