// Kernel timing registry: CUDA events around each launch on its stream.
#include <cuda_runtime.h>

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
