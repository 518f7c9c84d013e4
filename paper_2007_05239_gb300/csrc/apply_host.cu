// ml_fastsum_apply: the multilayer operator of Eq. I-L_1 (or the raw W, or
// the degrees) applied to a block of vectors, one layer after another on the
// caller's stream so that the FP64 output accumulates in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "ml_internal.h"

namespace ml {

#define ML_DECL_LAYER(P, D)                                                                                 \
    ml_status run_layer_##P##_d##D(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, const LayerWork &w, \
                                   cudaStream_t st);
ML_DECL_LAYER(f32, 1)
ML_DECL_LAYER(f32, 2)
ML_DECL_LAYER(f32, 3)
ML_DECL_LAYER(f64, 1)
ML_DECL_LAYER(f64, 2)
ML_DECL_LAYER(f64, 3)
ml_status run_batch_f32_d1(ml_plan_s *const *L, int T, const ApplyVec &v, const ApplyOpts &o, cudaStream_t st);
ml_status run_batch_f32_d2(ml_plan_s *const *L, int T, const ApplyVec &v, const ApplyOpts &o, cudaStream_t st);
ml_status run_batch_f32_d3(ml_plan_s *const *L, int T, const ApplyVec &v, const ApplyOpts &o, cudaStream_t st);

bool batchable(ml_plan_s *const *L, int T)
{
    if (T < 2) return false;
    const ml_plan_s *p0 = L[0];
    for (int t = 0; t < T; ++t) {
        const ml_plan_s *p = L[t];
        if (p->dense || p->kernel != ML_KERNEL_GAUSS || p->prec != ML_F32 || p->d != p0->d || p->W != p0->W ||
            p->g.nbins() != 1 || p->nsub != p0->nsub)
            return false;
        if (p->sub_max > kBatchPtsTotal) return false;
    }
    return true;
}

// per-layer outputs (ApplyOpts::layer_vecs): any FP32 layers of one d and W
bool batchable_layers(ml_plan_s *const *L, int T)
{
    if (T < 2) return false;
    for (int t = 0; t < T; ++t)
        if (L[t]->dense || L[t]->kernel != ML_KERNEL_GAUSS || L[t]->prec != ML_F32 || L[t]->d != L[0]->d ||
            L[t]->W != L[0]->W)
            return false;
    return true;
}

ml_status run_batch(ml_plan_s *const *L, int T, const ApplyVec &v, const ApplyOpts &o, cudaStream_t st)
{
    for (int t = 0; t < T; ++t) ML_TRY(ensure_workspace(L[t], v.nv));
    switch (L[0]->d) {
    case 1: return run_batch_f32_d1(L, T, v, o, st);
    case 2: return run_batch_f32_d2(L, T, v, o, st);
    default: return run_batch_f32_d3(L, T, v, o, st);
    }
}

ml_status run_layer_ws(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, const LayerWork &w, cudaStream_t st)
{
    if (v.nv < 1 || v.nv > kMaxVec) return fail(ML_ERR_ARG, "vectors per pass out of range");
    p->applied += v.nv;
    if (p->dense) return run_dense(p, v, o, st);
    ml_status r;
    if (p->prec == ML_F32) {
        switch (p->d) {
        case 1: r = run_layer_f32_d1(p, v, o, w, st); break;
        case 2: r = run_layer_f32_d2(p, v, o, w, st); break;
        default: r = run_layer_f32_d3(p, v, o, w, st); break;
        }
    } else {
        switch (p->d) {
        case 1: r = run_layer_f64_d1(p, v, o, w, st); break;
        case 2: r = run_layer_f64_d2(p, v, o, w, st); break;
        default: r = run_layer_f64_d3(p, v, o, w, st); break;
        }
    }
    // Laplacian: the near-field term, added to the same output after Alg. 1
    if (r == ML_OK && p->kernel == ML_KERNEL_LAPLACE) r = run_near(p, v, o, st);
    return r;
}

ml_status apply_layer(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, cudaStream_t st)
{
    if (v.nv < 1 || v.nv > kMaxVec) return fail(ML_ERR_ARG, "vectors per pass out of range");
    ML_TRY(ensure_workspace(p, v.nv));
    const LayerWork w{p->scratch.p, p->work[0].p, p->work[1].p};
    return run_layer_ws(p, v, o, w, st);
}

// vectors in the next pass: 8 or 4 when the plan's tile holds them and the
// window is small (W <= 8), else 1
int pass_width(const ml_plan_s *p, int remaining)
{
    if (p->W <= 8) {
        if (remaining >= 8 && p->vp >= 8) return 8;
        if (remaining >= 4 && p->vp >= 4) return 4;
    }
    return 1;
}

// Y[i, c] = sum_t parts[t][i, c] in layer order (the layers' terms of a
// multilayer product computed concurrently)
// Layer terms written in each layer's sorted order (ApplyOpts::sorted_final),
// gathered back to input order and summed in layer order:
// Y[i, c] = sum_t parts_t[iperm_t[i], c].  The interpolation then writes
// its output coalesced instead of read-modify-writing 32-byte sectors at
// random input positions; one random read per layer remains, here.
constexpr int kGatherLayers = 8;
struct LayerPerms {
    const int *iperm[kGatherLayers];
};
__global__ void k_gather_layers(const double *__restrict__ parts, LayerPerms lp, int T, int64_t n, int b, double *Y,
                                int ldy)
{
    const int64_t nb = n * b;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nb; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / b;
        const int c = (int)(e - i * b);
        double s = parts[(int64_t)lp.iperm[0][i] * b + c];
        for (int t = 1; t < T; ++t) s += parts[(int64_t)t * nb + (int64_t)lp.iperm[t][i] * b + c];
        Y[i * ldy + c] = s;
    }
}

__global__ void k_sum_layers(const double *__restrict__ parts, int T, int64_t n, int b, double *Y, int ldy)
{
    const int64_t nb = n * b;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nb; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / b;
        const int c = (int)(e - i * b);
        double s = parts[e];
        for (int t = 1; t < T; ++t) s += parts[(int64_t)t * nb + e];
        Y[i * ldy + c] = s;
    }
}

// Non-blocking streams and events kept for the process lifetime, one set
// per device, for the concurrent layer terms of a multilayer product.
struct LayerStreams {
    std::vector<cudaStream_t> s;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
};
static std::mutex g_ls_mu;
static std::vector<LayerStreams> g_ls;   // by device

// the caller holds g_ls_mu for the whole fork / enqueue / join sequence, so
// that calls from several host threads do not share the fork and join events
static ml_status layer_streams(int T, LayerStreams **out)
{
    int dev = 0;
    ML_CUDA(cudaGetDevice(&dev));
    if ((int)g_ls.size() <= dev) g_ls.resize(dev + 1);
    LayerStreams &L = g_ls[dev];
    if (!L.fork) ML_CUDA(cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming));
    while ((int)L.s.size() < T) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        ML_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        ML_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        L.s.push_back(s);
        L.join.push_back(e);
    }
    *out = &L;
    return ML_OK;
}

// Y[perm[i]] = (accumulate ? Y : 0) + alpha * deg[i]
__global__ void k_degree_out(const double *__restrict__ deg, const int *__restrict__ perm, int64_t n, double alpha,
                             int accumulate, double *Y)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double *y = Y + perm[i];
        *y = (accumulate ? *y : 0.0) + alpha * deg[i];
    }
}

static bool is_device_ptr(const void *ptr)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free error of an unregistered pointer
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Apply on device buffers (no staging).
ml_status apply_device(ml_plan_s *const *layers, int T, const double *X, int b, double *Y, int mode,
                       cudaStream_t st)
{
    const int64_t n = layers[0]->n;
    const bool per_layer = (mode & ML_PER_LAYER) != 0;
    const int base = mode & ~ML_PER_LAYER;
    if (base == ML_DEGREE) {
        if (b != 1) return fail(ML_ERR_ARG, "ML_DEGREE needs b = 1");
        for (int t = 0; t < T; ++t) {
            double *Yt = per_layer ? Y + (int64_t)t * n : Y;
            const double alpha = per_layer ? 1.0 : 1.0 / T;
            const int acc = (!per_layer && t > 0) ? 1 : 0;
            const int blocks = (int)std::min<int64_t>((n + 255) / 256, sm_count() * 16);
            ProfScope pr("degree_out", st);
            k_degree_out<<<blocks, 256, 0, st>>>(layers[t]->deg.as<double>(), layers[t]->perm.as<int>(), n, alpha,
                                                 acc, Yt);
            ML_CUDA(cudaGetLastError());
        }
        return ML_OK;
    }
    if (!per_layer && batchable(layers, T)) {
        // every layer's grid is one tile and the points keep their input
        // order: one launch per stage for all layers, layer sum in registers
        for (int c0 = 0, nv = 0; c0 < b; c0 += nv) {
            nv = 8;
            for (int t = 0; t < T; ++t) nv = std::min(nv, pass_width(layers[t], b - c0));
            ApplyVec v{X + c0, b, Y + c0, b, nv};
            ApplyOpts o;
            o.normalized = base == ML_NORMALIZED_A;
            o.alpha = 1.0 / T;
            ML_TRY(run_batch(layers, T, v, o, st));
        }
        return ML_OK;
    }
    if (per_layer && batchable_layers(layers, T)) {
        // FP32 layers of one d and W: one launch per stage for all layers,
        // each layer applying its operator to its own block
        std::vector<ApplyVec> vs(T);
        for (int c0 = 0, nv = 0; c0 < b; c0 += nv) {
            nv = 8;
            for (int t = 0; t < T; ++t) nv = std::min(nv, pass_width(layers[t], b - c0));
            for (int t = 0; t < T; ++t)
                vs[t] = ApplyVec{X + (int64_t)t * n * b + c0, b, Y + (int64_t)t * n * b + c0, b, nv};
            ApplyOpts o;
            o.normalized = base == ML_NORMALIZED_A;
            o.layer_vecs = vs.data();
            ML_TRY(run_batch(layers, T, vs[0], o, st));
        }
        return ML_OK;
    }
    bool distinct = true;
    for (int a = 0; a < T; ++a)
        for (int c = a + 1; c < T; ++c)
            if (layers[a] == layers[c]) distinct = false;
    if (!per_layer && T >= 2 && distinct && !profiling()) {
        // the layers' terms on concurrent streams into per-layer buffers, then
        // summed in layer order (the same FP64 additions as accumulating)
        std::lock_guard<std::mutex> lk(g_ls_mu);
        LayerStreams *ls = nullptr;
        ML_TRY(layer_streams(T, &ls));
        ml_plan_s *p0 = layers[0];
        ML_TRY(p0->sum_parts.ensure((size_t)T * n * b * sizeof(double)));
        double *parts = p0->sum_parts.as<double>();
        // Gaussian fast-summation layers: terms in sorted order, gathered after
        bool gather = T <= kGatherLayers;
        for (int t = 0; t < T; ++t)
            gather = gather && !layers[t]->dense && layers[t]->kernel == ML_KERNEL_GAUSS && layers[t]->iperm.p;
        ML_CUDA(cudaEventRecord(ls->fork, st));
        for (int t = 0; t < T; ++t) {
            cudaStream_t s = ls->s[t];
            ML_CUDA(cudaStreamWaitEvent(s, ls->fork, 0));
            for (int c0 = 0, nv = 0; c0 < b; c0 += nv) {
                nv = pass_width(layers[t], b - c0);
                ApplyVec v{X + c0, b, parts + (int64_t)t * n * b + c0, b, nv};
                ApplyOpts o;
                o.normalized = base == ML_NORMALIZED_A;
                o.alpha = 1.0 / T;
                o.sorted_final = gather;
                ML_TRY(apply_layer(layers[t], v, o, s));
            }
            ML_CUDA(cudaEventRecord(ls->join[t], s));
            ML_CUDA(cudaStreamWaitEvent(st, ls->join[t], 0));
        }
        ProfScope pr("vector", st);
        const int blocks = (int)std::min<int64_t>((n * b + 255) / 256, sm_count() * 16);
        if (gather) {
            LayerPerms lp{};
            for (int t = 0; t < T; ++t) lp.iperm[t] = layers[t]->iperm.as<int>();
            k_gather_layers<<<blocks, 256, 0, st>>>(parts, lp, T, n, b, Y, b);
        } else {
            k_sum_layers<<<blocks, 256, 0, st>>>(parts, T, n, b, Y, b);
        }
        ML_CUDA(cudaGetLastError());
        return ML_OK;
    }
    for (int t = 0; t < T; ++t) {
        ml_plan_s *p = layers[t];
        const double *Xt = per_layer ? X + (int64_t)t * n * b : X;
        double *Yt = per_layer ? Y + (int64_t)t * n * b : Y;
        for (int c0 = 0, nv = 0; c0 < b; c0 += nv) {
            nv = pass_width(p, b - c0);
            ApplyVec v{Xt + c0, b, Yt + c0, b, nv};
            ApplyOpts o;
            o.normalized = base == ML_NORMALIZED_A;
            o.accumulate = !per_layer && t > 0;
            o.alpha = per_layer ? 1.0 : 1.0 / T;
            ML_TRY(apply_layer(p, v, o, st));
        }
    }
    return ML_OK;
}

}  // namespace ml

extern "C" ml_status ml_fastsum_apply(const ml_plan_t *layers, int T, const double *X, int b, double *Y, int mode,
                                      void *stream)
{
    using namespace ml;
    if (!layers || T < 1) return fail(ML_ERR_ARG, "layers is null or T < 1");
    for (int t = 0; t < T; ++t)
        if (!layers[t]) return fail(ML_ERR_ARG, "layer " + std::to_string(t) + " is null");
    const int64_t n = layers[0]->n;
    for (int t = 1; t < T; ++t)
        if (layers[t]->n != n) return fail(ML_ERR_ARG, "layers do not share n");
    if (b < 1 || b > 64) return fail(ML_ERR_ARG, "b must be in [1, 64]");
    const int base = mode & ~ML_PER_LAYER;
    if ((mode & ~(ML_PER_LAYER | 3)) != 0 || base > ML_DEGREE) return fail(ML_ERR_ARG, "unknown mode");
    if (!Y) return fail(ML_ERR_ARG, "Y is null");
    if (base == ML_NORMALIZED_A)
        for (int t = 0; t < T; ++t)
            if (!layers[t]->deg_ok)
                return fail(ML_ERR_DEGREE, "layer " + std::to_string(t) +
                                               " has a degree <= 0: D^{-1/2} is undefined (isolated point or too "
                                               "coarse an approximation)");
    if (base != ML_DEGREE && !X) return fail(ML_ERR_ARG, "X is null");
    cudaStream_t st = (cudaStream_t)stream;
    const bool per_layer = (mode & ML_PER_LAYER) != 0;
    const int64_t elems = n * b * (per_layer ? T : 1);
    const bool x_dev = base == ML_DEGREE || is_device_ptr(X);
    const bool y_dev = is_device_ptr(Y);
    {
        // the output buffer must not overlap the input
        const char *xb = (const char *)X, *yb = (const char *)Y;
        const size_t bytes = (size_t)elems * sizeof(double);
        if (X && xb < yb + bytes && yb < xb + bytes) return fail(ML_ERR_ARG, "X and Y overlap");
    }
    ml_plan_s *p0 = layers[0];
    const double *Xd = X;
    double *Yd = Y;
    if (!x_dev) {
        ML_TRY(p0->stage_x.ensure((size_t)elems * sizeof(double)));
        ML_CUDA(cudaMemcpyAsync(p0->stage_x.p, X, (size_t)elems * sizeof(double), cudaMemcpyHostToDevice, st));
        Xd = p0->stage_x.as<double>();
    }
    if (!y_dev) {
        ML_TRY(p0->stage_y.ensure((size_t)elems * sizeof(double)));
        Yd = p0->stage_y.as<double>();
    }
    ML_TRY(apply_device(layers, T, Xd, b, Yd, mode, st));
    if (!y_dev) {
        ML_CUDA(cudaMemcpyAsync(Y, Yd, (size_t)elems * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    if (!x_dev || !y_dev) ML_CUDA(cudaStreamSynchronize(st));
    return ML_OK;
}
