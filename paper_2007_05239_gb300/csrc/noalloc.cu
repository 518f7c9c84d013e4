// ml_fastsum_apply_noalloc: ml_fastsum_apply for callers that cannot
// allocate device memory.  All of its scratch (the spreading tiles and the
// grid-transform buffers) lives in one file-scope device array of fixed
// size; the plans' own data (sorted points, tables, degrees) were allocated
// when the plans were made.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "ml_internal.h"

namespace ml {

ml_status apply_device(ml_plan_s *const *layers, int T, const double *X, int b, double *Y, int mode, cudaStream_t st);

// 32 MiB, held by every GPU that loads the library until the process exits.
constexpr size_t kNoAllocBytes = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[256];   // device address of the array, per device id

// The array's name in host code is only a host-side stand-in; its device
// address is looked up once per device, with that device current.
static ml_status noalloc_base(void **out)
{
    int dev = 0;
    ML_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return fail(ML_ERR_CUDA, "device id out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
        g_noalloc_addr[dev] = ptr;
    }
    *out = g_noalloc_addr[dev];
    return ML_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static bool device_resident(const void *ptr)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace ml

extern "C" ml_status ml_fastsum_apply_noalloc(const ml_plan_t *layers, int T, const double *X, int b, double *Y,
                                              int mode, void *stream)
{
    using namespace ml;
    NoProfileScope no_events;
    if (!layers || T < 1) return fail(ML_ERR_ARG, "layers is null or T < 1");
    for (int t = 0; t < T; ++t)
        if (!layers[t]) return fail(ML_ERR_ARG, "null layer");
    const int64_t n = layers[0]->n;
    for (int t = 1; t < T; ++t)
        if (layers[t]->n != n) return fail(ML_ERR_ARG, "layers do not share n");
    if (b < 1 || b > 64) return fail(ML_ERR_ARG, "b must be in [1, 64]");
    const int base = mode & ~ML_PER_LAYER;
    if ((mode & ~(ML_PER_LAYER | 3)) != 0 || base > ML_DEGREE) return fail(ML_ERR_ARG, "unknown mode");
    if (!Y || !device_resident(Y)) return fail(ML_ERR_ARG, "Y must be device memory (host buffers need staging)");
    if (base != ML_DEGREE && (!X || !device_resident(X)))
        return fail(ML_ERR_ARG, "X must be device memory (host buffers need staging)");
    const bool per_layer = (mode & ML_PER_LAYER) != 0;
    const int64_t elems = n * b * (per_layer ? T : 1);
    if (X) {
        const char *xb = (const char *)X, *yb = (const char *)Y;
        const size_t bytes = (size_t)elems * sizeof(double);
        if (xb < yb + bytes && yb < xb + bytes) return fail(ML_ERR_ARG, "X and Y overlap");
    }
    if (base == ML_NORMALIZED_A)
        for (int t = 0; t < T; ++t)
            if (!layers[t]->deg_ok) return fail(ML_ERR_DEGREE, "a layer has a degree <= 0: D^{-1/2} is undefined");
    cudaStream_t st = (cudaStream_t)stream;
    if (base == ML_DEGREE) return apply_device(layers, T, X, b, Y, mode, st);  // stored degrees, no scratch

    // one layout for every layer and pass: [tiles | work0 | work1] at the widest pass
    size_t need = 0, sb_max = 0, wb_max = 0;
    for (int t = 0; t < T; ++t) {
        size_t sb = 0, wb = 0;
        workspace_bytes(layers[t], pass_width(layers[t], b), &sb, &wb);
        sb_max = std::max(sb_max, sb);
        wb_max = std::max(wb_max, wb);
    }
    need = align256(sb_max) + 2 * align256(wb_max);
    if (need > kNoAllocBytes)
        return fail(ML_ERR_ARG, "the layers need " + std::to_string(need) +
                                    " bytes of scratch; the static limit of ml_fastsum_apply_noalloc is " +
                                    std::to_string(kNoAllocBytes) + " bytes");
    void *mem = nullptr;
    ML_TRY(noalloc_base(&mem));
    char *m = static_cast<char *>(mem);
    const LayerWork w{m, m + align256(sb_max), m + align256(sb_max) + align256(wb_max)};
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
            ML_TRY(run_layer_ws(p, v, o, w, st));
        }
    }
    return ML_OK;
}
