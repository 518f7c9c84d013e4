// Dense layers: the explicit regime for small graphs (Sec. 2 defines W for
// any feature dimension; the fast summation of Sec. 4 needs d <= 3).  The
// plan stores W (n x n, zero diagonal, FP64 or FP32) built on the GPU from
// the points, W_ij = exp(-||x_i - x_j||^2 / sigma^2), or copied from a given
// symmetric weight matrix (e.g. the adjacency of a stochastic block model).
// A product is one streaming pass over W: one warp per row, lanes strided
// over the columns, FP64 accumulation, then the same epilogue as the fast
// summation (D^{-1/2} pre/post scaling, alpha, shift, accumulate).  Such a
// plan works everywhere a fast-summation plan does: products, degrees, the
// eigensolvers and the Allen-Cahn scheme.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "ml_internal.h"

namespace ml {
namespace {

constexpr int kDT = 32;   // W tile edge of the build kernel

// W[i][j] = exp(-||x_i - x_j||^2 * inv_s2), zero diagonal; squared distances
// summed from coordinate differences in FP64 (staged 32 features at a time)
template <typename T>
__global__ void __launch_bounds__(256) k_dense_build(const double *__restrict__ X, int64_t n, int d, double inv_s2,
                                                    T *W)
{
    __shared__ double xi[kDT][kDT + 1], xj[kDT][kDT + 1];
    const int64_t i0 = (int64_t)blockIdx.y * kDT, j0 = (int64_t)blockIdx.x * kDT;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads, 4 rows each
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int f0 = 0; f0 < d; f0 += kDT) {
        for (int e = threadIdx.x; e < kDT * kDT; e += blockDim.x) {
            const int r = e / kDT, f = e - r * kDT;
            xi[r][f] = (i0 + r < n && f0 + f < d) ? X[(i0 + r) * d + f0 + f] : 0.0;
            xj[r][f] = (j0 + r < n && f0 + f < d) ? X[(j0 + r) * d + f0 + f] : 0.0;
        }
        __syncthreads();
        const int fl = min(kDT, d - f0);
        for (int f = 0; f < fl; ++f) {
            const double b = xj[tx][f];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const double t = xi[ty + 8 * q][f] - b;
                acc[q] = fma(t, t, acc[q]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t i = i0 + ty + 8 * q, j = j0 + tx;
        if (i < n && j < n) W[i * n + j] = (T)(i == j ? 0.0 : exp(-acc[q] * inv_s2));
    }
}

// copy of a given weight matrix with the diagonal set to zero (no self-edges)
template <typename T>
__global__ void k_dense_copy(const double *__restrict__ Win, int64_t n, T *W)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / n;
        W[e] = (T)((e - i * n) == i ? 0.0 : Win[e]);
    }
}

struct DenseArgs {
    const void *W;
    int64_t n;
    const double *X;   // input block (row stride ldx) or null (ones)
    int ldx;
    double *Y;
    int ldy;
    const double *dinv;   // pre/post scaling or null
    double alpha, shift;
    int accumulate, sorted_out;
};

// one warp per row i: acc_c = sum_j W[i][j] u_j[c], u = D^{-1/2} x (or x)
template <typename T, int NV>
__global__ void __launch_bounds__(256) k_dense_apply(const DenseArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const T *W = static_cast<const T *>(a.W);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < a.n; i += nw) {
        double acc[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) acc[c] = 0.0;
        const T *row = W + i * a.n;
        for (int64_t j = lane; j < a.n; j += 32) {
            const double w = (double)row[j];
            const double s = a.dinv ? a.dinv[j] : 1.0;
#pragma unroll
            for (int c = 0; c < NV; ++c) acc[c] = fma(w, (a.X ? a.X[j * a.ldx + c] : 1.0) * s, acc[c]);
        }
#pragma unroll
        for (int c = 0; c < NV; ++c)
            for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
        if (lane == 0) {
            const double ds = a.dinv ? a.dinv[i] : 1.0;
#pragma unroll
            for (int c = 0; c < NV; ++c) {
                double *yp = a.Y + i * a.ldy + c;
                if (a.sorted_out) {
                    *yp = acc[c];
                } else {
                    double out = a.alpha * ds * acc[c] + a.shift * (a.X ? a.X[i * a.ldx + c] : 1.0);
                    if (a.accumulate) out += *yp;
                    *yp = out;
                }
            }
        }
    }
}

__global__ void k_dense_dinv(const double *__restrict__ deg, int64_t n, double *dinv, int *bad)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = deg[i];
        if (!(v > 0.0) || !isfinite(v)) {
            atomicExch(bad, 1);
            dinv[i] = 0.0;
        } else {
            dinv[i] = 1.0 / sqrt(v);
        }
    }
}

__global__ void k_iota(int64_t n, int *perm)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        perm[i] = (int)i;
}

int blocks_for(int64_t work) { return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, sm_count() * 16)); }

template <typename T, int NV>
ml_status launch_dense(const DenseArgs &a, cudaStream_t st)
{
    const int rows_per_cta = 8;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((a.n + rows_per_cta - 1) / rows_per_cta, sm_count() * 32));
    ProfScope pr("dense", st);
    k_dense_apply<T, NV><<<grid, 256, 0, st>>>(a);
    ML_CUDA(cudaGetLastError());
    return ML_OK;
}

// the plan's common part once W is stored: identity order, degrees, D^{-1/2}
ml_status dense_finish(ml_plan_s *p, cudaStream_t st)
{
    const int64_t n = p->n;
    ML_TRY(p->perm.ensure((size_t)n * sizeof(int)));
    ML_TRY(p->deg.ensure((size_t)n * sizeof(double)));
    ML_TRY(p->dinv.ensure((size_t)n * sizeof(double)));
    ML_TRY(ensure_workspace(p, 1));
    k_iota<<<blocks_for(n), 256, 0, st>>>(n, p->perm.as<int>());
    ApplyVec v{nullptr, 1, p->deg.as<double>(), 1, 1};
    ApplyOpts o;
    o.sorted_out = true;
    ML_TRY(run_dense(p, v, o, st));
    ML_CUDA(cudaMemsetAsync(p->status.p, 0, sizeof(int), st));
    k_dense_dinv<<<blocks_for(n), 256, 0, st>>>(p->deg.as<double>(), n, p->dinv.as<double>(), p->status.as<int>());
    ML_CUDA(cudaGetLastError());
    int bad = 0;
    ML_CUDA(cudaMemcpyAsync(&bad, p->status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    std::vector<double> hd(n);
    ML_CUDA(cudaMemcpyAsync(hd.data(), p->deg.p, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    ML_CUDA(cudaStreamSynchronize(st));
    p->deg_min = *std::min_element(hd.begin(), hd.end());
    p->deg_max = *std::max_element(hd.begin(), hd.end());
    p->deg_ok = !bad;
    p->applied = 0;
    return ML_OK;
}

ml_status dense_new(ml_plan_t *out, int64_t n, int d, ml_prec prec, ml_plan_s **pp)
{
    if (!out) return fail(ML_ERR_ARG, "out is null");
    *out = nullptr;
    if (n < 2 || n > (1 << 17)) return fail(ML_ERR_ARG, "dense layers need 2 <= n <= 131072");
    if (prec != ML_F32 && prec != ML_F64) return fail(ML_ERR_ARG, "prec must be ML_F32 or ML_F64");
    ml_plan_s *p = new (std::nothrow) ml_plan_s;
    if (!p) return fail(ML_ERR_OOM, "host allocation failed");
    p->n = n;
    p->d = d;
    p->prec = prec;
    p->dense = true;
    p->vp = kMaxVec;
    *pp = p;
    return ML_OK;
}

}  // namespace

ml_status run_dense(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, cudaStream_t st)
{
    DenseArgs a;
    a.W = p->Wd.p;
    a.n = p->n;
    a.X = v.X;
    a.ldx = v.ldx;
    a.Y = v.Y;
    a.ldy = v.ldy;
    a.dinv = o.normalized ? p->dinv.as<double>() : nullptr;
    a.alpha = o.alpha;
    a.shift = o.shift;
    a.accumulate = o.accumulate ? 1 : 0;
    a.sorted_out = o.sorted_out ? 1 : 0;
    const bool f32 = p->prec == ML_F32;
    switch (v.nv) {
    case 1: return f32 ? launch_dense<float, 1>(a, st) : launch_dense<double, 1>(a, st);
    case 4: return f32 ? launch_dense<float, 4>(a, st) : launch_dense<double, 4>(a, st);
    case 8: return f32 ? launch_dense<float, 8>(a, st) : launch_dense<double, 8>(a, st);
    default: return fail(ML_ERR_ARG, "unsupported vectors per pass");
    }
}

}  // namespace ml

extern "C" ml_status ml_dense_plan(ml_plan_t *out, const double *points, int64_t n, int d, double sigma, ml_prec prec,
                                   void *stream)
{
    using namespace ml;
    if (!points) return fail(ML_ERR_ARG, "points is null");
    if (d < 1) return fail(ML_ERR_ARG, "d must be >= 1");
    if (!(sigma > 0) || !std::isfinite(sigma)) return fail(ML_ERR_ARG, "sigma must be positive and finite");
    ml_plan_s *p = nullptr;
    ML_TRY(dense_new(out, n, d, prec, &p));
    cudaStream_t st = (cudaStream_t)stream;
    p->sigma = sigma;
    const size_t es = prec == ML_F32 ? 4 : 8;
    ml_status s = p->Wd.ensure((size_t)n * n * es);
    if (s == ML_OK) {
        const dim3 grid((unsigned)((n + kDT - 1) / kDT), (unsigned)((n + kDT - 1) / kDT));
        {
            ProfScope pr("plan", st);
            if (prec == ML_F32) k_dense_build<float><<<grid, 256, 0, st>>>(points, n, d, 1.0 / (sigma * sigma), p->Wd.as<float>());
            else k_dense_build<double><<<grid, 256, 0, st>>>(points, n, d, 1.0 / (sigma * sigma), p->Wd.as<double>());
        }
        const cudaError_t e = cudaGetLastError();
        s = e == cudaSuccess ? dense_finish(p, st) : cuda_fail(e, "k_dense_build", __FILE__, __LINE__);
    }
    if (s != ML_OK) {
        ml_plan_destroy(p);
        return s;
    }
    *out = p;
    return ML_OK;
}

extern "C" ml_status ml_dense_plan_matrix(ml_plan_t *out, const double *W, int64_t n, ml_prec prec, void *stream)
{
    using namespace ml;
    if (!W) return fail(ML_ERR_ARG, "W is null");
    ml_plan_s *p = nullptr;
    ML_TRY(dense_new(out, n, 0, prec, &p));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t es = prec == ML_F32 ? 4 : 8;
    ml_status s = p->Wd.ensure((size_t)n * n * es);
    if (s == ML_OK) {
        {
            ProfScope pr("plan", st);
            if (prec == ML_F32) k_dense_copy<float><<<blocks_for(n * n), 256, 0, st>>>(W, n, p->Wd.as<float>());
            else k_dense_copy<double><<<blocks_for(n * n), 256, 0, st>>>(W, n, p->Wd.as<double>());
        }
        const cudaError_t e = cudaGetLastError();
        s = e == cudaSuccess ? dense_finish(p, st) : cuda_fail(e, "k_dense_copy", __FILE__, __LINE__);
    }
    if (s != ML_OK) {
        ml_plan_destroy(p);
        return s;
    }
    *out = p;
    return ML_OK;
}
