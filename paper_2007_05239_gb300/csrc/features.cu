// Direct summation of selected rows (the exact product, Sec. 2 / Sec. 4) and
// the point-cloud statistics used by the learned parameter model.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ml_internal.h"

namespace ml {

// out[r] = sum_{j != rows[r]} exp(-||x_{rows[r]} - x_j||^2 / sigma^2) v_j, one
// CTA per row, fixed-order block reduction
__global__ void __launch_bounds__(256) k_direct_rows(const double *__restrict__ X, int64_t n, int d, double inv_s2,
                                                     const double *__restrict__ v, const int64_t *__restrict__ rows,
                                                     double *out)
{
    __shared__ double red[8];
    const int64_t r = rows[blockIdx.x];
    double xr[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) xr[a] = X[r * d + a];
    double s = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        if (j == r) continue;
        double r2 = 0.0;
        for (int a = 0; a < d; ++a) {
            const double t = xr[a] - X[j * d + a];
            r2 += t * t;
        }
        s += exp(-r2 * inv_s2) * v[j];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        out[blockIdx.x] = t;
    }
}

// nearest-neighbour distance of each sample point among the sample
__global__ void k_sample_nn(const double *__restrict__ X, int64_t n, int d, int S, int64_t stride, double *nn)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S) return;
    const int64_t pi = (int64_t)i * stride;
    double best = INFINITY;
    for (int j = 0; j < S; ++j) {
        if (j == i) continue;
        const int64_t pj = (int64_t)j * stride;
        double r2 = 0.0;
        for (int a = 0; a < d; ++a) {
            const double t = X[pi * d + a] - X[pj * d + a];
            r2 += t * t;
        }
        best = fmin(best, r2);
    }
    nn[i] = sqrt(best);
}


}  // namespace ml

extern "C" ml_status ml_direct_sum_rows(const double *points, int64_t n, int d, double sigma, const double *v,
                                        const int64_t *rows, int64_t nrows, double *out, void *stream)
{
    using namespace ml;
    if (!points || !v || !rows || !out) return fail(ML_ERR_ARG, "null pointer");
    if (n < 1 || d < 1 || d > 3 || nrows < 0 || nrows > INT32_MAX) return fail(ML_ERR_ARG, "bad sizes");
    if (!(sigma > 0)) return fail(ML_ERR_ARG, "sigma must be positive");
    if (nrows == 0) return ML_OK;
    cudaStream_t st = (cudaStream_t)stream;
    ProfScope pr("direct", st);
    k_direct_rows<<<(unsigned)nrows, 256, 0, st>>>(points, n, d, 1.0 / (sigma * sigma), v, rows, out);
    ML_CUDA(cudaGetLastError());
    return ML_OK;
}

namespace ml {
ml_status bounding_box(const double *points, int64_t n, int d, cudaStream_t st, double lo[3], double hi[3]);
}

extern "C" ml_status ml_cloud_features(const double *points, int64_t n, int d, double sigma, float *feat, void *stream)
{
    using namespace ml;
    if (!points || !feat) return fail(ML_ERR_ARG, "null pointer");
    if (n < 2 || d < 1 || d > 3) return fail(ML_ERR_ARG, "bad sizes");
    if (!(sigma > 0)) return fail(ML_ERR_ARG, "sigma must be positive");
    cudaStream_t st = (cudaStream_t)stream;
    double lo[3], hi[3];
    ML_TRY(bounding_box(points, n, d, st, lo, hi));
    double ext[3] = {0, 0, 0}, box = 0.0;
    for (int a = 0; a < d; ++a) {
        ext[a] = hi[a] - lo[a];
        box = std::max(box, ext[a]);
    }
    if (!(box > 0)) box = sigma;
    std::sort(ext, ext + 3, [](double x, double y) { return x > y; });
    const int S = (int)std::min<int64_t>(n, 2048);
    const int64_t stride = n / S;
    DevBuf nn;
    ML_TRY(nn.ensure((size_t)S * sizeof(double)));
    {
        ProfScope pr("features", st);
        k_sample_nn<<<(S + 127) / 128, 128, 0, st>>>(points, n, d, S, stride, nn.as<double>());
    }
    ML_CUDA(cudaGetLastError());
    std::vector<double> h(S);
    ML_CUDA(cudaMemcpyAsync(h.data(), nn.p, S * sizeof(double), cudaMemcpyDeviceToHost, st));
    ML_CUDA(cudaStreamSynchronize(st));
    std::sort(h.begin(), h.end());
    auto q = [&](double f) {
        const double v = h[std::min<int>(S - 1, (int)std::floor(f * (S - 1)))] / sigma;
        return (float)std::log10(std::max(v, 1e-12));
    };
    feat[0] = (float)std::log10((double)n);
    feat[1] = (float)d;
    feat[2] = (float)std::log10(sigma / box);
    for (int a = 0; a < 3; ++a) feat[3 + a] = (float)(ext[a] / box);
    feat[6] = q(0.05);
    feat[7] = q(0.5);
    feat[8] = q(0.95);
    return ML_OK;
}
