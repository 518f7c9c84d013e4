// The learned parameter model: a small FP32 MLP (n_in -> h -> h -> n_out,
// tanh hidden layers) trained and evaluated by the library's own kernels,
// and the planner that uses it to pick the NFFT parameters of a layer.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ml_internal.h"

struct ml_mlp_s {
    int nin = 0, h = 0, nout = 0;
    int64_t nparam = 0;
    ml::DevBuf params, grad, adam_m, adam_v, norm, ws, part;
    int ws_batch = 0;
    int64_t adam_t = 0;
    double margins[3] = {0.0, 0.0, 0.0};   // per bandwidth factor of the planner (0: unset)
    int64_t offW1() const { return 0; }
    int64_t offb1() const { return (int64_t)h * nin; }
    int64_t offW2() const { return offb1() + h; }
    int64_t offb2() const { return offW2() + (int64_t)h * h; }
    int64_t offW3() const { return offb2() + h; }
    int64_t offb3() const { return offW3() + (int64_t)nout * h; }
};

namespace ml {

__global__ void k_standardise(const float *__restrict__ X, int64_t rows, int cols, const float *__restrict__ mean,
                              const float *__restrict__ stdv, float *out)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % cols);
        out[e] = (X[e] - mean[c]) / stdv[c];
    }
}

__global__ void k_unstandardise(const float *__restrict__ Z, int64_t rows, int cols, const float *__restrict__ mean,
                                const float *__restrict__ stdv, float *out)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % cols);
        out[e] = mean[c] + stdv[c] * Z[e];
    }
}

// Out[b][j] = act(sum_k In[b][k] W[j][k] + bias[j]), act = tanh or identity
__global__ void k_dense(const float *__restrict__ In, const float *__restrict__ W, const float *__restrict__ bias,
                        int B, int K, int N, int act_tanh, float *Out)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)B * N; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / N), j = (int)(e % N);
        float s = bias[j];
        for (int k = 0; k < K; ++k) s = fmaf(In[(int64_t)b * K + k], W[(int64_t)j * K + k], s);
        Out[e] = act_tanh ? tanhf(s) : s;
    }
}

// dY = 2 (Y - T) / (B * O); per-block partial sums of (Y - T)^2
__global__ void __launch_bounds__(256) k_mse(const float *__restrict__ Y, const float *__restrict__ Tg, int64_t cnt,
                                             float *dY, float *part)
{
    __shared__ float red[8];
    float s = 0.0f;
    const float sc = 2.0f / (float)cnt;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
        const float r = Y[e] - Tg[e];
        dY[e] = sc * r;
        s = fmaf(r, r, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// dW[j][k] = sum_b dZ[b][j] In[b][k];  db[j] = sum_b dZ[b][j]  (k == K)
__global__ void k_dense_grad_w(const float *__restrict__ dZ, const float *__restrict__ In, int B, int K, int N,
                               float *dW, float *db)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)N * (K + 1); e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / (K + 1)), k = (int)(e % (K + 1));
        float s = 0.0f;
        if (k < K) {
            for (int b = 0; b < B; ++b) s = fmaf(dZ[(int64_t)b * N + j], In[(int64_t)b * K + k], s);
            dW[(int64_t)j * K + k] = s;
        } else {
            for (int b = 0; b < B; ++b) s += dZ[(int64_t)b * N + j];
            db[j] = s;
        }
    }
}

// dZin[b][k] = (sum_j dZ[b][j] W[j][k]) * (1 - A[b][k]^2)  (tanh derivative)
__global__ void k_dense_grad_in(const float *__restrict__ dZ, const float *__restrict__ W, const float *__restrict__ A,
                                int B, int K, int N, float *dZin)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)B * K; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / K), k = (int)(e % K);
        float s = 0.0f;
        for (int j = 0; j < N; ++j) s = fmaf(dZ[(int64_t)b * N + j], W[(int64_t)j * K + k], s);
        const float a = A[e];
        dZin[e] = s * (1.0f - a * a);
    }
}

// Adam (Kingma & Ba), bias-corrected
__global__ void k_adam(float *p, const float *__restrict__ g, float *m, float *v, int64_t n, float lr, float b1,
                       float b2, float eps, float c1, float c2)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[e];
        const float mi = b1 * m[e] + (1.0f - b1) * gi;
        const float vi = b2 * v[e] + (1.0f - b2) * gi * gi;
        m[e] = mi;
        v[e] = vi;
        p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

static int blocks_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096)); }

// workspace: Xn (B nin), A1 (B h), A2 (B h), Z3 (B nout), T (B nout), dY (B nout), dZ2 (B h), dZ1 (B h)
static ml_status mlp_ws(ml_mlp_s *m, int B)
{
    if (B <= m->ws_batch) return ML_OK;
    const int64_t fl = (int64_t)B * (m->nin + 4 * m->h + 3 * m->nout);
    ML_TRY(m->ws.ensure((size_t)fl * sizeof(float)));
    ML_TRY(m->part.ensure(4096 * sizeof(float)));
    m->ws_batch = B;
    return ML_OK;
}

struct MlpBufs {
    float *Xn, *A1, *A2, *Z3, *T, *dY, *dZ2, *dZ1;
};

static MlpBufs bufs_of(ml_mlp_s *m, int B)
{
    float *p = m->ws.as<float>();
    MlpBufs b;
    b.Xn = p;
    p += (int64_t)B * m->nin;
    b.A1 = p;
    p += (int64_t)B * m->h;
    b.A2 = p;
    p += (int64_t)B * m->h;
    b.Z3 = p;
    p += (int64_t)B * m->nout;
    b.T = p;
    p += (int64_t)B * m->nout;
    b.dY = p;
    p += (int64_t)B * m->nout;
    b.dZ2 = p;
    p += (int64_t)B * m->h;
    b.dZ1 = p;
    return b;
}

static void forward_std(ml_mlp_s *m, const MlpBufs &b, int B, cudaStream_t st)
{
    const float *P = m->params.as<float>();
    k_dense<<<blocks_for((int64_t)B * m->h), 256, 0, st>>>(b.Xn, P + m->offW1(), P + m->offb1(), B, m->nin, m->h, 1, b.A1);
    k_dense<<<blocks_for((int64_t)B * m->h), 256, 0, st>>>(b.A1, P + m->offW2(), P + m->offb2(), B, m->h, m->h, 1, b.A2);
    k_dense<<<blocks_for((int64_t)B * m->nout), 256, 0, st>>>(b.A2, P + m->offW3(), P + m->offb3(), B, m->h, m->nout,
                                                            0, b.Z3);
}

// loss (mean squared error of standardised outputs) and gradient into m->grad
static ml_status loss_grad_std(ml_mlp_s *m, const MlpBufs &b, int B, cudaStream_t st, float *loss)
{
    const float *P = m->params.as<float>();
    float *G = m->grad.as<float>();
    forward_std(m, b, B, st);
    const int64_t cnt = (int64_t)B * m->nout;
    const int nb = blocks_for(cnt);
    k_mse<<<nb, 256, 0, st>>>(b.Z3, b.T, cnt, b.dY, m->part.as<float>());
    k_dense_grad_w<<<blocks_for((int64_t)m->nout * (m->h + 1)), 256, 0, st>>>(b.dY, b.A2, B, m->h, m->nout,
                                                                              G + m->offW3(), G + m->offb3());
    k_dense_grad_in<<<blocks_for((int64_t)B * m->h), 256, 0, st>>>(b.dY, P + m->offW3(), b.A2, B, m->h, m->nout, b.dZ2);
    k_dense_grad_w<<<blocks_for((int64_t)m->h * (m->h + 1)), 256, 0, st>>>(b.dZ2, b.A1, B, m->h, m->h, G + m->offW2(),
                                                                           G + m->offb2());
    k_dense_grad_in<<<blocks_for((int64_t)B * m->h), 256, 0, st>>>(b.dZ2, P + m->offW2(), b.A1, B, m->h, m->h, b.dZ1);
    k_dense_grad_w<<<blocks_for((int64_t)m->h * (m->nin + 1)), 256, 0, st>>>(b.dZ1, b.Xn, B, m->nin, m->h,
                                                                             G + m->offW1(), G + m->offb1());
    ML_CUDA(cudaGetLastError());
    if (loss) {
        std::vector<float> hp(nb);
        ML_CUDA(cudaMemcpyAsync(hp.data(), m->part.p, nb * sizeof(float), cudaMemcpyDeviceToHost, st));
        ML_CUDA(cudaStreamSynchronize(st));
        double s = 0.0;
        for (float v : hp) s += v;
        *loss = (float)(s / (double)cnt);
    }
    return ML_OK;
}

static bool on_device(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// copy (host or device) rows x cols floats into dst (device) and standardise
static ml_status load_std(const float *src, int64_t rows, int cols, const float *mean, const float *stdv, float *dst,
                          cudaStream_t st)
{
    ML_CUDA(cudaMemcpyAsync(dst, src, (size_t)rows * cols * sizeof(float),
                            on_device(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    k_standardise<<<blocks_for(rows * cols), 256, 0, st>>>(dst, rows, cols, mean, stdv, dst);
    ML_CUDA(cudaGetLastError());
    return ML_OK;
}

int auto_bandwidth_box(double sigma, double box, int d, double target);

}  // namespace ml

using namespace ml;

extern "C" {

ml_status ml_mlp_create(ml_mlp_t *out, int n_in, int hidden, int n_out, uint64_t seed)
{
    if (!out || n_in < 1 || hidden < 1 || n_out < 1 || n_in > 4096 || hidden > 4096 || n_out > 4096)
        return fail(ML_ERR_ARG, "bad MLP sizes");
    ml_mlp_s *m = new (std::nothrow) ml_mlp_s;
    if (!m) return fail(ML_ERR_OOM, "host allocation failed");
    m->nin = n_in;
    m->h = hidden;
    m->nout = n_out;
    m->nparam = m->offb3() + n_out;
    std::vector<float> p(m->nparam, 0.0f);
    // Glorot-uniform weights from a SplitMix64 stream, zero biases
    uint64_t z = seed;
    auto uni = [&]() {
        z += 0x9E3779B97F4A7C15ULL;
        uint64_t x = z;
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
        x ^= x >> 31;
        return (double)(x >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    };
    auto fill = [&](int64_t off, int rows, int cols) {
        const double a = std::sqrt(6.0 / (rows + cols));
        for (int64_t i = 0; i < (int64_t)rows * cols; ++i) p[off + i] = (float)(a * uni());
    };
    fill(m->offW1(), hidden, n_in);
    fill(m->offW2(), hidden, hidden);
    fill(m->offW3(), n_out, hidden);
    ml_status st;
    if ((st = m->params.ensure(m->nparam * 4)) != ML_OK || (st = m->grad.ensure(m->nparam * 4)) != ML_OK ||
        (st = m->adam_m.ensure(m->nparam * 4)) != ML_OK || (st = m->adam_v.ensure(m->nparam * 4)) != ML_OK ||
        (st = m->norm.ensure((size_t)2 * (n_in + n_out) * 4)) != ML_OK) {
        delete m;
        return st;
    }
    std::vector<float> nrm(2 * (n_in + n_out), 0.0f);
    for (int i = 0; i < n_in; ++i) nrm[n_in + i] = 1.0f;
    for (int i = 0; i < n_out; ++i) nrm[2 * n_in + n_out + i] = 1.0f;
    cudaMemcpy(m->params.p, p.data(), m->nparam * 4, cudaMemcpyHostToDevice);
    cudaMemset(m->adam_m.p, 0, m->nparam * 4);
    cudaMemset(m->adam_v.p, 0, m->nparam * 4);
    cudaError_t e = cudaMemcpy(m->norm.p, nrm.data(), nrm.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        delete m;
        return cuda_fail(e, "cudaMemcpy", __FILE__, __LINE__);
    }
    *out = m;
    return ML_OK;
}

int64_t ml_mlp_param_count(ml_mlp_t m) { return m ? m->nparam : -1; }

ml_status ml_mlp_get_params(ml_mlp_t m, float *params, int64_t count)
{
    if (!m || !params || count < m->nparam) return fail(ML_ERR_ARG, "bad arguments");
    ML_CUDA(cudaMemcpy(params, m->params.p, m->nparam * 4, cudaMemcpyDeviceToHost));
    return ML_OK;
}

ml_status ml_mlp_set_params(ml_mlp_t m, const float *params, int64_t count)
{
    if (!m || !params || count != m->nparam) return fail(ML_ERR_ARG, "bad arguments");
    ML_CUDA(cudaMemcpy(m->params.p, params, m->nparam * 4, cudaMemcpyHostToDevice));
    ML_CUDA(cudaMemset(m->adam_m.p, 0, m->nparam * 4));
    ML_CUDA(cudaMemset(m->adam_v.p, 0, m->nparam * 4));
    m->adam_t = 0;
    return ML_OK;
}

ml_status ml_mlp_set_norm(ml_mlp_t m, const float *in_mean, const float *in_std, const float *out_mean,
                          const float *out_std)
{
    if (!m || !in_mean || !in_std || !out_mean || !out_std) return fail(ML_ERR_ARG, "null argument");
    std::vector<float> nrm;
    nrm.insert(nrm.end(), in_mean, in_mean + m->nin);
    nrm.insert(nrm.end(), in_std, in_std + m->nin);
    nrm.insert(nrm.end(), out_mean, out_mean + m->nout);
    nrm.insert(nrm.end(), out_std, out_std + m->nout);
    for (int i = 0; i < m->nin; ++i)
        if (!(in_std[i] > 0)) return fail(ML_ERR_ARG, "in_std must be positive");
    for (int i = 0; i < m->nout; ++i)
        if (!(out_std[i] > 0)) return fail(ML_ERR_ARG, "out_std must be positive");
    ML_CUDA(cudaMemcpy(m->norm.p, nrm.data(), nrm.size() * 4, cudaMemcpyHostToDevice));
    return ML_OK;
}

ml_status ml_mlp_set_margins(ml_mlp_t mlp, const double *margins, int count)
{
    if (!mlp || !margins || count != 3) return fail(ML_ERR_ARG, "margins: a model and 3 values are needed");
    for (int f = 0; f < 3; ++f) {
        if (!(margins[f] >= 0.0) || !std::isfinite(margins[f])) return fail(ML_ERR_ARG, "margins must be >= 0");
        mlp->margins[f] = margins[f];
    }
    return ML_OK;
}

ml_status ml_mlp_forward(ml_mlp_t m, const float *X, int batch, float *Y)
{
    if (!m || !X || !Y || batch < 1) return fail(ML_ERR_ARG, "bad arguments");
    cudaStream_t st = 0;
    ML_TRY(mlp_ws(m, batch));
    MlpBufs b = bufs_of(m, batch);
    const float *nrm = m->norm.as<float>();
    {
        ProfScope pr("mlp", st);
        ML_TRY(load_std(X, batch, m->nin, nrm, nrm + m->nin, b.Xn, st));
        forward_std(m, b, batch, st);
        k_unstandardise<<<blocks_for((int64_t)batch * m->nout), 256, 0, st>>>(
            b.Z3, batch, m->nout, nrm + 2 * m->nin, nrm + 2 * m->nin + m->nout, b.T);
    }
    ML_CUDA(cudaGetLastError());
    ML_CUDA(cudaMemcpyAsync(Y, b.T, (size_t)batch * m->nout * 4,
                            on_device(Y) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    ML_CUDA(cudaStreamSynchronize(st));
    return ML_OK;
}

ml_status ml_mlp_loss_grad(ml_mlp_t m, const float *X, const float *Yt, int batch, float *loss, float *grad)
{
    if (!m || !X || !Yt || batch < 1) return fail(ML_ERR_ARG, "bad arguments");
    cudaStream_t st = 0;
    ML_TRY(mlp_ws(m, batch));
    MlpBufs b = bufs_of(m, batch);
    const float *nrm = m->norm.as<float>();
    ML_TRY(load_std(X, batch, m->nin, nrm, nrm + m->nin, b.Xn, st));
    ML_TRY(load_std(Yt, batch, m->nout, nrm + 2 * m->nin, nrm + 2 * m->nin + m->nout, b.T, st));
    ML_TRY(loss_grad_std(m, b, batch, st, loss));
    if (grad) ML_CUDA(cudaMemcpy(grad, m->grad.p, m->nparam * 4, cudaMemcpyDeviceToHost));
    return ML_OK;
}

ml_status ml_mlp_train(ml_mlp_t m, const float *X, const float *Yt, int batch, int epochs, float lr, float *losses)
{
    if (!m || !X || !Yt || batch < 1 || epochs < 0 || !(lr > 0)) return fail(ML_ERR_ARG, "bad arguments");
    cudaStream_t st = 0;
    ML_TRY(mlp_ws(m, batch));
    MlpBufs b = bufs_of(m, batch);
    const float *nrm = m->norm.as<float>();
    ML_TRY(load_std(X, batch, m->nin, nrm, nrm + m->nin, b.Xn, st));
    ML_TRY(load_std(Yt, batch, m->nout, nrm + 2 * m->nin, nrm + 2 * m->nin + m->nout, b.T, st));
    const float b1 = 0.9f, b2 = 0.999f;
    for (int ep = 0; ep < epochs; ++ep) {
        float l = 0.0f;
        ProfScope pr("mlp", st);
        ML_TRY(loss_grad_std(m, b, batch, st, losses ? &l : nullptr));
        m->adam_t += 1;
        const float c1 = 1.0f - std::pow(b1, (float)m->adam_t), c2 = 1.0f - std::pow(b2, (float)m->adam_t);
        k_adam<<<blocks_for(m->nparam), 256, 0, st>>>(m->params.as<float>(), m->grad.as<float>(), m->adam_m.as<float>(),
                                                    m->adam_v.as<float>(), m->nparam, lr, b1, b2, 1e-8f, c1, c2);
        ML_CUDA(cudaGetLastError());
        if (losses) losses[ep] = l;
    }
    ML_CUDA(cudaStreamSynchronize(st));
    return ML_OK;
}

ml_status ml_mlp_destroy(ml_mlp_t m)
{
    if (!m) return ML_OK;
    m->params.release();
    m->grad.release();
    m->adam_m.release();
    m->adam_v.release();
    m->norm.release();
    m->ws.release();
    m->part.release();
    delete m;
    return ML_OK;
}

ml_status ml_fastsum_plan_learned(ml_plan_t *out, const double *points, int64_t n, int d, double sigma, ml_prec prec,
                                  double target_rel_err, ml_mlp_t mlp, double margin, double *chosen, void *stream)
{
    if (!out || !points) return fail(ML_ERR_ARG, "null pointer");
    const double target = target_rel_err > 0 ? target_rel_err : (prec == ML_F32 ? 1e-4 : 1e-6);
    ml_plan_params prm{};
    prm.prec = prec;
    prm.target_rel_err = target;
    double pick[3] = {0.0, 0.0, 0.0};
    if (mlp) {
        if (mlp->nin != ML_FEATURES + 3 || mlp->nout != 2) return fail(ML_ERR_ARG, "model has the wrong shape");
        float feat[ML_FEATURES];
        ML_TRY(ml_cloud_features(points, n, d, sigma, feat, stream));
        const double box = sigma / std::pow(10.0, (double)feat[2]);
        const int N0 = auto_bandwidth_box(sigma, box, d, target);
        const double fs[3] = {0.7, 0.85, 1.0}, ss[3] = {2.0, 2.5, 3.0};
        std::vector<float> Xc;
        std::vector<double> cand;
        for (double f : fs)
            for (int W = 4; W <= 8; ++W)
                for (double s : ss) {
                    Xc.insert(Xc.end(), feat, feat + ML_FEATURES);
                    Xc.push_back((float)f);
                    Xc.push_back((float)W);
                    Xc.push_back((float)s);
                    cand.push_back(f);
                    cand.push_back(W);
                    cand.push_back(s);
                }
        const int B = (int)cand.size() / 3;
        std::vector<float> Yp((size_t)B * 2);
        ML_TRY(ml_mlp_forward(mlp, Xc.data(), B, Yp.data()));
        // per bandwidth factor: the model's own calibrated margin when set, else the caller's
        double lim[3];
        for (int f = 0; f < 3; ++f) {
            const double m = mlp->margins[f] > 0.0 ? mlp->margins[f] : margin;
            lim[f] = std::log10(target / (m > 1.0 ? m : 1.0));
        }
        double best = INFINITY;
        for (int i = 0; i < B; ++i)
            if (Yp[2 * i] <= lim[i / (B / 3)] && Yp[2 * i + 1] < best) {
                best = Yp[2 * i + 1];
                pick[0] = cand[3 * i];
                pick[1] = cand[3 * i + 1];
                pick[2] = cand[3 * i + 2];
            }
        if (best < INFINITY) {
            int N = 2 * (int)std::lround(0.5 * pick[0] * N0);
            prm.N = std::max(4, std::min(N, kMaxN));
            prm.taps = (int)pick[1];
            prm.oversampling = pick[2];
        }
    }
    if (chosen) {
        chosen[0] = pick[0];
        chosen[1] = pick[1];
        chosen[2] = pick[2];
    }
    return ml_fastsum_plan_ex(out, points, n, d, sigma, &prm, stream);
}

}  // extern "C"
