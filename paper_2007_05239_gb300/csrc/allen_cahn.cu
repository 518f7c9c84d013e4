// ml_allen_cahn: the multiclass multilayer graph Allen-Cahn scheme (Alg. 2,
// Sec. 6-7) on the GPU, from the eigenpairs (Phi_k, Lambda_k) of the
// (power mean) Laplacian.
//
// Iteration l of Alg. 2, with Z = D^{-1} Phi_k^T, D = (1 + c dt) I + eps dt Lambda_k:
//   R^l     = (1 + c dt) U^l - dt/(2 eps) T(U^l) - dt omega (U^l - F)   (row-local)
//   V^{l+1} = D^{-1} Phi_k^T R^l                                        (reduction over rows)
//   U^{l+1} = rows of Phi_k V^{l+1} projected onto the Gibbs simplex     (row-local)
//   change  = max_i ||u_i^{l+1} - u_i^l||^2 / max_i ||u_i^{l+1}||^2      (reduction)
// One pass per iteration does the row-local work of U^{l+1} and R^{l+1}
// together and accumulates Phi_k^T R^{l+1} (each warp stages 32 rows of
// Phi and R in shared memory and its lanes own output entries), then a
// small kernel sums the per-CTA partials in a fixed order.  U is double
// buffered so that the host can test the change of iteration l while the
// pass of iteration l+1 runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ml_internal.h"

namespace ml {
namespace {

constexpr int kAcMaxK = 64;
constexpr int kAcWarps = 4;

struct AcArgs {
    const double *Phi;   // n x k, column-major
    int64_t n;
    int k;
    const int *labels;   // class id or -1
    const double *V;     // k x M (row-major), null on the first pass
    const double *Uin;   // n x M
    double *Uout;        // n x M (may equal Uin on the first pass)
    double a1;           // 1 + c dt
    double a2;           // dt / (2 eps)
    double a3;           // dt * omega0
    double *partV;       // gridDim.x x (k M)
    double *partC;       // gridDim.x x 2
};

// Gibbs-simplex projection of y (length M) by sort-and-threshold (Chen & Ye 2011)
template <int M>
__device__ __forceinline__ void project_simplex(const double *y, double *x)
{
    double s[M];
#pragma unroll
    for (int q = 0; q < M; ++q) s[q] = y[q];
    // insertion sort, ascending
#pragma unroll
    for (int q = 1; q < M; ++q) {
        const double v = s[q];
        int r = q - 1;
        while (r >= 0 && s[r] > v) {
            s[r + 1] = s[r];
            --r;
        }
        s[r + 1] = v;
    }
    double tot = 0.0;
#pragma unroll
    for (int q = 0; q < M; ++q) tot += s[q];
    double t = (tot - 1.0) / M;
    double tail = 0.0;
    for (int i = M - 1; i >= 1; --i) {   // threshold over the top M - i entries
        tail += s[i];
        const double ti = (tail - 1.0) / (M - i);
        if (ti >= s[i - 1]) {
            t = ti;
            break;
        }
    }
#pragma unroll
    for (int q = 0; q < M; ++q) x[q] = fmax(y[q] - t, 0.0);
}

template <int M>
__global__ void __launch_bounds__(kAcWarps * 32) k_ac_pass(const AcArgs a)
{
    extern __shared__ double acs[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = a.k, KM = k * M;
    double *Vs = acs;                                           // k x M
    double *Ps = Vs + KM + (warp * 32) * (k + 1 + M + 1);       // this warp: 32 x (k+1), then 32 x (M+1)
    double *Rs = Ps + 32 * (k + 1);
    double *red = acs + KM + kAcWarps * 32 * (k + 1 + M + 1);   // kAcWarps x KM, then kAcWarps x 2
    double *acc = red + warp * KM;   // this warp's partial Phi^T R; entry e owned by lane e % 32
    for (int e = threadIdx.x; e < KM; e += blockDim.x) Vs[e] = a.V ? a.V[e] : 0.0;
    for (int e = lane; e < KM; e += 32) acc[e] = 0.0;
    __syncthreads();
    double mx_d = 0.0, mx_u = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + warp * 32; base < a.n; base += stride) {
        const int64_t i = base + lane;
        const bool live = i < a.n;
        double u[M], r[M];
        if (live) {
            for (int j = 0; j < k; ++j) Ps[lane * (k + 1) + j] = a.Phi[(int64_t)j * a.n + i];
            if (a.V) {
                double y[M];
#pragma unroll
                for (int c = 0; c < M; ++c) y[c] = 0.0;
                for (int j = 0; j < k; ++j) {
                    const double ph = Ps[lane * (k + 1) + j];
#pragma unroll
                    for (int c = 0; c < M; ++c) y[c] = fma(ph, Vs[j * M + c], y[c]);
                }
                project_simplex<M>(y, u);
                double dd = 0.0, uu = 0.0;
#pragma unroll
                for (int c = 0; c < M; ++c) {
                    const double old = a.Uin[i * M + c];
                    dd += (u[c] - old) * (u[c] - old);
                    uu += u[c] * u[c];
                    a.Uout[i * M + c] = u[c];
                }
                mx_d = fmax(mx_d, dd);
                mx_u = fmax(mx_u, uu);
            } else {
#pragma unroll
                for (int c = 0; c < M; ++c) u[c] = a.Uin[i * M + c];
            }
            // T(u): a_q = ||u - e_q||_1, P_q = a_q^2 / 4, g_q = a_q prod_{p != q} P_p,
            // T_j = (1/2) sum_q g_q - g_j
            double sabs = 0.0;
#pragma unroll
            for (int c = 0; c < M; ++c) sabs += fabs(u[c]);
            double aq[M], pre[M + 1], suf[M + 1];
#pragma unroll
            for (int q = 0; q < M; ++q) aq[q] = sabs - fabs(u[q]) + fabs(u[q] - 1.0);
            pre[0] = 1.0;
#pragma unroll
            for (int q = 0; q < M; ++q) pre[q + 1] = pre[q] * 0.25 * aq[q] * aq[q];
            suf[M] = 1.0;
#pragma unroll
            for (int q = M - 1; q >= 0; --q) suf[q] = suf[q + 1] * 0.25 * aq[q] * aq[q];
            double g[M], G = 0.0;
#pragma unroll
            for (int q = 0; q < M; ++q) {
                g[q] = aq[q] * pre[q] * suf[q + 1];
                G += g[q];
            }
            const int lab = a.labels[i];
#pragma unroll
            for (int c = 0; c < M; ++c) {
                const double T = 0.5 * G - g[c];
                const double fid = lab >= 0 ? a.a3 * (u[c] - (c == lab ? 1.0 : 0.0)) : 0.0;
                r[c] = a.a1 * u[c] - a.a2 * T - fid;
            }
        } else {
            for (int j = 0; j < k; ++j) Ps[lane * (k + 1) + j] = 0.0;
#pragma unroll
            for (int c = 0; c < M; ++c) r[c] = 0.0;
        }
#pragma unroll
        for (int c = 0; c < M; ++c) Rs[lane * (M + 1) + c] = r[c];
        __syncwarp();
        // lane owns output entries e = lane + 32 q of Phi^T R (row-major k x M)
        for (int e = lane; e < KM; e += 32) {
            const int j = e / M, c = e - j * M;
            double s = acc[e];
#pragma unroll 8
            for (int rr = 0; rr < 32; ++rr) s = fma(Ps[rr * (k + 1) + j], Rs[rr * (M + 1) + c], s);
            acc[e] = s;
        }
        __syncwarp();
    }
    // CTA partials (fixed order over warps)
    for (int o = 16; o > 0; o >>= 1) {
        mx_d = fmax(mx_d, __shfl_xor_sync(0xffffffffu, mx_d, o));
        mx_u = fmax(mx_u, __shfl_xor_sync(0xffffffffu, mx_u, o));
    }
    double *redc = red + kAcWarps * KM;
    if (lane == 0) {
        redc[warp * 2] = mx_d;
        redc[warp * 2 + 1] = mx_u;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < KM; e += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < kAcWarps; ++w) s += red[w * KM + e];
        a.partV[(int64_t)blockIdx.x * KM + e] = s;
    }
    if (threadIdx.x == 0) {
        double d = 0.0, uu = 0.0;
        for (int w = 0; w < kAcWarps; ++w) {
            d = fmax(d, redc[w * 2]);
            uu = fmax(uu, redc[w * 2 + 1]);
        }
        a.partC[blockIdx.x * 2] = d;
        a.partC[blockIdx.x * 2 + 1] = uu;
    }
}

// One CTA per output entry e < KM: V[e] = dinv[e / M] * sum_b partV[b][e], the
// sum over the nblk partials as strided per-thread sums and a shared-memory
// tree (fixed order); CTA KM: change = max_b d_b / max_b u_b.
__global__ void __launch_bounds__(256) k_ac_reduce(const double *__restrict__ partV, const double *__restrict__ partC,
                                                  int nblk, int KM, int M, const double *__restrict__ dinv, double *V,
                                                  double *change)
{
    __shared__ double sa[256], sb[256];
    const int e = blockIdx.x;
    double x = 0.0, y = 0.0;
    if (e < KM) {
        for (int b = threadIdx.x; b < nblk; b += blockDim.x) x += partV[(int64_t)b * KM + e];
    } else {
        for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
            x = fmax(x, partC[b * 2]);
            y = fmax(y, partC[b * 2 + 1]);
        }
    }
    sa[threadIdx.x] = x;
    sb[threadIdx.x] = y;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            if (e < KM) {
                sa[threadIdx.x] += sa[threadIdx.x + h];
            } else {
                sa[threadIdx.x] = fmax(sa[threadIdx.x], sa[threadIdx.x + h]);
                sb[threadIdx.x] = fmax(sb[threadIdx.x], sb[threadIdx.x + h]);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (e < KM) V[e] = dinv[e / M] * sa[0];
        else *change = sb[0] > 0.0 ? sa[0] / sb[0] : 0.0;
    }
}

// U^0: e_j for labelled rows, 1/M elsewhere
__global__ void k_ac_init(const int *__restrict__ labels, int64_t n, int M, double *U)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * M; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / M;
        const int c = (int)(e - i * M);
        const int lab = labels[i];
        U[e] = lab >= 0 ? (c == lab ? 1.0 : 0.0) : 1.0 / M;
    }
}

// row-wise argmax, ties to the lowest class id
__global__ void k_ac_predict(const double *__restrict__ U, int64_t n, int M, int *pred)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int best = 0;
        double bv = U[i * M];
        for (int c = 1; c < M; ++c)
            if (U[i * M + c] > bv) {
                bv = U[i * M + c];
                best = c;
            }
        pred[i] = best;
    }
}

__global__ void k_ac_labels_ok(const int *__restrict__ labels, int64_t n, int M, int *bad)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (labels[i] < -1 || labels[i] >= M) atomicOr(bad, 1);
}

template <int M>
ml_status launch_pass(const AcArgs &a, int nblk, cudaStream_t st)
{
    const size_t smem =
        ((size_t)a.k * M + (size_t)kAcWarps * 32 * (a.k + 1 + M + 1) + (size_t)kAcWarps * (a.k * M + 2)) *
        sizeof(double);
    if (smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_ac_pass<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute", __FILE__, __LINE__);
    }
    ProfScope pr("allen_cahn", st);
    k_ac_pass<M><<<nblk, kAcWarps * 32, smem, st>>>(a);
    ML_CUDA(cudaGetLastError());
    return ML_OK;
}

ml_status pass_dispatch(int M, const AcArgs &a, int nblk, cudaStream_t st)
{
    switch (M) {
#define ML_AC_CASE(MM) \
    case MM: return launch_pass<MM>(a, nblk, st);
        ML_AC_CASE(2)
        ML_AC_CASE(3)
        ML_AC_CASE(4)
        ML_AC_CASE(5)
        ML_AC_CASE(6)
        ML_AC_CASE(7)
        ML_AC_CASE(8)
        ML_AC_CASE(9)
        ML_AC_CASE(10)
        ML_AC_CASE(11)
        ML_AC_CASE(12)
        ML_AC_CASE(13)
        ML_AC_CASE(14)
        ML_AC_CASE(15)
        ML_AC_CASE(16)
#undef ML_AC_CASE
    default: return fail(ML_ERR_ARG, "m must be in [2, 16]");
    }
}

}  // namespace
}  // namespace ml

extern "C" ml_status ml_allen_cahn(const double *Phi, const double *lambda, int64_t n, int k, const int *labels, int m,
                                   const ml_ac_params *prm, double *U, int *pred, int *iters, double *last_change,
                                   void *stream)
{
    using namespace ml;
    if (!Phi || !lambda || !labels || !prm || !U) return fail(ML_ERR_ARG, "null argument");
    if (n < 1 || k < 1 || k > kAcMaxK) return fail(ML_ERR_ARG, "need n >= 1 and 1 <= k <= 64");
    if (m < 2 || m > 16) return fail(ML_ERR_ARG, "m must be in [2, 16]");
    if (!(prm->eps > 0) || !(prm->dt > 0) || !(prm->omega0 >= 0) || prm->max_iter < 1)
        return fail(ML_ERR_ARG, "need eps > 0, dt > 0, omega0 >= 0, max_iter >= 1");
    const double c = prm->c > 0 ? prm->c : prm->omega0 + 3.0 / prm->eps;
    cudaStream_t st = (cudaStream_t)stream;
    const int KM = k * m;
    const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>((n + kAcWarps * 32 - 1) / (kAcWarps * 32), sm_count() * 8));
    DevBuf Ub, partV, partC, Vd, dinv, scal;
    ML_TRY(Ub.ensure((size_t)n * m * sizeof(double)));
    ML_TRY(partV.ensure((size_t)nblk * KM * sizeof(double)));
    ML_TRY(partC.ensure((size_t)nblk * 2 * sizeof(double)));
    ML_TRY(Vd.ensure((size_t)KM * sizeof(double)));
    ML_TRY(dinv.ensure((size_t)k * sizeof(double)));
    ML_TRY(scal.ensure(4 * sizeof(double)));
    {
        ML_CUDA(cudaMemsetAsync(scal.p, 0, sizeof(int), st));
        k_ac_labels_ok<<<(int)std::min<int64_t>((n + 255) / 256, sm_count() * 8), 256, 0, st>>>(labels, n, m, scal.as<int>());
        int bad = 0;
        ML_CUDA(cudaMemcpyAsync(&bad, scal.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        ML_CUDA(cudaStreamSynchronize(st));
        if (bad) return fail(ML_ERR_ARG, "labels must be -1 or in [0, m)");
    }
    std::vector<double> dh(k);
    for (int j = 0; j < k; ++j) dh[j] = 1.0 / ((1.0 + c * prm->dt) + prm->eps * prm->dt * lambda[j]);
    ML_CUDA(cudaMemcpyAsync(dinv.p, dh.data(), k * sizeof(double), cudaMemcpyHostToDevice, st));
    // U (caller's buffer) and Ub alternate; iterate l's result lands in buf[l & 1]
    double *buf[2] = {U, Ub.as<double>()};
    {
        ProfScope pr("allen_cahn", st);
        k_ac_init<<<(int)std::min<int64_t>((n * m + 255) / 256, sm_count() * 16), 256, 0, st>>>(labels, n, m, buf[0]);
    }
    ML_CUDA(cudaGetLastError());
    AcArgs a;
    a.Phi = Phi;
    a.n = n;
    a.k = k;
    a.labels = labels;
    a.a1 = 1.0 + c * prm->dt;
    a.a2 = prm->dt / (2.0 * prm->eps);
    a.a3 = prm->dt * prm->omega0;
    a.partV = partV.as<double>();
    a.partC = partC.as<double>();
    // pass 0: R^0 from U^0 -> V^1
    a.V = nullptr;
    a.Uin = buf[0];
    a.Uout = buf[0];
    ML_TRY(pass_dispatch(m, a, nblk, st));
    double *chg = scal.as<double>() + 1;
    {
        ProfScope pr("allen_cahn", st);
        k_ac_reduce<<<KM + 1, 256, 0, st>>>(partV.as<double>(), partC.as<double>(), nblk, KM, m, dinv.as<double>(),
                                       Vd.as<double>(), chg);
    }
    ML_CUDA(cudaGetLastError());
    // iterations l = 1..max_iter: U^l = P(Phi V^l) into buf[l & 1], change of l,
    // R^l -> V^{l+1}; the change of l is read on the host while pass l+1 runs
    double *hchg = nullptr;
    ML_CUDA(cudaMallocHost(&hchg, 2 * sizeof(double)));
    cudaEvent_t ev[2] = {nullptr, nullptr};
    ml_status s = ML_OK;
    for (int q = 0; q < 2 && s == ML_OK; ++q) {
        const cudaError_t e = cudaEventCreateWithFlags(&ev[q], cudaEventDisableTiming);
        if (e != cudaSuccess) s = cuda_fail(e, "cudaEventCreate", __FILE__, __LINE__);
    }
    int done_at = 0;
    double final_change = 0.0;
    for (int l = 1; l <= prm->max_iter && s == ML_OK && done_at == 0; ++l) {
        a.V = Vd.as<double>();
        a.Uin = buf[(l - 1) & 1];
        a.Uout = buf[l & 1];
        s = pass_dispatch(m, a, nblk, st);
        if (s != ML_OK) break;
        {
            ProfScope pr("allen_cahn", st);
            k_ac_reduce<<<KM + 1, 256, 0, st>>>(partV.as<double>(), partC.as<double>(), nblk, KM, m, dinv.as<double>(),
                                           Vd.as<double>(), chg);
        }
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(hchg + (l & 1), chg, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaEventRecord(ev[l & 1], st);
        if (e != cudaSuccess) {
            s = cuda_fail(e, "Allen-Cahn iteration", __FILE__, __LINE__);
            break;
        }
        // test iteration l-1 (lagged), and iteration l itself at the limit
        if (l >= 2) {
            e = cudaEventSynchronize(ev[(l - 1) & 1]);
            if (e != cudaSuccess) {
                s = cuda_fail(e, "cudaEventSynchronize", __FILE__, __LINE__);
                break;
            }
            if (!(hchg[(l - 1) & 1] > prm->tol)) {
                done_at = l - 1;
                final_change = hchg[(l - 1) & 1];
            }
        }
        if (done_at == 0 && l == prm->max_iter) {
            e = cudaEventSynchronize(ev[l & 1]);
            if (e != cudaSuccess) {
                s = cuda_fail(e, "cudaEventSynchronize", __FILE__, __LINE__);
                break;
            }
            done_at = l;
            final_change = hchg[l & 1];
        }
    }
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    cudaFreeHost(hchg);
    if (s != ML_OK) return s;
    // the result of iteration done_at sits in buf[done_at & 1]
    if (done_at & 1)
        ML_CUDA(cudaMemcpyAsync(U, buf[1], (size_t)n * m * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (pred) {
        ProfScope pr("allen_cahn", st);
        k_ac_predict<<<(int)std::min<int64_t>((n + 255) / 256, sm_count() * 16), 256, 0, st>>>(U, n, m, pred);
    }
    ML_CUDA(cudaGetLastError());
    ML_CUDA(cudaStreamSynchronize(st));
    if (iters) *iters = done_at;
    if (last_change) *last_change = final_change;
    return ML_OK;
}
