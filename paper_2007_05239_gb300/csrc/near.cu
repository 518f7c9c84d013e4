// The Laplacian kernel K(y) = exp(-||y||/sigma) of Sec. 4 in the fast
// summation: its parameter choices, the Fourier coefficients b_l of its
// regularised form K_R, and the near-field pass that adds K - K_R back on
// ||x_i - x_j|| < eps_I (the scheme for non-smooth radial kernels of the fast
// summation that Sec. 4 cites).
//
// Layout of the near field: the points sorted by a cell list of edge
// h >= eps_I over the scaled domain [-1/4, 1/4]^d, so every pair closer than
// eps_I lies in the same or in adjacent cells.  Each point keeps its
// coordinates relative to its cell's corner (float4 in the FP32 form, double4
// in the FP64 form), so a pair difference is (cell offset) * h + (local
// difference), exact to a few ulp of h instead of ulp of the domain.  One CTA
// of kNearThreads threads takes up to kNearThreads targets of one cell and
// streams the 3^d neighbour cells through shared memory.  The kernel
// difference K - K_R is evaluated in the form's precision: in FP32 a
// systematic rounding bias of ~1e-8 per pair would add up over the near
// pairs, so the FP64 form evaluates it on the FP64 pipes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ml_internal.h"

namespace ml {

// ------------------------------------------------------------- choices
// Largest |K_RF - K_R| measured on probe distances (regularisers of degree
// p = 8, eps_B = max(1/16, c/N), sigma' from 0.005 to 0.3, d = 1..3) by the
// number c = N eps_I of grid cells across the inner region.
static const struct {
    int c;
    double err;
} kCellsErr[] = {{4, 1e-4}, {6, 1.2e-5}, {8, 1.5e-6}, {10, 2.5e-7}, {12, 6e-8}, {14, 1.5e-8}, {16, 4e-9}};

int laplace_cells(double target)
{
    for (const auto &e : kCellsErr)
        if (e.err <= 0.5 * target) return e.c;
    return 16;
}

// One product's time, in picoseconds on a GB300 (per-unit costs measured on
// 1e6-point clouds): the pruned grid transforms, 2 d (N+1) (N+W)^d
// multiply-adds (0.23 ps each in FP32, 2.1 ps in the FP64 form's double-word
// arithmetic), against the near-field pairs a uniform cloud in the ball of
// radius 1/4 - eps_B/2 gives, n rho (3 eps_I)^d examined pairs (0.8 ps each
// in FP32, 39 ps on the FP64 pipes of the FP64 form).
int laplace_bandwidth(int64_t n, int d, int c, int W, ml_prec prec)
{
    static const int cand[] = {16, 24, 32, 40, 48, 64, 80, 96, 128, 160, 192, 256, 320, 384, 448, 512};
    const double wf = prec == ML_F32 ? 0.23 : 2.1, wp = prec == ML_F32 ? 0.8 : 39.0;
    double best = INFINITY;
    int bestN = 0;
    for (int N : cand) {
        if (N < 4 * c + 8) continue;  // eps_I and eps_B = max(1/16, eps_I) leave the ball room
        const double eI = (double)c / N, eB = std::max(1.0 / 16, eI);
        const double r = 0.25 - 0.5 * eB;
        const double vol = d == 1 ? 2.0 * r : d == 2 ? M_PI * r * r : 4.0 / 3.0 * M_PI * r * r * r;
        const double nn = (double)n;
        const double near = std::min(nn * nn, nn * (nn / vol) * std::pow(3.0 * eI, d)) * wp;
        const double far = 2.0 * d * (N + 1) * std::pow((double)(N + W), d) * wf;
        if (near + far < best) {
            best = near + far;
            bestN = N;
        }
    }
    return bestN > 0 ? bestN : 4 * c + 8;
}

// ------------------------------------------------- Fourier coefficients
struct LapRegDev {
    double s, eps_B, eps_I;
    double q[16];
    double c[8];
    int nq, nc;
};

__device__ double lap_reg_eval(double r, const LapRegDev &g)
{
    if (r < g.eps_I) {
        const double r2 = r * r;
        double v = 0.0;
        for (int j = g.nc - 1; j >= 0; --j) v = fma(v, r2, g.c[j]);
        return v;
    }
    if (r <= 0.5 - g.eps_B) return exp(-r / g.s);
    const double t = fmin((r - (0.5 - g.eps_B)) / g.eps_B, 1.0);
    double v = 0.0;
    for (int j = g.nq - 1; j >= 0; --j) v = fma(v, t, g.q[j]);
    return v;
}

// K_R on the grid k/N, k in I_N^d, stored at index k + N/2 per dim (dim 0 fastest)
__global__ void k_lap_samples(double *out, int N, int d, int64_t total, LapRegDev g)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e;
        double r2 = 0.0;
        for (int a = 0; a < d; ++a) {
            const int k = (int)(r % N);
            r /= N;
            const double t = (double)(k - N / 2) / N;
            r2 += t * t;
        }
        out[e] = lap_reg_eval(sqrt(r2), g);
    }
}

// one axis of the cosine sums b_l = N^{-d} sum_k K_R(k/N) prod_a cos(2 pi l_a k_a / N):
// out[o][l][i] = N^{-1} sum_k C[l][k] in[o][k][i], l = 0..N/2
__global__ void k_cos_axis(const double *__restrict__ in, double *__restrict__ out, const double *__restrict__ C,
                           int N, int H, int64_t inner, int64_t total)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % inner;
        const int64_t rest = e / inner;
        const int l = (int)(rest % H);
        const int64_t o = rest / H;
        const double *src = in + o * N * inner + i;
        const double *cr = C + (int64_t)l * N;
        double acc = 0.0;
        for (int k = 0; k < N; ++k) acc = fma(cr[k], src[(int64_t)k * inner], acc);
        out[e] = acc / N;
    }
}

static int blocks_for(int64_t work) { return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, sm_count() * 32)); }

ml_status laplace_fourier(ml_plan_s *p, const LaplaceReg &g, cudaStream_t st)
{
    const int N = p->N, d = p->d, H = N / 2 + 1;
    if (g.q.size() > 16 || g.c.size() > 8) return fail(ML_ERR_ARG, "regulariser degree beyond the limit");
    int64_t total = 1;
    for (int a = 0; a < d; ++a) total *= N;
    DevBuf A, B, Cd;
    ML_TRY(A.ensure((size_t)total * 8));
    ML_TRY(B.ensure((size_t)total * 8));
    std::vector<double> C((size_t)H * N);
    for (int l = 0; l < H; ++l)
        for (int k = 0; k < N; ++k) {
            // reduce l (k - N/2) mod N exactly before scaling to radians
            const long long t = (((long long)l * (long long)(k - N / 2)) % N + N) % N;
            C[(size_t)l * N + k] = std::cos(2.0 * M_PI * (double)t / N);
        }
    ML_TRY(Cd.ensure(C.size() * 8));
    ML_CUDA(cudaMemcpyAsync(Cd.p, C.data(), C.size() * 8, cudaMemcpyHostToDevice, st));
    LapRegDev gd{};
    gd.s = g.s;
    gd.eps_B = g.eps_B;
    gd.eps_I = g.eps_I;
    gd.nq = (int)g.q.size();
    gd.nc = (int)g.c.size();
    for (int j = 0; j < gd.nq; ++j) gd.q[j] = g.q[j];
    for (int j = 0; j < gd.nc; ++j) gd.c[j] = g.c[j];
    {
        ProfScope pr("plan", st);
        k_lap_samples<<<blocks_for(total), 256, 0, st>>>(A.as<double>(), N, d, total, gd);
    }
    ML_CUDA(cudaGetLastError());
    double *cur = A.as<double>(), *nxt = B.as<double>();
    int64_t ext[3] = {1, 1, 1};
    for (int a = 0; a < d; ++a) ext[a] = N;
    for (int a = 0; a < d; ++a) {
        int64_t inner = 1, outer = 1;
        for (int b = 0; b < a; ++b) inner *= ext[b];
        for (int b = a + 1; b < d; ++b) outer *= ext[b];
        const int64_t out_total = outer * H * inner;
        {
            ProfScope pr("plan", st);
            k_cos_axis<<<blocks_for(out_total), 256, 0, st>>>(cur, nxt, Cd.as<double>(), N, H, inner, out_total);
        }
        ML_CUDA(cudaGetLastError());
        std::swap(cur, nxt);
        ext[a] = H;
    }
    int64_t hd = 1;
    for (int a = 0; a < d; ++a) hd *= H;
    p->bhat.assign((size_t)hd, 0.0);
    ML_CUDA(cudaMemcpyAsync(p->bhat.data(), cur, (size_t)hd * 8, cudaMemcpyDeviceToHost, st));
    ML_CUDA(cudaStreamSynchronize(st));
    return ML_OK;
}

// ------------------------------------------------------ near-field plan
struct NfGeom {
    double c[3];
    double s;   // x' = s (x - c); cell coordinate (x' + 1/4) / h
    double h;
    int nc[3];
    int d;
};

__device__ __forceinline__ int nf_cell(double u, double h, int nc)
{
    int c = (int)floor(u / h);
    return min(max(c, 0), nc - 1);
}

// key = cell index << 2d | Morton code of the point's sub-cell on a 4^d
// split of its cell: inside a cell the points of one warp sit close
// together, so a source is in range for all or none of a warp's targets
// except near the shell r = eps_I, and whole warps skip the evaluation
__global__ void k_nf_keys(const double *__restrict__ X, int64_t n, NfGeom g, uint32_t *keys, int *idx)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int cc[3] = {0, 0, 0};
        uint32_t morton = 0;
        for (int a = 0; a < g.d; ++a) {
            const double u = g.s * (X[i * g.d + a] - g.c[a]) + 0.25;
            cc[a] = nf_cell(u, g.h, g.nc[a]);
            const int sub = min(max((int)floor(4.0 * (u - cc[a] * g.h) / g.h), 0), 3);
            morton |= (uint32_t)(sub & 1) << a;
            morton |= (uint32_t)(sub >> 1) << (g.d + a);
        }
        const uint32_t cell = (uint32_t)(((int64_t)cc[2] * g.nc[1] + cc[1]) * g.nc[0] + cc[0]);
        keys[i] = (cell << (2 * g.d)) | morton;
        idx[i] = (int)i;
    }
}

template <typename T> struct Vec4;
template <> struct Vec4<float> {
    using type = float4;
    static __device__ __forceinline__ float4 make(float x, float y, float z) { return make_float4(x, y, z, 0.f); }
};
template <> struct Vec4<double> {
    using type = double4;
    static __device__ __forceinline__ double4 make(double x, double y, double z) { return make_double4(x, y, z, 0.0); }
};

template <typename T>
__global__ void k_nf_fill(const double *__restrict__ X, const int *__restrict__ order, const int *__restrict__ iperm,
                          int64_t n, NfGeom g, typename Vec4<T>::type *loc, int *orig, int *sidx)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int o = order[k];
        T l[3] = {0, 0, 0};
        for (int a = 0; a < g.d; ++a) {
            const double u = g.s * (X[(int64_t)o * g.d + a] - g.c[a]) + 0.25;
            const int c = nf_cell(u, g.h, g.nc[a]);
            l[a] = (T)(u - (double)c * g.h);
        }
        loc[k] = Vec4<T>::make(l[0], l[1], l[2]);
        orig[k] = o;
        sidx[k] = iperm[o];
    }
}

__global__ void k_nf_iperm(const int *__restrict__ perm, int64_t n, int *iperm)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        iperm[perm[i]] = (int)i;
}

__global__ void k_nf_count(const uint32_t *__restrict__ keys, int64_t n, int shift, int *counts)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&counts[keys[i] >> shift], 1);
}

ml_status near_plan(ml_plan_s *p, const double *points, cudaStream_t st)
{
    const int64_t n = p->n;
    const int d = p->d;
    NfGeom g;
    for (int a = 0; a < 3; ++a) {
        g.c[a] = p->center[a];
        g.nc[a] = 1;
    }
    g.s = p->scale;
    g.d = d;
    g.h = p->eps_I * (1.0 + 1e-9);  // pairs closer than eps_I never skip a cell
    int64_t ncells = 1;
    for (int a = 0; a < d; ++a) {
        g.nc[a] = std::max(1, (int)std::ceil(0.5 / g.h));
        ncells *= g.nc[a];
    }
    if (ncells << (2 * d) > (1LL << 31)) return fail(ML_ERR_ARG, "eps_I gives too many near-field cells");
    p->nf_h = g.h;
    for (int a = 0; a < 3; ++a) p->nf_nc[a] = g.nc[a];
    DevBuf keys, keys2, idx, idx2, iperm, counts;
    ML_TRY(keys.ensure((size_t)n * 4));
    ML_TRY(keys2.ensure((size_t)n * 4));
    ML_TRY(idx.ensure((size_t)n * 4));
    ML_TRY(idx2.ensure((size_t)n * 4));
    ML_TRY(iperm.ensure((size_t)n * 4));
    ML_TRY(counts.ensure((size_t)ncells * 4));
    {
        ProfScope pr("plan", st);
        k_nf_keys<<<blocks_for(n), 256, 0, st>>>(points, n, g, keys.as<uint32_t>(), idx.as<int>());
        k_nf_iperm<<<blocks_for(n), 256, 0, st>>>(p->perm.as<int>(), n, iperm.as<int>());
    }
    ML_CUDA(cudaGetLastError());
    int bits = 2 * d;
    while ((1LL << bits) < (ncells << (2 * d))) ++bits;
    int *order = idx.as<int>();
    if (bits > 0) ML_TRY(radix_sort(keys.as<uint32_t>(), idx.as<int>(), keys2.as<uint32_t>(), idx2.as<int>(), n, bits, st, &order));
    const bool f32 = p->prec == ML_F32;
    ML_TRY(p->nf_loc.ensure((size_t)n * (f32 ? sizeof(float4) : sizeof(double4))));
    ML_TRY(p->nf_orig.ensure((size_t)n * 4));
    ML_TRY(p->nf_sidx.ensure((size_t)n * 4));
    ML_CUDA(cudaMemsetAsync(counts.p, 0, (size_t)ncells * 4, st));
    {
        ProfScope pr("plan", st);
        if (f32)
            k_nf_fill<float><<<blocks_for(n), 256, 0, st>>>(points, order, iperm.as<int>(), n, g, p->nf_loc.as<float4>(),
                                                            p->nf_orig.as<int>(), p->nf_sidx.as<int>());
        else
            k_nf_fill<double><<<blocks_for(n), 256, 0, st>>>(points, order, iperm.as<int>(), n, g,
                                                             p->nf_loc.as<double4>(), p->nf_orig.as<int>(),
                                                             p->nf_sidx.as<int>());
        k_nf_count<<<blocks_for(n), 256, 0, st>>>(keys.as<uint32_t>(), n, 2 * d, counts.as<int>());
    }
    ML_CUDA(cudaGetLastError());
    std::vector<int> hc((size_t)ncells);
    ML_CUDA(cudaMemcpyAsync(hc.data(), counts.p, (size_t)ncells * 4, cudaMemcpyDeviceToHost, st));
    ML_CUDA(cudaStreamSynchronize(st));
    std::vector<int> start((size_t)ncells + 1);
    std::vector<int> tasks;
    int64_t pos = 0;
    for (int64_t c = 0; c < ncells; ++c) {
        start[c] = (int)pos;
        for (int q = 0; q < hc[c]; q += kNearThreads) {
            tasks.push_back((int)c);
            tasks.push_back((int)(pos + q));
            tasks.push_back(std::min(kNearThreads, hc[c] - q));
            tasks.push_back(0);
        }
        pos += hc[c];
    }
    start[ncells] = (int)pos;
    // pairs examined: every point against the points of its 3^d neighbour cells
    int64_t pairs = 0;
    const int n0 = g.nc[0], n1 = g.nc[1], n2 = g.nc[2];
    for (int z = 0; z < n2; ++z)
        for (int y = 0; y < n1; ++y)
            for (int x = 0; x < n0; ++x) {
                const int64_t c = ((int64_t)z * n1 + y) * n0 + x;
                if (hc[c] == 0) continue;
                int64_t nb = 0;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int X2 = x + dx, Y2 = y + dy, Z2 = z + dz;
                            if (X2 < 0 || X2 >= n0 || Y2 < 0 || Y2 >= n1 || Z2 < 0 || Z2 >= n2) continue;
                            nb += hc[((int64_t)Z2 * n1 + Y2) * n0 + X2];
                        }
                pairs += (int64_t)hc[c] * nb;
            }
    p->near_pairs = pairs;
    if (pairs > (1LL << 40))
        return fail(ML_ERR_DOMAIN, "near field of the Laplacian too dense (" + std::to_string(pairs) +
                                       " pairs per vector): the points cluster within eps_I");
    p->nf_ntask = (int)(tasks.size() / 4);
    ML_TRY(p->nf_start.ensure(start.size() * 4));
    ML_TRY(p->nf_task.ensure(std::max<size_t>(16, tasks.size() * 4)));
    ML_CUDA(cudaMemcpyAsync(p->nf_start.p, start.data(), start.size() * 4, cudaMemcpyHostToDevice, st));
    if (!tasks.empty())
        ML_CUDA(cudaMemcpyAsync(p->nf_task.p, tasks.data(), tasks.size() * 4, cudaMemcpyHostToDevice, st));
    ML_CUDA(cudaStreamSynchronize(st));
    return ML_OK;
}

// ------------------------------------------------------ near-field pass
struct NearArgs {
    const void *loc;      // float4 (FP32 form) or double4 (FP64 form) per point
    const int *orig, *sidx, *start;
    const int4 *task;
    const double *dinv;   // pre/post scale (normalised products) or null
    const double *X;      // input, point-major with row stride ldx, or null (ones)
    int ldx;
    double *Y;
    int ldy;
    int nv;
    int nc0, nc1, nc2;
    double h, eps2, inv_s;
    double c[8];          // inner polynomial in r^2, zero beyond its degree
    double alpha;
    int sorted_out;
};

// exp(-r / sigma') from r^2.  FP32: r = r^2 rsqrt(r^2) (the self pair r^2 = 0
// kept at r = 0) and 2^(-r k) with k = log2(e) / sigma' on the special-function
// unit, each within a few ulp, far inside the FP32 form's accuracy; FP64: the
// correctly rounded library functions.
__device__ __forceinline__ float kernel_of_r2(float r2, float k)
{
    const float r = r2 * rsqrtf(fmaxf(r2, 1e-30f));
    return exp2f(-r * k);
}
__device__ __forceinline__ double kernel_of_r2(double r2, double k) { return exp(-sqrt(r2) * k); }

// y_i += alpha * s_i * sum_{j: r_ij < eps_I} (exp(-r_ij/sigma') - P(r_ij^2)) u_j,
// u_j = s_j x_j (s = D^{-1/2} for normalised products, else 1); in sorted
// order and unscaled for the degree set-up.  T = float: the FP32 form
// (accumulated per staged chunk in FP32, then in FP64); T = double: the FP64
// form, every step in FP64.
template <typename T, int D, int NV>
__global__ void __launch_bounds__(kNearThreads) k_near(const NearArgs a)
{
    using V4 = typename Vec4<T>::type;
    __shared__ V4 sp[kNearThreads];
    __shared__ T su[kNearThreads * NV];
    const V4 *loc = static_cast<const V4 *>(a.loc);
    const int4 tk = a.task[blockIdx.x];
    const int cx = tk.x % a.nc0;
    const int cy = (D >= 2) ? (tk.x / a.nc0) % a.nc1 : 0;
    const int cz = (D >= 3) ? tk.x / (a.nc0 * a.nc1) : 0;
    const int t = threadIdx.x;
    const bool act = t < tk.z;
    const int k = tk.y + t;
    const V4 xi = act ? loc[k] : Vec4<T>::make(0, 0, 0);
    const T h = (T)a.h, eps2 = (T)a.eps2;
    const T kexp = sizeof(T) == 4 ? (T)(a.inv_s * 1.4426950408889634) : (T)a.inv_s;   // log2(e) / sigma' in FP32
    T cf[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) cf[j] = (T)a.c[j];
    double tot[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) tot[c] = 0.0;
    for (int dz = (D >= 3 ? -1 : 0); dz <= (D >= 3 ? 1 : 0); ++dz) {
        const int z = cz + dz;
        if (z < 0 || z >= a.nc2) continue;
        for (int dy = (D >= 2 ? -1 : 0); dy <= (D >= 2 ? 1 : 0); ++dy) {
            const int y = cy + dy;
            if (y < 0 || y >= a.nc1) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                const int x = cx + dx;
                if (x < 0 || x >= a.nc0) continue;
                const int nb = (z * a.nc1 + y) * a.nc0 + x;
                const int s0 = a.start[nb], s1 = a.start[nb + 1];
                const T ox = dx * h, oy = dy * h, oz = dz * h;
                for (int j0 = s0; j0 < s1; j0 += kNearThreads) {
                    __syncthreads();
                    const int j = j0 + t;
                    if (j < s1) {
                        const V4 q = loc[j];
                        sp[t] = Vec4<T>::make(q.x + ox, q.y + oy, q.z + oz);
                        const double ds = a.dinv ? a.dinv[a.sidx[j]] : 1.0;
                        const int64_t o = a.orig[j];
#pragma unroll
                        for (int c = 0; c < NV; ++c)
                            su[t * NV + c] = (c < a.nv) ? (T)((a.X ? a.X[o * a.ldx + c] : 1.0) * ds) : (T)0;
                    }
                    __syncthreads();
                    if (!act) continue;
                    const int m = min(kNearThreads, s1 - j0);
                    T acc[NV];
#pragma unroll
                    for (int c = 0; c < NV; ++c) acc[c] = 0;
#pragma unroll 4
                    for (int s = 0; s < m; ++s) {
                        const V4 q = sp[s];
                        const T ex = xi.x - q.x;
                        T r2 = ex * ex;
                        if (D >= 2) {
                            const T ey = xi.y - q.y;
                            r2 = fma(ey, ey, r2);
                        }
                        if (D >= 3) {
                            const T ez = xi.z - q.z;
                            r2 = fma(ez, ez, r2);
                        }
                        if (r2 < eps2) {
                            T P = cf[7];
#pragma unroll
                            for (int jj = 6; jj >= 0; --jj) P = fma(P, r2, cf[jj]);
                            const T delta = kernel_of_r2(r2, kexp) - P;
#pragma unroll
                            for (int c = 0; c < NV; ++c) acc[c] = fma(delta, su[s * NV + c], acc[c]);
                        }
                    }
#pragma unroll
                    for (int c = 0; c < NV; ++c) tot[c] += (double)acc[c];
                }
            }
        }
    }
    if (!act) return;
    if (a.sorted_out) {
        const int64_t i = a.sidx[k];
#pragma unroll
        for (int c = 0; c < NV; ++c)
            if (c < a.nv) a.Y[i * a.ldy + c] += tot[c];
    } else {
        const double ds = a.dinv ? a.dinv[a.sidx[k]] : 1.0;
        const int64_t o = a.orig[k];
#pragma unroll
        for (int c = 0; c < NV; ++c)
            if (c < a.nv) a.Y[o * a.ldy + c] += a.alpha * ds * tot[c];
    }
}

template <typename T, int D>
static void launch_near(const NearArgs &a, int ntask, cudaStream_t st)
{
    if (a.nv <= 1) k_near<T, D, 1><<<ntask, kNearThreads, 0, st>>>(a);
    else if (a.nv <= 4) k_near<T, D, 4><<<ntask, kNearThreads, 0, st>>>(a);
    else k_near<T, D, 8><<<ntask, kNearThreads, 0, st>>>(a);
}

template <typename T>
static void launch_near_d(const NearArgs &a, int d, int ntask, cudaStream_t st)
{
    switch (d) {
    case 1: launch_near<T, 1>(a, ntask, st); break;
    case 2: launch_near<T, 2>(a, ntask, st); break;
    default: launch_near<T, 3>(a, ntask, st); break;
    }
}

ml_status run_near(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, cudaStream_t st)
{
    if (p->nf_ntask == 0) return ML_OK;
    if (v.nv < 1 || v.nv > kMaxVec) return fail(ML_ERR_ARG, "vectors per pass out of range");
    NearArgs a;
    a.loc = p->nf_loc.p;
    a.orig = p->nf_orig.as<int>();
    a.sidx = p->nf_sidx.as<int>();
    a.start = p->nf_start.as<int>();
    a.task = p->nf_task.as<int4>();
    a.dinv = o.normalized ? p->dinv.as<double>() : nullptr;
    a.X = v.X;
    a.ldx = v.ldx;
    a.Y = v.Y;
    a.ldy = v.ldy;
    a.nv = v.nv;
    a.nc0 = p->nf_nc[0];
    a.nc1 = p->nf_nc[1];
    a.nc2 = p->nf_nc[2];
    a.h = p->nf_h;
    a.eps2 = p->eps_I * p->eps_I;
    a.inv_s = 1.0 / p->sigma_s;
    for (int j = 0; j < 8; ++j) a.c[j] = j < (int)p->nf_poly.size() ? p->nf_poly[j] : 0.0;
    a.alpha = o.alpha;
    a.sorted_out = o.sorted_out ? 1 : 0;
    {
        ProfScope pr("near", st);
        if (p->prec == ML_F32) launch_near_d<float>(a, p->d, p->nf_ntask, st);
        else launch_near_d<double>(a, p->d, p->nf_ntask, st);
    }
    ML_CUDA(cudaGetLastError());
    return ML_OK;
}

}  // namespace ml
