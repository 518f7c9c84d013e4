// ml_lanczos_eigs: k smallest eigenpairs of L_1 (Eq. I-L_1) or L_{-1,delta}
// (Eq. L_p_delta_power_p) by the Lanczos method (Sec. 3).
//
// Thick-restart Lanczos (Wu & Simon) on the symmetric operator
//   p =  1: Op = I - L_1 = (1/T) sum_t D_t^{-1/2} W_t D_t^{-1/2}
//   p < 0:  Op = L_{p,delta}^p = (1/T) sum_t (L_sym^(t) + delta I)^p,
//           delta = log(1 + |p|): for p = -1 each term by conjugate gradients,
//           otherwise by the Lanczos approximation of the matrix power (PowerOp)
// for its k largest eigenvalues.  The Krylov basis Q (n x (ncv+1), column
// major, FP64) lives on the device; every new vector has the three-term
// recurrence's terms removed and is then orthogonalised against all columns
// by classical Gram-Schmidt, a second time where the first pass removed
// most of its norm (Workspace::lanczos_step), with deterministic block
// reductions.  The projected (ncv x ncv) matrix and its
// eigendecomposition are on the host in FP64.  For p = -1 each term
// (L_sym^(t) + delta I)^{-1} x is a conjugate-gradient solve whose matvec is
// the fast summation of layer t (the polynomial Krylov approach of Sec. 3
// specialised to the inverse, an SPD solve with condition <= (2+delta)/delta).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <string>
#include <vector>

#include "dword.cuh"
#include "ml_internal.h"

namespace ml {

ml_status apply_device(ml_plan_s *const *layers, int T, const double *X, int b, double *Y, int mode, cudaStream_t st);

constexpr int kDotThreads = 256;
// outputs of every 16 that the Ritz combination gives to the FP64 pipe: a
// double-word multiply-add costs about 12 FP32 issue slots, a DFMA 1/64 of
// the FP32 rate; two of sixteen balance the two pipes
constexpr int kCombineFp64 = 2;

// partial dot products of columns c0.. of Q (column stride n) with x
__global__ void __launch_bounds__(kDotThreads) k_dots(const double *__restrict__ Q, int64_t ldq, int64_t n, int ncol,
                                                      const double *__restrict__ x, double *part)
{
    __shared__ double red[kDotThreads / 32][8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c0 = 0; c0 < ncol; c0 += 8) {
        double acc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = 0.0;
        for (int64_t r = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; r < n; r += (int64_t)gridDim.x * kDotThreads) {
            const double xr = x[r];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (c0 + k < ncol) acc[k] = fma(Q[(int64_t)(c0 + k) * ldq + r], xr, acc[k]);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            double v = acc[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][k] = v;
        }
        __syncthreads();
        if (threadIdx.x < 8 && c0 + (int)threadIdx.x < ncol) {
            double s = 0.0;
            for (int w = 0; w < kDotThreads / 32; ++w) s += red[w][threadIdx.x];
            part[(int64_t)blockIdx.x * ncol + c0 + threadIdx.x] = s;
        }
        __syncthreads();
    }
}

// out[c] = sum over blocks of part[b][c]: one warp per column, lanes stride
// over the blocks, then a shuffle tree (fixed order, deterministic)
__global__ void k_reduce_cols(const double *__restrict__ part, int nblk, int ncol, double *out)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int c = warp; c < ncol; c += nw) {
        double s = 0.0;
        for (int b = lane; b < nblk; b += 32) s += part[(int64_t)b * ncol + c];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[c] = s;
    }
}

// ---- conjugate gradient with device-resident scalars
// sc[0] = r.r (current), sc[1] = p.Ap, sc[2] = alpha, sc[3] = beta, sc[4] = r.r (new)

// partial sums of a.b per block
__global__ void __launch_bounds__(256) k_dot_part(const double *__restrict__ x, const double *__restrict__ y, int64_t n,
                                                  double *part)
{
    __shared__ double red[8];
    double s = 0.0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        s = fma(x[r], y[r], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// one warp: total of the partials, then the CG scalar update
//   which = 0: sc[1] = p.Ap, sc[2] = alpha = sc[0] / sc[1]
//   which = 1: sc[4] = r.r, sc[3] = beta = sc[4] / sc[0], sc[0] = sc[4]
//   which = 2: sc[0] = total (initial r.r)
__global__ void k_cg_scalars(const double *__restrict__ part, int nblk, int which, double *sc)
{
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) s += part[b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) {
        if (which == 0) {
            sc[1] = s;
            sc[2] = (s > 0.0) ? sc[0] / s : 0.0;
        } else if (which == 1) {
            sc[4] = s;
            sc[3] = (sc[0] > 0.0) ? s / sc[0] : 0.0;
            sc[0] = s;
        } else {
            sc[0] = s;
        }
    }
}

// y += alpha p; r -= alpha Ap; partial sums of r.r
__global__ void __launch_bounds__(256) k_cg_step(const double *__restrict__ sc, const double *__restrict__ p,
                                                 const double *__restrict__ ap, int64_t n, double *y, double *r,
                                                 double *part)
{
    __shared__ double red[8];
    const double alpha = sc[2];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        y[i] = fma(alpha, p[i], y[i]);
        const double ri = fma(-alpha, ap[i], r[i]);
        r[i] = ri;
        s = fma(ri, ri, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// p = r + beta p with beta on the device
__global__ void k_cg_dir(const double *__restrict__ sc, const double *__restrict__ r, int64_t n, double *p)
{
    const double beta = sc[3];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], r[i]);
}

// x -= Q[:, 0:ncol] h
__global__ void k_update(const double *__restrict__ Q, int64_t ldq, int64_t n, int ncol, const double *__restrict__ h,
                         double *x)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < ncol; ++c) s = fma(Q[(int64_t)c * ldq + r], h[c], s);
        x[r] -= s;
    }
}

// y = a * x
__global__ void k_scale(const double *__restrict__ x, double a, int64_t n, double *y)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        y[r] = a * x[r];
}

// y += a * x
__global__ void k_axpy(double a, const double *__restrict__ x, int64_t n, double *y)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        y[r] = fma(a, x[r], y[r]);
}

// p = r + beta p
__global__ void k_xpby(const double *__restrict__ r, double beta, int64_t n, double *p)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], r[i]);
}

// SplitMix64 (Steele, Lea, Flood 2014) of a counter, mapped to (-1, 1)
__device__ __forceinline__ double splitmix_uniform(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z = z ^ (z >> 31);
    return ((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
}

__global__ void k_random(uint64_t seed, int64_t n, double *x)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        x[r] = splitmix_uniform(seed, (uint64_t)r);
}

// out[:, i] = Q[:, 0:ncv] S[:, i] for i < kk  (S is ncv x kk, column-major)
__global__ void k_combine(const double *__restrict__ Q, int64_t ldq, int64_t n, int ncv, const double *__restrict__ S,
                          int kk, double *out, int64_t ldo)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        for (int i0 = 0; i0 < kk; i0 += 8) {
            double acc[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = 0.0;
            for (int c = 0; c < ncv; ++c) {
                const double q = Q[(int64_t)c * ldq + r];
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (i0 + k < kk) acc[k] = fma(q, S[(int64_t)(i0 + k) * ncv + c], acc[k]);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (i0 + k < kk) out[(int64_t)(i0 + k) * ldo + r] = acc[k];
        }
    }
}

// ---- products of the basis with one vector: on the FP64 pipe (DW = false)
// or in double-word FP32 (DW = true, ~47 bits, dword.cuh)
template <bool DW>
struct BasisArith;
template <>
struct BasisArith<false> {
    using op_t = double;
    using acc_t = double;
    static __device__ __forceinline__ op_t op(double v) { return v; }
    static __device__ __forceinline__ acc_t zero() { return 0.0; }
    static __device__ __forceinline__ void mac(acc_t &a, op_t q, op_t x) { a = fma(q, x, a); }
    static __device__ __forceinline__ double value(acc_t a) { return a; }
};
template <>
struct BasisArith<true> {
    using op_t = float2;
    using acc_t = float2;
    static __device__ __forceinline__ op_t op(double v) { return dword::from_double(v); }
    static __device__ __forceinline__ acc_t zero() { return make_float2(0.0f, 0.0f); }
    static __device__ __forceinline__ void mac(acc_t &a, op_t q, op_t x) { dword::fma_acc(a, q, x); }
    static __device__ __forceinline__ double value(acc_t a) { return dword::to_double(a); }
};

// block sum of one double per thread into *out (all threads call it)
__device__ __forceinline__ void block_sum_to(double v, double *out)
{
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *out = t;
    }
}

// Row tiles of the basis products: a block walks tiles of kDotThreads *
// kTileRows consecutive rows (thread t owns rows r0 + t + kDotThreads k,
// k < kTileRows: coalesced) and, within a tile, streams the basis column by
// column, so that the memory sees long runs of one column (16 KB per tile)
// instead of short pieces of all columns at once; each thread keeps
// kTileRows loads in flight.
constexpr int kTileRows = 8;

// part[blk * nout + c] = sum over this block's rows of col_c(r) x_r, where
// col_c is Q[:, c] for c < ncol and x itself for c = ncol when self = 1
// (nout = ncol + self).  Row tiles as the update (below); the columns in
// chunks of kDotCols: for each chunk the block walks all its tiles, each
// thread accumulating its rows' products per column in registers, and
// reduces once at the end of the chunk (warp shuffles, then the warps in a
// fixed order).  x is read once per chunk (the block's rows stay in L2).
// When gate is non-null and *gate == 0 the pass was skipped by the device
// and every block returns at once.
constexpr int kDotCols = 4;
template <bool DW>
__global__ void __launch_bounds__(kDotThreads) k_basis_dots(const double *__restrict__ Q, int64_t ldq, int64_t n,
                                                            int ncol, int self, const double *__restrict__ x,
                                                            const int *__restrict__ gate, double *part)
{
    using A = BasisArith<DW>;
    if (gate && *gate == 0) return;
    __shared__ double red[kDotThreads / 32][kDotCols];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nout = ncol + self;
    constexpr int64_t tile = (int64_t)kDotThreads * kTileRows;
    for (int c0 = 0; c0 < nout; c0 += kDotCols) {
        typename A::acc_t acc[kDotCols];
#pragma unroll
        for (int k = 0; k < kDotCols; ++k) acc[k] = A::zero();
        for (int64_t r0 = (int64_t)blockIdx.x * tile; r0 < n; r0 += (int64_t)gridDim.x * tile) {
            double xv[kTileRows];
#pragma unroll
            for (int k = 0; k < kTileRows; ++k) {
                const int64_t r = r0 + threadIdx.x + (int64_t)kDotThreads * k;
                xv[k] = r < n ? x[r] : 0.0;
            }
            typename A::op_t xo[kTileRows];
#pragma unroll
            for (int k = 0; k < kTileRows; ++k) xo[k] = A::op(xv[k]);
#pragma unroll
            for (int j = 0; j < kDotCols; ++j) {
                const int c = c0 + j;
                if (c >= nout) break;
                double q[kTileRows];
#pragma unroll
                for (int k = 0; k < kTileRows; ++k) {
                    const int64_t r = r0 + threadIdx.x + (int64_t)kDotThreads * k;
                    q[k] = c < ncol ? (r < n ? Q[(int64_t)c * ldq + r] : 0.0) : xv[k];
                }
#pragma unroll
                for (int k = 0; k < kTileRows; ++k) A::mac(acc[j], A::op(q[k]), xo[k]);
            }
        }
#pragma unroll
        for (int j = 0; j < kDotCols; ++j) {
            double v = A::value(acc[j]);
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][j] = v;
        }
        __syncthreads();
        if (threadIdx.x < kDotCols && c0 + (int)threadIdx.x < nout) {
            double sacc = 0.0;
            for (int w = 0; w < kDotThreads / 32; ++w) sacc += red[w][threadIdx.x];
            part[(int64_t)blockIdx.x * nout + c0 + threadIdx.x] = sacc;
        }
        __syncthreads();
    }
}

// x -= Q[:, 0:ncol] h over row tiles (each thread's
// kTileRows rows accumulated in registers while the columns stream by), h
// staged once per block (dynamic shared memory of ncol operands); with
// norm_part, also the block's sum of the new x_r^2.  Gate as in k_basis_dots.
template <bool DW>
__global__ void __launch_bounds__(kDotThreads) k_basis_update(const double *__restrict__ Q, int64_t ldq, int64_t n,
                                                              int ncol, const double *__restrict__ h,
                                                              const int *__restrict__ gate, double *x,
                                                              double *norm_part)
{
    using A = BasisArith<DW>;
    if (gate && *gate == 0) return;
    extern __shared__ __align__(16) unsigned char basis_smem[];
    auto *hs = reinterpret_cast<typename A::op_t *>(basis_smem);
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) hs[c] = A::op(h[c]);
    __syncthreads();
    double s2 = 0.0;
    constexpr int64_t tile = (int64_t)kDotThreads * kTileRows;
    for (int64_t r0 = (int64_t)blockIdx.x * tile; r0 < n; r0 += (int64_t)gridDim.x * tile) {
        typename A::acc_t acc[kTileRows];
#pragma unroll
        for (int k = 0; k < kTileRows; ++k) acc[k] = A::zero();
        for (int c = 0; c < ncol; ++c) {
            double q[kTileRows];
#pragma unroll
            for (int k = 0; k < kTileRows; ++k) {
                const int64_t r = r0 + threadIdx.x + (int64_t)kDotThreads * k;
                q[k] = r < n ? Q[(int64_t)c * ldq + r] : 0.0;
            }
            const typename A::op_t hc = hs[c];
#pragma unroll
            for (int k = 0; k < kTileRows; ++k) A::mac(acc[k], A::op(q[k]), hc);
        }
#pragma unroll
        for (int k = 0; k < kTileRows; ++k) {
            const int64_t r = r0 + threadIdx.x + (int64_t)kDotThreads * k;
            if (r < n) {
                const double v = x[r] - A::value(acc[k]);
                x[r] = v;
                s2 = fma(v, v, s2);
            }
        }
    }
    if (norm_part) block_sum_to(s2, norm_part + blockIdx.x);
}

// the three-term part of a Lanczos step: x -= beta qprev (qprev may be
// null), then the block's sum of qj_r x_r (alpha's partial)
__global__ void __launch_bounds__(256) k_three_term(const double *__restrict__ qprev, double beta,
                                                   const double *__restrict__ qj, int64_t n, double *x, double *part)
{
    double s = 0.0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double v = x[r];
        if (qprev) {
            v = fma(-beta, qprev[r], v);
            x[r] = v;
        }
        s = fma(qj[r], v, s);
    }
    block_sum_to(s, part + blockIdx.x);
}

// x -= alpha qj with alpha on the device
__global__ void k_sub_scaled(const double *__restrict__ alpha, const double *__restrict__ qj, int64_t n, double *x)
{
    const double a = *alpha;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        x[r] = fma(-a, qj[r], x[r]);
}

// one warp: norm2 = total of the partials (fixed order); flag = 1 when the
// pass removed more than 1 - eta2 of the norm squared it started from
// (*before2), i.e. the second Gram-Schmidt pass is needed
__global__ void k_dgks(const double *__restrict__ part, int nblk, const double *__restrict__ before2, double eta2,
                       double *norm2, int *flag, double *flag_copy)
{
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) s += part[b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) {
        *norm2 = s;
        if (flag) {
            const int f = s < eta2 * *before2 ? 1 : 0;
            *flag = f;
            *flag_copy = (double)f;
        }
    }
}

// out[:, i] = Q[:, 0:ncv] S[:, i] for i < kk (S column-major ncv x kk), in
// double-word; each row's accumulators for 16 columns at a time in registers
__global__ void __launch_bounds__(256, 3) k_combine_dw(const double *__restrict__ Q, int64_t ldq, int64_t n, int ncv,
                                                   const double *__restrict__ S, int kk, double *out, int64_t ldo)
{
    // the first kCombineFp64 of every 16 outputs on the FP64 pipe (its own
    // rate, beside the FP32 pipe's double-word work), the rest double-word
    constexpr int KF = kCombineFp64;
    extern __shared__ float2 ss[];                 // [ncv][kk] double-word, then [ncv][kk] FP64
    double *sd = reinterpret_cast<double *>(ss + (size_t)ncv * kk);
    for (int e = threadIdx.x; e < ncv * kk; e += blockDim.x) {
        const int c = e / kk, i = e - c * kk;
        const double v = S[(int64_t)i * ncv + c];
        ss[e] = dword::from_double(v);
        sd[e] = v;
    }
    __syncthreads();
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        for (int i0 = 0; i0 < kk; i0 += 16) {
            float2 acc[16];
            double dacc[KF];
#pragma unroll
            for (int k = 0; k < 16; ++k) acc[k] = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int k = 0; k < KF; ++k) dacc[k] = 0.0;
            double qn = Q[r];                            // the next column's value, loaded a column ahead
            for (int c = 0; c < ncv; ++c) {
                const double qd = qn;
                if (c + 1 < ncv) qn = Q[(int64_t)(c + 1) * ldq + r];
                const float2 q = dword::from_double(qd);
                const float2 *srow = ss + (int64_t)c * kk + i0;
                const double *drow = sd + (int64_t)c * kk + i0;
#pragma unroll
                for (int k = 0; k < KF; ++k)
                    if (i0 + k < kk) dacc[k] = fma(qd, drow[k], dacc[k]);
#pragma unroll
                for (int k = KF; k < 16; ++k)
                    if (i0 + k < kk) dword::fma_acc(acc[k], q, srow[k]);
            }
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (i0 + k < kk) out[(int64_t)(i0 + k) * ldo + r] = k < KF ? dacc[k < KF ? k : 0] : dword::to_double(acc[k]);
        }
    }
}

// per-block (max |x|, signed value at the first maximum) of each column
__global__ void k_colmax(const double *__restrict__ V, int64_t ldv, int64_t n, int k, double *part)
{
    __shared__ double sa[256], sv[256];
    __shared__ long long si[256];
    for (int c = 0; c < k; ++c) {
        double ba = -1.0, bv = 0.0;
        long long bi = LLONG_MAX;
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
            const double v = V[(int64_t)c * ldv + r];
            const double a = fabs(v);
            if (a > ba) {
                ba = a;
                bv = v;
                bi = r;
            }
        }
        sa[threadIdx.x] = ba;
        sv[threadIdx.x] = bv;
        si[threadIdx.x] = bi;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) {
                const int o = threadIdx.x + s;
                if (sa[o] > sa[threadIdx.x] || (sa[o] == sa[threadIdx.x] && si[o] < si[threadIdx.x])) {
                    sa[threadIdx.x] = sa[o];
                    sv[threadIdx.x] = sv[o];
                    si[threadIdx.x] = si[o];
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            part[((int64_t)blockIdx.x * k + c) * 3 + 0] = sa[0];
            part[((int64_t)blockIdx.x * k + c) * 3 + 1] = sv[0];
            part[((int64_t)blockIdx.x * k + c) * 3 + 2] = (double)si[0];
        }
        __syncthreads();
    }
}

__global__ void k_scale_cols(double *V, int64_t ldv, int64_t n, int k, const double *__restrict__ f)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        for (int c = 0; c < k; ++c) V[(int64_t)c * ldv + r] *= f[c];
}

// at most one full wave of resident CTAs of `kernel` (blocks of `threads`
// threads with `smem` bytes of dynamic shared memory), and at most `want`
template <typename K>
static int one_wave(K kernel, int threads, size_t smem, int64_t want)
{
    int r = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, kernel, threads, smem) != cudaSuccess || r <= 0) {
        cudaGetLastError();
        r = 1;
    }
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm_count() * r));
}

static int vec_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, sm_count() * 8)); }

struct Workspace {
    cudaStream_t st = nullptr;
    int64_t n = 0;
    int nblk = 1;
    bool tensor = false;   // products of the basis on the tensor cores (ozaki.cu)
    bool dword = false;    // products of the basis in double-word FP32 (dword.cuh)
    // The single-vector products Q^T x and x - Q h stream the basis once for
    // one multiply-add per element: on the tensor cores they would spend most
    // of the instruction's width on padding, so only the Ritz vectors Q S
    // (many columns) take them there
    bool matvec_tc = false;
    DevBuf part, hdev, scal, lay0, npart, flag;
    long long second_passes = 0, steps = 0;

    ml_status init(int64_t n_, int maxcol, cudaStream_t s, int kind = 0)
    {
        n = n_;
        st = s;
        tensor = kind == 2;
        dword = kind == 1;
        nblk = (int)std::max<int64_t>(1, std::min<int64_t>((n + kDotThreads - 1) / kDotThreads, 456));
        const int nb_oz = oz_gram_blocks(1, n);
        ML_TRY(part.ensure((size_t)std::max(std::max(nblk, nb_oz), dw_blocks()) * (std::max(maxcol, 1) + 1) *
                           sizeof(double)));
        ML_TRY(hdev.ensure((size_t)(2 * maxcol + 8) * sizeof(double)));
        ML_TRY(npart.ensure((size_t)std::max(vec_blocks(n), dw_blocks()) * sizeof(double)));
        ML_TRY(flag.ensure(sizeof(int)));
        ML_TRY(scal.ensure(64 * sizeof(double)));
        ML_TRY(lay0.ensure(sizeof(int)));
        ML_CUDA(cudaMemsetAsync(lay0.p, 0, sizeof(int), st));
        return ML_OK;
    }
    // grids of the basis products: one full wave of resident CTAs (a partial
    // last wave leaves SMs idle); the update at most one CTA per row tile.
    // dw_blocks() and vec_blocks() bound these grids (the partial-sum buffers
    // are sized with them).
    int64_t row_tiles() const { return (n + (int64_t)kDotThreads * kTileRows - 1) / ((int64_t)kDotThreads * kTileRows); }
    int dw_blocks() const
    {
        return dword ? one_wave(k_basis_dots<true>, kDotThreads, 0, row_tiles())
                     : one_wave(k_basis_dots<false>, kDotThreads, 0, row_tiles());
    }
    static size_t update_smem(int ncol, bool dw) { return (size_t)ncol * (dw ? sizeof(float2) : sizeof(double)); }
    int update_blocks(int ncol) const
    {
        return dword ? one_wave(k_basis_update<true>, kDotThreads, update_smem(ncol, true), row_tiles())
                     : one_wave(k_basis_update<false>, kDotThreads, update_smem(ncol, false), row_tiles());
    }
    // out (device, ncol) = Q[:, 0:ncol]^T x for the orthonormal basis Q (column
    // major) and a vector with |x_i| < 2: on the tensor cores when enabled
    ml_status basis_dots(const double *Q, int64_t ldq, int ncol, const double *x, double *out)
    {
        if (dword) {
            const int nb = dw_blocks();
            {
                ProfScope pr("dots", st);
                k_basis_dots<true><<<nb, kDotThreads, 0, st>>>(Q, ldq, n, ncol, 0, x, nullptr, part.as<double>());
            }
            {
                ProfScope pr("dots_reduce", st);
                k_reduce_cols<<<1, 256, 0, st>>>(part.as<double>(), nb, ncol, out);
            }
            ML_CUDA(cudaGetLastError());
            return ML_OK;
        }
        if (!(tensor && matvec_tc && oz_gram_ok(ncol, 1))) return dots(Q, ldq, ncol, x, out);
        const int nb = oz_gram_blocks(1, n);
        {
            ProfScope pr("dots", st);
            ML_TRY(oz_gram(OzMat{Q, 0, 1, ldq}, ncol, OzMat{x, 0, 1, n}, 1, lay0.as<int>(), 1, n, nb,
                           part.as<double>(), st));
        }
        {
            ProfScope pr("dots_reduce", st);
            k_reduce_cols<<<1, 256, 0, st>>>(part.as<double>(), nb, ncol, out);
        }
        ML_CUDA(cudaGetLastError());
        return ML_OK;
    }
    // x -= Q[:, 0:ncol] h (h device)
    ml_status basis_update(const double *Q, int64_t ldq, int ncol, const double *h, double *x)
    {
        ProfScope pr("update", st);
        if (dword) {
            k_basis_update<true><<<update_blocks(ncol), kDotThreads, update_smem(ncol, true), st>>>(
                Q, ldq, n, ncol, h, nullptr, x, nullptr);
            ML_CUDA(cudaGetLastError());
            return ML_OK;
        }
        if (tensor && matvec_tc && oz_gemm_ok(ncol))
            return oz_gemm(OzMat{Q, 0, 1, ldq}, ncol, h, 1, 1, 0, 1, OzOut{x, 0, 1, n}, lay0.as<int>(), 1, n, true, st);
        k_update<<<vec_blocks(n), 256, 0, st>>>(Q, ldq, n, ncol, h, x);
        ML_CUDA(cudaGetLastError());
        return ML_OK;
    }
    // out (device, ncol) = Q[:, 0:ncol]^T x
    ml_status dots(const double *Q, int64_t ldq, int ncol, const double *x, double *out)
    {
        {
            ProfScope pr("dots", st);
            k_dots<<<nblk, kDotThreads, 0, st>>>(Q, ldq, n, ncol, x, part.as<double>());
        }
        {
            ProfScope pr("dots_reduce", st);
            k_reduce_cols<<<1, 256, 0, st>>>(part.as<double>(), nblk, ncol, out);
        }
        ML_CUDA(cudaGetLastError());
        return ML_OK;
    }
    ml_status dot_host(const double *a, const double *b, double *out)
    {
        ML_TRY(dots(a, n, 1, b, scal.as<double>()));
        ML_CUDA(cudaMemcpyAsync(out, scal.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        ML_CUDA(cudaStreamSynchronize(st));
        return ML_OK;
    }
    // x <- x - Q h twice (CGS2); hsum_host (ncol) receives h1 + h2, beta the norm of x after
    ml_status orthogonalize(const double *Q, int64_t ldq, int ncol, double *x, std::vector<double> &hsum,
                            double *beta)
    {
        double *h1 = hdev.as<double>(), *h2 = h1 + ncol, *nrm = h2 + ncol;
        if (ncol > 0) {
            ML_TRY(basis_dots(Q, ldq, ncol, x, h1));
            ML_TRY(basis_update(Q, ldq, ncol, h1, x));
            ML_TRY(basis_dots(Q, ldq, ncol, x, h2));
            ML_TRY(basis_update(Q, ldq, ncol, h2, x));
        }
        ML_TRY(dots(x, n, 1, x, nrm));
        std::vector<double> hh(2 * ncol + 1);
        ML_CUDA(cudaMemcpyAsync(hh.data(), h1, (2 * ncol + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
        ML_CUDA(cudaStreamSynchronize(st));
        hsum.assign(ncol, 0.0);
        for (int c = 0; c < ncol; ++c) hsum[c] = hh[c] + hh[ncol + c];
        *beta = std::sqrt(std::max(hh[2 * ncol], 0.0));
        return ML_OK;
    }
    // One Lanczos step for column j of the basis, x = Op q_j on entry (FP64
    // pipe or double-word products; the tensor-core kind uses orthogonalize).
    // The three-term part first: x -= beta_prev q_{j-1} (when use_prev),
    // alpha = q_j . x, x -= alpha q_j.  Then one classical Gram-Schmidt pass
    // against Q[:, 0:j+1], and a second pass only when the first removed more
    // than half of the norm squared it started from (the criterion of Daniel,
    // Gragg, Kaufman and Stewart 1976), decided on the device.  x is then
    // close to orthogonal to the basis before the pass, so the second pass is
    // rare; without the three-term part the pass would remove the large alpha
    // component and the criterion would ask for a second pass in nearly every
    // step.  hsum (j + 1) receives x's coefficients against the columns,
    // alpha and beta_prev included; beta the norm of x after.
    ml_status lanczos_step(const double *Q, int64_t ldq, int j, bool use_prev, double beta_prev, double *x,
                           std::vector<double> &hsum, double *beta)
    {
        const int ncol = j + 1;
        const double *qj = Q + (int64_t)j * ldq;
        double *h1 = hdev.as<double>();      // ncol coefficients + |x|^2 before the pass
        double *h2 = h1 + ncol + 1;          // second pass
        double *sc = h2 + ncol;              // alpha, |x|^2 after pass 1, after pass 2, flag
        const int nbv = vec_blocks(n), nbd = dw_blocks(), nbu = update_blocks(ncol);
        int *fl = flag.as<int>();
        {
            ProfScope pr("vector", st);
            k_three_term<<<nbv, 256, 0, st>>>(use_prev ? qj - ldq : nullptr, beta_prev, qj, n, x, npart.as<double>());
            k_reduce_cols<<<1, 32, 0, st>>>(npart.as<double>(), nbv, 1, sc);
            k_sub_scaled<<<nbv, 256, 0, st>>>(sc, qj, n, x);
        }
        const size_t hsm = update_smem(ncol, dword);
        for (int pass = 0; pass < 2; ++pass) {
            double *h = pass == 0 ? h1 : h2;
            const int *gate = pass == 0 ? nullptr : fl;
            const int self = pass == 0 ? 1 : 0;
            // the second pass's kernels are timed under their own names (a skipped
            // pass costs one early-returning launch each)
            {
                ProfScope pr(pass == 0 ? "dots" : "dots2", st);
                if (dword)
                    k_basis_dots<true><<<nbd, kDotThreads, 0, st>>>(Q, ldq, n, ncol, self, x, gate, part.as<double>());
                else
                    k_basis_dots<false><<<nbd, kDotThreads, 0, st>>>(Q, ldq, n, ncol, self, x, gate, part.as<double>());
            }
            {
                ProfScope pr("dots_reduce", st);
                k_reduce_cols<<<1, 256, 0, st>>>(part.as<double>(), nbd, ncol + self, h);
            }
            {
                ProfScope pr(pass == 0 ? "update" : "update2", st);
                if (dword)
                    k_basis_update<true><<<nbu, kDotThreads, hsm, st>>>(Q, ldq, n, ncol, h, gate, x, npart.as<double>());
                else
                    k_basis_update<false><<<nbu, kDotThreads, hsm, st>>>(Q, ldq, n, ncol, h, gate, x, npart.as<double>());
                k_dgks<<<1, 32, 0, st>>>(npart.as<double>(), nbu, h1 + ncol, 0.5, sc + 1 + pass,
                                         pass == 0 ? fl : nullptr, sc + 3);
            }
        }
        ML_CUDA(cudaGetLastError());
        const int nread = 2 * ncol + 1 + 4;
        std::vector<double> hh(nread);
        ML_CUDA(cudaMemcpyAsync(hh.data(), h1, nread * sizeof(double), cudaMemcpyDeviceToHost, st));
        ML_CUDA(cudaStreamSynchronize(st));
        const double *r1 = hh.data(), *r2 = r1 + ncol + 1, *rs = r2 + ncol;
        const bool second = rs[3] != 0.0;
        hsum.assign(ncol, 0.0);
        for (int c = 0; c < ncol; ++c) hsum[c] = r1[c] + (second ? r2[c] : 0.0);
        hsum[j] += rs[0];
        if (use_prev) hsum[j - 1] += beta_prev;
        *beta = std::sqrt(std::max(second ? rs[2] : rs[1], 0.0));
        ++steps;
        second_passes += second ? 1 : 0;
        return ML_OK;
    }
};

// y = (1/T) sum_t (L_sym^(t) + delta I)^{-1} x by CG per layer.  The T
// solves are independent: each runs on its own non-blocking stream with its
// own vectors and scalars, so the layers' small kernels (transforms, folds,
// CG scalars) overlap with the other layers' spreading and interpolation.
// The streams fork from and join the caller's stream through events; the
// layer results are summed on the caller's stream in layer order.
struct InverseOp {
    ml_plan_s *const *layers;
    int T;
    double delta;
    int64_t n;
    Workspace *ws;
    int inner_max = 200;
    double inner_tol = 1e-12;
    long long inner_iters = 0;
    struct Lane {
        DevBuf r, p, ap, y, part, sc;
        cudaStream_t s = nullptr;
        cudaEvent_t ev[2] = {nullptr, nullptr};   // residual of iterations i, i+1 (lagged host check)
        cudaEvent_t join = nullptr;
        // one CG iteration captured as a CUDA graph (its pointers never change
        // during the solve) and replayed while kernel timing is off, since
        // per-kernel events cannot be recorded inside a graph
        cudaGraphExec_t graph = nullptr;
    };
    std::vector<Lane> lanes;
    cudaEvent_t fork = nullptr;
    double *hrr = nullptr;   // pinned: T x 2 residuals
    bool graphs_ok = true;

    bool own_streams = true;   // false: one stream for all layers (a plan passed twice shares its
                               // workspace; kernel timing wants kernels alone)

    ml_status init()
    {
        lanes.resize(T);
        const int pb = ws->nblk;
        for (int a = 0; a < T; ++a)
            for (int b = a + 1; b < T; ++b)
                if (layers[a] == layers[b]) own_streams = false;
        // while kernels are timed, one stream: each event pair then brackets one kernel alone
        if (profiling()) own_streams = false;
        for (int t = 0; t < T; ++t) {
            Lane &L = lanes[t];
            ML_TRY(L.r.ensure(n * 8));
            ML_TRY(L.p.ensure(n * 8));
            ML_TRY(L.ap.ensure(n * 8));
            ML_TRY(L.y.ensure(n * 8));
            ML_TRY(L.part.ensure((size_t)pb * 8));
            ML_TRY(L.sc.ensure(8 * 8));
            if (own_streams || t == 0) ML_CUDA(cudaStreamCreateWithFlags(&L.s, cudaStreamNonBlocking));
            else L.s = lanes[0].s;
            for (auto &e : L.ev) ML_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            ML_CUDA(cudaEventCreateWithFlags(&L.join, cudaEventDisableTiming));
        }
        ML_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        ML_CUDA(cudaMallocHost(&hrr, (size_t)2 * T * sizeof(double)));
        return ML_OK;
    }
    ~InverseOp()
    {
        // finish all work first (lanes may share one stream), then release
        for (int t = 0; t < (int)lanes.size(); ++t)
            if (lanes[t].s && (own_streams || t == 0)) cudaStreamSynchronize(lanes[t].s);
        for (int t = 0; t < (int)lanes.size(); ++t) {
            Lane &L = lanes[t];
            if (L.graph) cudaGraphExecDestroy(L.graph);
            for (auto &e : L.ev)
                if (e) cudaEventDestroy(e);
            if (L.join) cudaEventDestroy(L.join);
            if (L.s && (own_streams || t == 0)) cudaStreamDestroy(L.s);
        }
        if (fork) cudaEventDestroy(fork);
        if (hrr) cudaFreeHost(hrr);
        cudaGetLastError();   // nothing from the clean-up may leak into the caller's next check
    }
    // ap = (L_sym + delta I) v = (1 + delta) v - A v
    ml_status shifted(ml_plan_s *L, const double *v, double *out, cudaStream_t st)
    {
        ApplyVec av{v, 1, out, 1, 1};
        ApplyOpts o;
        o.normalized = true;
        o.alpha = -1.0;
        o.shift = 1.0 + delta;
        return apply_layer(L, av, o, st);
    }
    // one CG iteration of layer t on its stream: Ap, alpha, x/r update, beta, new direction
    ml_status iteration(int t)
    {
        Lane &L = lanes[t];
        const int nb = vec_blocks(n), pb = ws->nblk;
        double *part = L.part.as<double>(), *sc = L.sc.as<double>();
        ML_TRY(shifted(layers[t], L.p.as<double>(), L.ap.as<double>(), L.s));
        {
            ProfScope pr("cg", L.s);
            k_dot_part<<<pb, 256, 0, L.s>>>(L.p.as<double>(), L.ap.as<double>(), n, part);
            k_cg_scalars<<<1, 32, 0, L.s>>>(part, pb, 0, sc);
            k_cg_step<<<pb, 256, 0, L.s>>>(sc, L.p.as<double>(), L.ap.as<double>(), n, L.y.as<double>(),
                                           L.r.as<double>(), part);
            k_cg_scalars<<<1, 32, 0, L.s>>>(part, pb, 1, sc);
            k_cg_dir<<<nb, 256, 0, L.s>>>(sc, L.r.as<double>(), n, L.p.as<double>());
        }
        ML_CUDA(cudaGetLastError());
        return ML_OK;
    }
    // run iteration it of layer t: eagerly, or through its graph (captured at it = 1)
    ml_status step(int t, int it)
    {
        Lane &L = lanes[t];
        const bool use_graph = graphs_ok && !profiling() && it >= 1;
        if (use_graph && !L.graph) {
            // the first iteration ran eagerly (workspace, attributes): capture the second
            cudaGraph_t g = nullptr;
            const int64_t applied0 = layers[t]->applied;   // capturing runs no work
            cudaError_t e = cudaStreamBeginCapture(L.s, cudaStreamCaptureModeThreadLocal);
            ml_status cs = ML_OK;
            if (e == cudaSuccess) {
                cs = iteration(t);
                e = cudaStreamEndCapture(L.s, &g);
            }
            if (e == cudaSuccess && cs == ML_OK && g) e = cudaGraphInstantiate(&L.graph, g, 0);
            if (g) cudaGraphDestroy(g);
            layers[t]->applied = applied0;
            if (e != cudaSuccess || cs != ML_OK || !L.graph) {
                cudaGetLastError();   // capture not possible here: run eagerly from now on
                graphs_ok = false;
                L.graph = nullptr;
            }
        }
        if (graphs_ok && !profiling() && L.graph) {
            ML_CUDA(cudaGraphLaunch(L.graph, L.s));
            layers[t]->applied += 1;   // the replayed product's work counter
            count_graph_replay();
        } else {
            ML_TRY(iteration(t));
        }
        ++inner_iters;
        return ML_OK;
    }
    ml_status apply(const double *x, double *out, cudaStream_t st)
    {
        const int nb = vec_blocks(n), pb = ws->nblk;
        // ||x||^2 for the relative stopping test (x is ready on st)
        double bb;
        ML_TRY(ws->dot_host(x, x, &bb));
        const double stop2 = inner_tol * inner_tol * bb;
        ML_CUDA(cudaEventRecord(fork, st));
        std::vector<char> done(T, !(bb > 0) ? 1 : 0);
        for (int t = 0; t < T; ++t) {
            Lane &L = lanes[t];
            ML_CUDA(cudaStreamWaitEvent(L.s, fork, 0));
            // x0 = 0: r = x, p = x, r.r = ||x||^2
            ML_CUDA(cudaMemcpyAsync(L.r.p, x, n * 8, cudaMemcpyDeviceToDevice, L.s));
            ML_CUDA(cudaMemcpyAsync(L.p.p, x, n * 8, cudaMemcpyDeviceToDevice, L.s));
            ML_CUDA(cudaMemsetAsync(L.y.p, 0, n * 8, L.s));
            {
                ProfScope pr("cg", L.s);
                k_dot_part<<<pb, 256, 0, L.s>>>(x, x, n, L.part.as<double>());
                k_cg_scalars<<<1, 32, 0, L.s>>>(L.part.as<double>(), pb, 2, L.sc.as<double>());
            }
            ML_CUDA(cudaGetLastError());
        }
        // all layers advance together; the residual of iteration it is read
        // while iteration it+1 runs (one iteration of lag, no pipeline bubble)
        for (int it = 0; it < inner_max; ++it) {
            bool any = false;
            for (int t = 0; t < T; ++t) {
                if (done[t]) continue;
                any = true;
                Lane &L = lanes[t];
                ML_TRY(step(t, it));
                ML_CUDA(cudaMemcpyAsync(hrr + 2 * t + (it & 1), L.sc.p, sizeof(double), cudaMemcpyDeviceToHost, L.s));
                ML_CUDA(cudaEventRecord(L.ev[it & 1], L.s));
            }
            if (!any) break;
            if (it >= 1)
                for (int t = 0; t < T; ++t) {
                    if (done[t]) continue;
                    ML_CUDA(cudaEventSynchronize(lanes[t].ev[(it - 1) & 1]));
                    done[t] = hrr[2 * t + ((it - 1) & 1)] <= stop2;
                }
        }
        for (int t = 0; t < T; ++t) {
            Lane &L = lanes[t];
            ML_CUDA(cudaStreamSynchronize(L.s));
            if (!done[t]) {
                double hs[2];
                ML_CUDA(cudaMemcpy(hs, L.sc.p, 2 * sizeof(double), cudaMemcpyDeviceToHost));
                if (hs[0] > stop2)
                    return fail(ML_ERR_BREAKDOWN, !(hs[1] > 0) ? "CG: operator not positive definite (p^T A p <= 0)"
                                                               : "CG: inner solve did not converge");
            }
            ML_CUDA(cudaEventRecord(L.join, L.s));
            ML_CUDA(cudaStreamWaitEvent(st, L.join, 0));
        }
        // out = (1/T) sum_t y_t in layer order, on the caller's stream
        ML_CUDA(cudaMemsetAsync(out, 0, n * 8, st));
        for (int t = 0; t < T; ++t) {
            ProfScope pr("vector", st);
            k_axpy<<<nb, 256, 0, st>>>(1.0 / T, lanes[t].y.as<double>(), n, out);
        }
        ML_CUDA(cudaGetLastError());
        return ML_OK;
    }
};

// f(T) e1 for the symmetric tridiagonal T (diagonal a[0..m-1], off-diagonal
// b[0..m-2]) and f(x) = x^p, p < 0.  Integer p: |p| solves with T (Thomas
// elimination; T is positive definite here, eigenvalues in [delta, 2+delta]);
// otherwise through the eigendecomposition of T.
static void tridiag_power_e1(const std::vector<double> &a, const std::vector<double> &b, int m, double p,
                             std::vector<double> &c)
{
    c.assign(m, 0.0);
    const double pr = std::round(p);
    if (std::fabs(p - pr) < 1e-12 && pr < 0) {
        std::vector<double> x(m, 0.0), cp(m), dp(m);
        x[0] = 1.0;
        for (int rep = 0; rep < (int)(-pr); ++rep) {
            // solve T y = x in place (no pivoting: T is symmetric positive definite)
            double den = a[0];
            cp[0] = (m > 1 ? b[0] : 0.0) / den;
            dp[0] = x[0] / den;
            for (int i = 1; i < m; ++i) {
                den = a[i] - b[i - 1] * cp[i - 1];
                cp[i] = (i + 1 < m ? b[i] : 0.0) / den;
                dp[i] = (x[i] - b[i - 1] * dp[i - 1]) / den;
            }
            x[m - 1] = dp[m - 1];
            for (int i = m - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
        }
        c = x;
        return;
    }
    std::vector<double> A((size_t)m * m, 0.0), ev, V;
    for (int i = 0; i < m; ++i) {
        A[(size_t)i * m + i] = a[i];
        if (i + 1 < m) A[(size_t)i * m + i + 1] = A[(size_t)(i + 1) * m + i] = b[i];
    }
    sym_eig(m, A, ev, V);
    for (int j = 0; j < m; ++j) {
        const double w = std::pow(std::max(ev[j], 1e-300), p) * V[(size_t)0 * m + j];
        for (int i = 0; i < m; ++i) c[i] += V[(size_t)i * m + j] * w;
    }
}

// Device-scalar helpers of the Lanczos approximation of a matrix power:
// *out = sum of the partials (or its square root), y += sign * (*a) * x,
// y = x / (*b) (zero when *b is zero).
__global__ void k_sum_to(const double *__restrict__ part, int nblk, int take_sqrt, double *out)
{
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) s += part[b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = take_sqrt ? sqrt(fmax(s, 0.0)) : s;
}

__global__ void k_axpy_dev(const double *__restrict__ a, double sign, const double *__restrict__ x, int64_t n,
                           double *y)
{
    const double f = sign * (*a);
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        y[r] = fma(f, x[r], y[r]);
}

__global__ void k_div_dev(const double *__restrict__ b, const double *__restrict__ x, int64_t n, double *y)
{
    const double bb = *b;
    const double f = bb != 0.0 ? 1.0 / bb : 0.0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        y[r] = f * x[r];
}

// y = (1/T) sum_t (L_sym^(t) + delta I)^p x for p < 0, p != -1: each term by
// the Lanczos approximation of the matrix function (Lanczos-FA): m steps of
// the three-term recurrence on B_t = L_sym^(t) + delta I from q_1 = x/||x||,
// then f(B_t) x ~ ||x|| Q_m f(T_m) e1, stopped when the coefficient vector
// changes by less than the tolerance (relative).  The polynomial Krylov
// approach of Sec. 3 for a general power.  The recurrence scalars stay on
// the device (alpha_j, beta_j are read on the host one step late, for the
// convergence test only) and every layer runs on its own non-blocking
// stream, as the conjugate-gradient solves do.
struct PowerOp {
    ml_plan_s *const *layers;
    int T;
    double p, delta;
    int64_t n;
    Workspace *ws;
    int mmax = 80;
    double tol = 1e-12;
    long long inner_iters = 0;
    struct Lane {
        DevBuf Q, w, part, ab, cd;   // basis n x (mmax+1), product, partial sums, alpha|beta, coefficients
        cudaStream_t s = nullptr;
        cudaEvent_t ev[2] = {nullptr, nullptr};
        cudaEvent_t join = nullptr;
        std::vector<double> a, b, c, cprev;
        bool done = false;
        int m = 0;
    };
    std::vector<Lane> lanes;
    cudaEvent_t fork = nullptr;
    double *hab = nullptr;   // pinned: T x 2 x 2 (alpha, beta of the last two steps)
    bool own_streams = true;

    ml_status init()
    {
        lanes.resize(T);
        for (int a = 0; a < T; ++a)
            for (int b = a + 1; b < T; ++b)
                if (layers[a] == layers[b]) own_streams = false;
        if (profiling()) own_streams = false;
        const int pb = ws->nblk;
        for (int t = 0; t < T; ++t) {
            Lane &L = lanes[t];
            ML_TRY(L.Q.ensure((size_t)n * (mmax + 1) * 8));
            ML_TRY(L.w.ensure((size_t)n * 8));
            ML_TRY(L.part.ensure((size_t)pb * 8));
            ML_TRY(L.ab.ensure((size_t)2 * mmax * 8));
            ML_TRY(L.cd.ensure((size_t)mmax * 8));
            if (own_streams || t == 0) ML_CUDA(cudaStreamCreateWithFlags(&L.s, cudaStreamNonBlocking));
            else L.s = lanes[0].s;
            for (auto &e : L.ev) ML_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            ML_CUDA(cudaEventCreateWithFlags(&L.join, cudaEventDisableTiming));
        }
        ML_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        ML_CUDA(cudaMallocHost(&hab, (size_t)4 * T * sizeof(double)));
        return ML_OK;
    }
    ~PowerOp()
    {
        for (int t = 0; t < (int)lanes.size(); ++t)
            if (lanes[t].s && (own_streams || t == 0)) cudaStreamSynchronize(lanes[t].s);
        for (int t = 0; t < (int)lanes.size(); ++t) {
            Lane &L = lanes[t];
            for (auto &e : L.ev)
                if (e) cudaEventDestroy(e);
            if (L.join) cudaEventDestroy(L.join);
            if (L.s && (own_streams || t == 0)) cudaStreamDestroy(L.s);
        }
        if (fork) cudaEventDestroy(fork);
        if (hab) cudaFreeHost(hab);
        cudaGetLastError();
    }
    // step j of layer t on its stream: w = B q_j - beta_{j-1} q_{j-1}, alpha_j,
    // w -= alpha_j q_j, beta_j = ||w||, q_{j+1} = w / beta_j
    ml_status step(int t, int j)
    {
        Lane &L = lanes[t];
        const int nb = vec_blocks(n), pb = ws->nblk;
        double *Q = L.Q.as<double>(), *wp = L.w.as<double>(), *ab = L.ab.as<double>(), *part = L.part.as<double>();
        double *qj = Q + (int64_t)j * n;
        ApplyVec av{qj, 1, wp, 1, 1};
        ApplyOpts o;
        o.normalized = true;
        o.alpha = -1.0;
        o.shift = 1.0 + delta;
        ML_TRY(apply_layer(layers[t], av, o, L.s));
        ++inner_iters;
        {
            ProfScope pr("vector", L.s);
            if (j > 0) k_axpy_dev<<<nb, 256, 0, L.s>>>(ab + mmax + j - 1, -1.0, Q + (int64_t)(j - 1) * n, n, wp);
            k_dot_part<<<pb, 256, 0, L.s>>>(qj, wp, n, part);
            k_sum_to<<<1, 32, 0, L.s>>>(part, pb, 0, ab + j);
            k_axpy_dev<<<nb, 256, 0, L.s>>>(ab + j, -1.0, qj, n, wp);
            k_dot_part<<<pb, 256, 0, L.s>>>(wp, wp, n, part);
            k_sum_to<<<1, 32, 0, L.s>>>(part, pb, 1, ab + mmax + j);
            k_div_dev<<<nb, 256, 0, L.s>>>(ab + mmax + j, wp, n, Q + (int64_t)(j + 1) * n);
        }
        ML_CUDA(cudaGetLastError());
        ML_CUDA(cudaMemcpyAsync(hab + 4 * t + 2 * (j & 1), ab + j, sizeof(double), cudaMemcpyDeviceToHost, L.s));
        ML_CUDA(cudaMemcpyAsync(hab + 4 * t + 2 * (j & 1) + 1, ab + mmax + j, sizeof(double), cudaMemcpyDeviceToHost,
                                L.s));
        ML_CUDA(cudaEventRecord(L.ev[j & 1], L.s));
        return ML_OK;
    }
    // host side of step j (after its event): record alpha_j, beta_j, update f(T) e1, test
    ml_status check(int t, int j)
    {
        Lane &L = lanes[t];
        ML_CUDA(cudaEventSynchronize(L.ev[j & 1]));
        const double alpha = hab[4 * t + 2 * (j & 1)], beta = hab[4 * t + 2 * (j & 1) + 1];
        L.a.push_back(alpha);
        L.m = j + 1;
        tridiag_power_e1(L.a, L.b, L.m, p, L.c);
        double dn = 0.0, cn = 0.0;
        for (int i = 0; i < L.m; ++i) {
            const double prev = i < (int)L.cprev.size() ? L.cprev[i] : 0.0;
            dn += (L.c[i] - prev) * (L.c[i] - prev);
            cn += L.c[i] * L.c[i];
        }
        if (j > 0 && std::sqrt(dn) <= tol * std::sqrt(cn)) L.done = true;
        if (beta <= 1e-14 * std::fabs(alpha)) L.done = true;   // invariant subspace: exact
        L.cprev = L.c;
        if (!L.done) L.b.push_back(beta);
        return ML_OK;
    }
    ml_status apply(const double *x, double *out, cudaStream_t st)
    {
        const int nb = vec_blocks(n);
        double xx;
        ML_TRY(ws->dot_host(x, x, &xx));
        const double nrm = std::sqrt(xx);
        ML_CUDA(cudaMemsetAsync(out, 0, n * 8, st));
        if (!(nrm > 0)) return ML_OK;
        ML_CUDA(cudaEventRecord(fork, st));
        for (int t = 0; t < T; ++t) {
            Lane &L = lanes[t];
            L.a.clear();
            L.b.clear();
            L.c.clear();
            L.cprev.clear();
            L.done = false;
            L.m = 0;
            ML_CUDA(cudaStreamWaitEvent(L.s, fork, 0));
            ProfScope pr("vector", L.s);
            k_scale<<<nb, 256, 0, L.s>>>(x, 1.0 / nrm, n, L.Q.as<double>());
        }
        ML_CUDA(cudaGetLastError());
        // all layers advance together; step j's scalars are read while step j+1 runs
        for (int j = 0; j < mmax; ++j) {
            bool any = false;
            for (int t = 0; t < T; ++t)
                if (!lanes[t].done) {
                    any = true;
                    ML_TRY(step(t, j));
                }
            if (!any) break;
            if (j >= 1)
                for (int t = 0; t < T; ++t)
                    if (!lanes[t].done) ML_TRY(check(t, j - 1));
        }
        for (int t = 0; t < T; ++t) {
            Lane &L = lanes[t];
            if (!L.done && L.m < mmax) ML_TRY(check(t, mmax - 1));
            if (!L.done) return fail(ML_ERR_BREAKDOWN, "Lanczos-FA: the matrix power did not converge");
            // y_t = (nrm / T) Q_m c, then joined into out on the caller's stream
            std::vector<double> cs(L.c);
            for (double &v : cs) v *= nrm / T;
            ML_CUDA(cudaMemcpyAsync(L.cd.p, cs.data(), L.m * 8, cudaMemcpyHostToDevice, L.s));
            {
                ProfScope pr("ritz", L.s);
                k_combine<<<nb, 256, 0, L.s>>>(L.Q.as<double>(), n, n, L.m, L.cd.as<double>(), 1, L.w.as<double>(), n);
            }
            ML_CUDA(cudaGetLastError());
            ML_CUDA(cudaEventRecord(L.join, L.s));
            ML_CUDA(cudaStreamWaitEvent(st, L.join, 0));
            ML_CUDA(cudaStreamSynchronize(L.s));   // cs (host) is released at the end of this iteration
        }
        for (int t = 0; t < T; ++t) {
            ProfScope pr("vector", st);
            k_axpy<<<nb, 256, 0, st>>>(1.0, lanes[t].w.as<double>(), n, out);
        }
        ML_CUDA(cudaGetLastError());
        return ML_OK;
    }
};

// Fix the sign of each column of V (n x k, column-major) so that its
// largest-magnitude entry (the first one on ties) is positive.
ml_status sign_fix_cols(double *V, int64_t n, int k, cudaStream_t st)
{
    const int cb = std::min(vec_blocks(n), 256);
    DevBuf part, fd;
    ML_TRY(part.ensure((size_t)cb * k * 3 * 8));
    ML_TRY(fd.ensure((size_t)k * 8));
    {
        ProfScope pr_("vector", st);
        k_colmax<<<cb, 256, 0, st>>>(V, n, n, k, part.as<double>());
    }
    std::vector<double> hp((size_t)cb * k * 3);
    ML_CUDA(cudaMemcpyAsync(hp.data(), part.p, hp.size() * 8, cudaMemcpyDeviceToHost, st));
    ML_CUDA(cudaStreamSynchronize(st));
    std::vector<double> f(k, 1.0);
    for (int c = 0; c < k; ++c) {
        double ba = -1, bv = 0, bi = 1e300;
        for (int b = 0; b < cb; ++b) {
            const double *e = &hp[((size_t)b * k + c) * 3];
            if (e[0] > ba || (e[0] == ba && e[2] < bi)) {
                ba = e[0];
                bv = e[1];
                bi = e[2];
            }
        }
        f[c] = bv < 0 ? -1.0 : 1.0;
    }
    ML_CUDA(cudaMemcpyAsync(fd.p, f.data(), k * 8, cudaMemcpyHostToDevice, st));
    {
        ProfScope pr_("vector", st);
        k_scale_cols<<<vec_blocks(n), 256, 0, st>>>(V, n, n, k, fd.as<double>());
    }
    ML_CUDA(cudaGetLastError());
    ML_CUDA(cudaStreamSynchronize(st));
    return ML_OK;
}

// returned by lanczos_impl when a tensor-core product met an operand beyond its
// fixed scale: the solve is repeated with the FP64-pipe products
constexpr int kRetryFp64 = 1000;

static ml_status lanczos_impl(ml_plan_s *const *layers, int T, int k, double pw, double tol, int maxit,
                              uint64_t seed, double *evals, double *evecs_dev, int *nconv_out, cudaStream_t st,
                              bool tensor)
{
    const int64_t n = layers[0]->n;
    const int ncv = (int)std::min<int64_t>(std::max(2 * k + 1, 20), n - 1);
    const int kkeep = std::min(ncv - 2, std::max(k + 1, (ncv + k) / 2));
    Workspace ws;
    const int kind = tensor ? 2 : (dense_products_kind() == 1 ? 1 : 0);
    ML_TRY(ws.init(n, ncv + 1, st, kind));
    if (tensor) ML_TRY(oz_reset_error(st));
    DevBuf Qb, Qtmp, wv, Sd;
    ML_TRY(Qb.ensure((size_t)n * (ncv + 1) * 8));
    ML_TRY(Qtmp.ensure((size_t)n * (ncv + 1) * 8));
    ML_TRY(wv.ensure((size_t)n * 8));
    ML_TRY(Sd.ensure((size_t)ncv * ncv * 8));
    double *Q = Qb.as<double>(), *w = wv.as<double>();
    const double delta = pw < 0 ? std::log1p(std::fabs(pw)) : 0.0;
    InverseOp inv{layers, T, delta, n, &ws};
    PowerOp pow_op{layers, T, pw, delta, n, &ws};
    pow_op.tol = std::max(1e-12, 1e-2 * tol);
    const bool use_cg = pw == -1.0;
    // inner solves two orders below the outer residual tolerance (the outer
    // operator is then exact to well within what the Ritz test resolves)
    inv.inner_tol = std::max(1e-12, 1e-2 * tol);
    if (pw < 0 && use_cg) ML_TRY(inv.init());
    if (pw < 0 && !use_cg) ML_TRY(pow_op.init());
    auto op = [&](const double *x, double *y) -> ml_status {
        if (pw > 0) return apply_device(layers, T, x, 1, y, ML_NORMALIZED_A, st);
        if (use_cg) return inv.apply(x, y, st);
        return pow_op.apply(x, y, st);
    };
    const int nb = vec_blocks(n);
    // start vector
    { ProfScope pr_("vector", st);
    k_random<<<nb, 256, 0, st>>>(seed, n, Q);
    }
    std::vector<double> h;
    double beta = 0;
    ML_TRY(ws.orthogonalize(Q, n, 0, Q, h, &beta));
    if (!(beta > 0)) return fail(ML_ERR_BREAKDOWN, "zero start vector");
    { ProfScope pr_("vector", st);
    k_scale<<<nb, 256, 0, st>>>(Q, 1.0 / beta, n, Q);
    }

    std::vector<double> Tm((size_t)ncv * ncv, 0.0);
    std::vector<double> theta, S;
    int kk = 0;         // kept Ritz vectors at the front of Q
    int matvecs = 0;
    int nconv = 0;
    double beta_last = 0.0;
    uint64_t restart_seed = seed ^ 0xA5A5A5A5DEADBEEFULL;
    while (true) {
        for (int j = kk; j < ncv; ++j) {
            ML_TRY(op(Q + (int64_t)j * n, w));
            ++matvecs;
            if (ws.tensor)
                ML_TRY(ws.orthogonalize(Q, n, j + 1, w, h, &beta));
            else
                ML_TRY(ws.lanczos_step(Q, n, j, j > kk, beta, w, h, &beta));
            for (int i = 0; i <= j; ++i) {
                if (i < kk && j >= kk && j != kk) continue;  // keep the arrow structure exact
                Tm[(size_t)i * ncv + j] = h[i];
                Tm[(size_t)j * ncv + i] = h[i];
            }
            double tnorm = 0.0;
            for (int i = 0; i <= j; ++i) tnorm = std::max(tnorm, std::fabs(Tm[(size_t)i * ncv + i]));
            if (beta <= 1e-14 * std::max(tnorm, 1e-300) * std::sqrt((double)n)) {
                // invariant subspace found: continue with a fresh random direction
                { ProfScope pr_("vector", st);
                k_random<<<nb, 256, 0, st>>>(restart_seed++, n, w);
                }
                std::vector<double> hh;
                double b2;
                ML_TRY(ws.orthogonalize(Q, n, j + 1, w, hh, &b2));
                if (!(b2 > 0)) return fail(ML_ERR_BREAKDOWN, "Lanczos breakdown: no new direction");
                beta = 0.0;
                { ProfScope pr_("vector", st);
                k_scale<<<nb, 256, 0, st>>>(w, 1.0 / b2, n, Q + (int64_t)(j + 1) * n);
                }
            } else {
                { ProfScope pr_("vector", st);
                k_scale<<<nb, 256, 0, st>>>(w, 1.0 / beta, n, Q + (int64_t)(j + 1) * n);
                }
            }
            ML_CUDA(cudaGetLastError());
            beta_last = beta;
        }
        // Rayleigh-Ritz on the projected matrix
        std::vector<double> a = Tm;
        sym_eig(ncv, a, theta, S);
        double tmax = 0.0;
        for (double t : theta) tmax = std::max(tmax, std::fabs(t));
        nconv = 0;
        for (int i = ncv - 1; i >= ncv - k; --i) {
            const double res = std::fabs(beta_last * S[(size_t)(ncv - 1) * ncv + i]);
            if (res <= tol * std::max(tmax, 1e-300)) ++nconv;
            else break;
        }
        const bool done = nconv >= k || matvecs >= maxit;
        const int keep = done ? k : kkeep;
        // Ritz vectors of the largest `keep` values -> front of Qtmp
        std::vector<double> Sk((size_t)ncv * keep);
        for (int i = 0; i < keep; ++i) {
            const int col = ncv - 1 - i;  // descending theta
            for (int c = 0; c < ncv; ++c) Sk[(size_t)i * ncv + c] = S[(size_t)c * ncv + col];
        }
        ML_CUDA(cudaMemcpyAsync(Sd.p, Sk.data(), Sk.size() * 8, cudaMemcpyHostToDevice, st));
        {
            ProfScope pr("ritz", st);
            if (ws.dword && (size_t)ncv * keep * (sizeof(float2) + sizeof(double)) <= 48 * 1024) {
                const size_t sm = (size_t)ncv * keep * (sizeof(float2) + sizeof(double));
                k_combine_dw<<<one_wave(k_combine_dw, 256, sm, nb), 256, sm, st>>>(Q, n, n, ncv, Sd.as<double>(), keep,
                                                                                 Qtmp.as<double>(), n);
            } else if (ws.tensor && oz_gemm_ok(ncv)) {
                // Sk is ncv x keep column-major: M[r, j] = Sk[j * ncv + r]
                ML_TRY(oz_gemm(OzMat{Q, 0, 1, n}, ncv, Sd.as<double>(), 1, ncv, 0, keep, OzOut{Qtmp.as<double>(), 0, 1, n},
                               ws.lay0.as<int>(), 1, n, false, st));
            } else {
                k_combine<<<nb, 256, 0, st>>>(Q, n, n, ncv, Sd.as<double>(), keep, Qtmp.as<double>(), n);
            }
        }
        ML_CUDA(cudaGetLastError());
        if (done) {
            for (int i = 0; i < k; ++i) {
                const double th = theta[ncv - 1 - i];
                evals[i] = pw > 0 ? 1.0 - th : std::pow(th, 1.0 / pw);
            }
            // ascending eigenvalues of the Laplacian: p = 1 maps descending theta to
            // ascending 1 - theta already; p < 0 maps descending mu to ascending mu^(1/p).
            if (evecs_dev) {
                ML_CUDA(cudaMemcpyAsync(evecs_dev, Qtmp.p, (size_t)n * k * 8, cudaMemcpyDeviceToDevice, st));
                ML_TRY(sign_fix_cols(evecs_dev, n, k, st));
                ML_CUDA(cudaGetLastError());
            }
            ML_CUDA(cudaStreamSynchronize(st));
            if (tensor) {
                int flags = 0;
                ML_TRY(oz_read_error(&flags, st));
                if (flags & 2) return fail(ML_ERR_TIMEOUT, "tensor-core product: a bounded wait gave up");
                if (flags & 1) return (ml_status)kRetryFp64;
            }
            if (nconv_out) *nconv_out = std::min(nconv, k);
            if (nconv >= k) return ML_OK;
            set_error("Lanczos stopped after " + std::to_string(matvecs) + " operator applications (maxit " +
                      std::to_string(maxit) + ") with " + std::to_string(nconv) + " of " + std::to_string(k) +
                      " pairs converged");
            return ML_WARN_NOT_CONVERGED;
        }
        // thick restart: Q[:, 0:kk] = Ritz vectors, Q[:, kk] = last residual direction
        kk = keep;
        ML_CUDA(cudaMemcpyAsync(Q + (int64_t)kk * n, Q + (int64_t)ncv * n, n * 8, cudaMemcpyDeviceToDevice, st));
        ML_CUDA(cudaMemcpyAsync(Q, Qtmp.p, (size_t)n * kk * 8, cudaMemcpyDeviceToDevice, st));
        std::fill(Tm.begin(), Tm.end(), 0.0);
        for (int i = 0; i < kk; ++i) {
            const int col = ncv - 1 - i;
            Tm[(size_t)i * ncv + i] = theta[col];
            const double coup = beta_last * S[(size_t)(ncv - 1) * ncv + col];
            Tm[(size_t)i * ncv + kk] = coup;
            Tm[(size_t)kk * ncv + i] = coup;
        }
    }
}

}  // namespace ml

extern "C" ml_status ml_lanczos_eigs(const ml_plan_t *layers, int T, int k, double p, double tol, int maxit,
                                     int block, uint64_t seed, double *evals, double *evecs, int *nconv,
                                     void *stream)
{
    using namespace ml;
    if (!layers || T < 1) return fail(ML_ERR_ARG, "layers is null or T < 1");
    for (int t = 0; t < T; ++t)
        if (!layers[t]) return fail(ML_ERR_ARG, "null layer");
    const int64_t n = layers[0]->n;
    for (int t = 1; t < T; ++t)
        if (layers[t]->n != n) return fail(ML_ERR_ARG, "layers do not share n");
    if (k < 1 || k > n / 2) return fail(ML_ERR_ARG, "k must be in [1, n/2]");
    if (!(p == 1.0 || (p < 0 && p >= -64.0))) return fail(ML_ERR_ARG, "p must be 1 or in [-64, 0)");
    if (block > 1) return fail(ML_ERR_ARG, "block Lanczos is not available (block must be 1)");
    for (int t = 0; t < T; ++t)
        if (!layers[t]->deg_ok) return fail(ML_ERR_DEGREE, "a layer has a degree <= 0: L_sym is undefined");
    if (!evals) return fail(ML_ERR_ARG, "evals is null");
    if (tol <= 0) tol = 1e-10;
    if (maxit <= 0) maxit = 2000;
    cudaStream_t st = (cudaStream_t)stream;
    double *evd = nullptr;
    DevBuf stage;
    bool host_out = false;
    if (evecs) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, evecs) == cudaSuccess &&
            (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)) {
            evd = evecs;
        } else {
            cudaGetLastError();
            ML_TRY(stage.ensure((size_t)n * k * 8));
            evd = stage.as<double>();
            host_out = true;
        }
    }
    ml_status s = lanczos_impl(layers, T, k, p, tol, maxit, seed, evals, evd, nconv, st, oz_enabled());
    if ((int)s == kRetryFp64) s = lanczos_impl(layers, T, k, p, tol, maxit, seed, evals, evd, nconv, st, false);
    if ((s == ML_OK || s == ML_WARN_NOT_CONVERGED) && host_out) {
        ML_CUDA(cudaMemcpy(evecs, evd, (size_t)n * k * 8, cudaMemcpyDeviceToHost));
    }
    return s;
}
