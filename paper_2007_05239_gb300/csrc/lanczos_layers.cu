// ml_lanczos_eigs_layers: for every layer t on its own, the k smallest
// eigenpairs of L_sym^(t) = I - D_t^{-1/2} W_t D_t^{-1/2} (Sec. 2), i.e. the
// k largest eigenpairs of the normalised operator A_t = D_t^{-1/2} W_t D_t^{-1/2},
// by block thick-restart Lanczos with full reorthogonalisation (the Lanczos
// method of Sec. 3 in block form).  All T problems advance in lockstep: each
// block step applies every active layer's operator to its own block of b
// vectors in one batched fast summation, then orthogonalises every layer's
// block with kernels batched over the layers.
//
// Per layer t (FP64, device, point-major rows):
//   Q_t  n x ldq, ldq = ncv + b: columns 0..ncv-1 the basis of the cycle,
//        ncv..ncv+b-1 the next (residual) block;
//   W_t  n x b, the product block.
// One block step for the block Q_j = Q[:, c:c+b] (cq = c + b):
//   W = A_t Q_j
//   W -= Q_{j-1} R_{j-1}^T, A_j = Q_j^T W, W -= Q_j A_j   (three-term part, j >= 1)
//   H1 = Q[:, 0:cq]^T W,  W -= Q[:, 0:cq] H1          (classical Gram-Schmidt)
//   W = V1 R1                                         (SVQB)
//   H2 = Q[:, 0:cq]^T V1, V1 -= Q[:, 0:cq] H2         (second pass, only when
//                                                      the first removed over
//                                                      half of a column's norm^2)
//   V1 = V2 R2, Q[:, cq:cq+b] = V2                    (SVQB)
// so that A Q_j = Q[:, 0:cq] (H1 + three-term part + H2 R1) + Q[:, cq:cq+b] (R2 R1):
// the columns c..c+b-1 of the projected matrix T = Q^T A Q.  The tensor-core
// kind of products keeps both passes in every step (orthonormalise).
// SVQB (Stathopoulos & Wu, SIAM J. Sci. Comput. 23 (2002)): G = W^T W,
// S = diag(G)^{-1/2}, S G S = U L U^T, V = W S U L^{-1/2}, R = L^{1/2} U^T S^{-1};
// directions with L_i <= 1e-20 max L are dropped (zero columns: the block
// deflates instead of breaking down).
// After ncv columns the host diagonalises each layer's T (ncv x ncv), checks
// the residuals ||R_last S[last block, i]|| of the k largest Ritz values, and
// restarts with the kkeep largest Ritz vectors plus the residual block.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "dword.cuh"
#include "ml_internal.h"

namespace ml {

constexpr int kRows = 32;     // rows staged per chunk
constexpr int kMaxLd = 96;    // basis columns incl. the residual block
constexpr int kMaxBlk = 8;    // block size limit
constexpr int kGramOut = 768; // Gram outputs per CTA (3 per thread)

// per-layer row-major n x ld matrices at base + t * stride
struct LMat {
    double *base;
    int64_t stride;
    int ld;
    __device__ __forceinline__ double *at(int t) const { return base + (int64_t)t * stride; }
};

// part[(y * gridDim.x + x) * rc * cb + r * cb + s] = sum over this CTA's rows i
// of A_t[i, a0 + r] * B_t[i, b0 + s], t = lay[y]   (rc * cb <= kGramOut)
__global__ void __launch_bounds__(256) k_lgram(LMat A, int a0, int rc, LMat B, int b0, int cb,
                                              const int *__restrict__ lay, int64_t n, double *part,
                                              const int *__restrict__ gate)
{
    if (gate && *gate == 0) return;   // a pass the device decided to skip
    __shared__ double As[kRows][kMaxLd + 1];
    __shared__ double Bs[kRows][kMaxBlk + 1];
    const int t = lay[blockIdx.y];
    const double *Ab = A.at(t), *Bb = B.at(t);
    const int nout = rc * cb;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t i0 = (int64_t)blockIdx.x * kRows; i0 < n; i0 += (int64_t)gridDim.x * kRows) {
        const int rows = (int)min((int64_t)kRows, n - i0);
        for (int e = threadIdx.x; e < kRows * rc; e += blockDim.x) {
            const int rr = e / rc, cc = e - rr * rc;
            As[rr][cc] = rr < rows ? Ab[(i0 + rr) * A.ld + a0 + cc] : 0.0;
        }
        for (int e = threadIdx.x; e < kRows * cb; e += blockDim.x) {
            const int rr = e / cb, cc = e - rr * cb;
            Bs[rr][cc] = rr < rows ? Bb[(i0 + rr) * B.ld + b0 + cc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int e = threadIdx.x + q * 256;
            if (e < nout) {
                const int r = e / cb, s = e - r * cb;
                double v = acc[q];
#pragma unroll 8
                for (int rr = 0; rr < kRows; ++rr) v = fma(As[rr][r], Bs[rr][s], v);
                acc[q] = v;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int e = threadIdx.x + q * 256;
        if (e < nout) part[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * nout + e] = acc[q];
    }
}

// ---- double-word versions (FP32 pipes, ~47 bits) of the basis products
// k_lgram_dw: as k_lgram.  The CTA's outputs (r, s) are grouped in blocks of
// 4 r x 2 s; thread t works on block t % nblk over the rows of each staged
// chunk with index = t / nblk (mod the number of phases), and the phases'
// partial sums are added in a fixed order at the end.
constexpr int kDwRows = 32;
__global__ void __launch_bounds__(256) k_lgram_dw(LMat A, int a0, int rc, LMat B, int b0, int cb,
                                                 const int *__restrict__ lay, int64_t n, double *part,
                                                 const int *__restrict__ gate)
{
    if (gate && *gate == 0) return;
    __shared__ float2 As[kDwRows][kMaxLd + 1];
    __shared__ float2 Bs[kDwRows][kMaxBlk + 1];
    __shared__ double red[kGramOut];
    const int t = lay[blockIdx.y];
    const double *Ab = A.at(t), *Bb = B.at(t);
    const int rb = (rc + 3) / 4, sb = (cb + 1) / 2, nblk = rb * sb;
    const int phases = max(1, (int)blockDim.x / nblk);
    const int blk = threadIdx.x % nblk, ph = threadIdx.x / nblk;
    const bool active = ph < phases && (int)threadIdx.x < nblk * phases;
    const int r0 = (blk / sb) * 4, s0 = (blk % sb) * 2;
    float2 acc[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = make_float2(0.0f, 0.0f);
    for (int64_t i0 = (int64_t)blockIdx.x * kDwRows; i0 < n; i0 += (int64_t)gridDim.x * kDwRows) {
        const int rows = (int)min((int64_t)kDwRows, n - i0);
        for (int e = threadIdx.x; e < kDwRows * rc; e += blockDim.x) {
            const int rr = e / rc, cc = e - rr * rc;
            As[rr][cc] = rr < rows ? dword::from_double(Ab[(i0 + rr) * A.ld + a0 + cc]) : make_float2(0.0f, 0.0f);
        }
        for (int e = threadIdx.x; e < kDwRows * cb; e += blockDim.x) {
            const int rr = e / cb, cc = e - rr * cb;
            Bs[rr][cc] = rr < rows ? dword::from_double(Bb[(i0 + rr) * B.ld + b0 + cc]) : make_float2(0.0f, 0.0f);
        }
        __syncthreads();
        if (active)
            for (int rr = ph; rr < kDwRows; rr += phases) {
                float2 a[4], b[2];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = r0 + i < rc ? As[rr][r0 + i] : make_float2(0.0f, 0.0f);
#pragma unroll
                for (int j = 0; j < 2; ++j) b[j] = s0 + j < cb ? Bs[rr][s0 + j] : make_float2(0.0f, 0.0f);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 2; ++j) dword::fma_acc(acc[i][j], a[i], b[j]);
            }
        __syncthreads();
    }
    // phases -> one partial per output, summed in phase order
    const int nout = rc * cb;
    for (int e = threadIdx.x; e < nout; e += blockDim.x) red[e] = 0.0;
    __syncthreads();
    for (int p = 0; p < phases; ++p) {
        if (active && ph == p)
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j)
                    if (r0 + i < rc && s0 + j < cb) red[(r0 + i) * cb + s0 + j] += dword::to_double(acc[i][j]);
        __syncthreads();
    }
    for (int e = threadIdx.x; e < nout; e += blockDim.x)
        part[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * nout + e] = red[e];
}

// k_lgemm_dw: as k_lgemm (B_t[i, b0 + s] (-)= sum_r A_t[i, a0 + r] M_y[r, s]);
// one row per thread with its cb accumulators, the chunk of rows staged in
// double-word and M (double-word) read by all threads alike
constexpr int kDwGemmRows = 128;
// (M_y row-major with leading dimension ldm: M_y = M + y * rc * ldm, columns
// 0..cb-1 of it; cb <= 8)
__global__ void __launch_bounds__(kDwGemmRows) k_lgemm_dw(LMat A, int a0, int rc, const double *__restrict__ M, int ldm,
                                                         LMat B, int b0, int cb, const int *__restrict__ lay,
                                                         int64_t n, int sub, const int *__restrict__ gate)
{
    if (gate && *gate == 0) return;
    extern __shared__ float2 dsm[];
    float2 *Ms = dsm;                          // rc * cb
    float2 *As = dsm + rc * cb;                // kDwGemmRows x (rc + 1)
    const int t = lay[blockIdx.y];
    const double *Ab = A.at(t);
    double *Bb = B.at(t);
    const double *My = M + (int64_t)blockIdx.y * rc * ldm;
    for (int e = threadIdx.x; e < rc * cb; e += blockDim.x) {
        const int r = e / cb, s2 = e - r * cb;
        Ms[e] = dword::from_double(My[(int64_t)r * ldm + s2]);
    }
    const int lda = rc + 1;
    for (int64_t i0 = (int64_t)blockIdx.x * kDwGemmRows; i0 < n; i0 += (int64_t)gridDim.x * kDwGemmRows) {
        const int rows = (int)min((int64_t)kDwGemmRows, n - i0);
        __syncthreads();   // the previous chunk is no longer read (and Ms is ready)
        for (int e = threadIdx.x; e < rows * rc; e += blockDim.x) {
            const int rr = e / rc, cc = e - rr * rc;
            As[rr * lda + cc] = dword::from_double(Ab[(i0 + rr) * A.ld + a0 + cc]);
        }
        __syncthreads();
        const int rr = threadIdx.x;
        if (rr < rows) {
            float2 acc[kMaxBlk];
#pragma unroll
            for (int s = 0; s < kMaxBlk; ++s) acc[s] = make_float2(0.0f, 0.0f);
            for (int r = 0; r < rc; ++r) {
                const float2 a = As[rr * lda + r];
#pragma unroll
                for (int s = 0; s < kMaxBlk; ++s)
                    if (s < cb) dword::fma_acc(acc[s], a, Ms[r * cb + s]);
            }
            double *bp = Bb + (i0 + rr) * B.ld + b0;
#pragma unroll
            for (int s = 0; s < kMaxBlk; ++s)
                if (s < cb) bp[s] = sub ? bp[s] - dword::to_double(acc[s]) : dword::to_double(acc[s]);
        }
    }
}

// out[y][e] = sum over the nbx partial blocks in a fixed order; with rec,
// also rec[lay[y] * rstride + e] = out[y][e]
__global__ void k_lreduce(const double *__restrict__ part, int nbx, int nout, const int *__restrict__ lay,
                          double *out, double *rec, int64_t rstride, const int *__restrict__ gate)
{
    if (gate && *gate == 0) return;
    const int y = blockIdx.y;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nout; e += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int bx = 0; bx < nbx; ++bx) s += part[((int64_t)y * nbx + bx) * nout + e];
        out[(int64_t)y * nout + e] = s;
        if (rec) rec[(int64_t)lay[y] * rstride + e] = s;
    }
}

// B_t[i, b0 + s] = x  or  B_t[i, b0 + s] -= x,  x = sum_{r < rc} A_t[i, a0 + r] M_y[r, s]
// (M_y = M + y * rc * cb, row-major rc x cb).  Rows are staged per chunk, so
// B may be A (in place on the same columns).
__global__ void __launch_bounds__(256) k_lgemm(LMat A, int a0, int rc, const double *__restrict__ M, LMat B, int b0,
                                              int cb, const int *__restrict__ lay, int64_t n, int sub,
                                              const int *__restrict__ gate)
{
    if (gate && *gate == 0) return;
    extern __shared__ double lsm[];
    double *Ms = lsm;                 // rc * cb
    double *As = lsm + rc * cb;       // kRows x (rc + 1)
    const int t = lay[blockIdx.y];
    const double *Ab = A.at(t);
    double *Bb = B.at(t);
    const double *My = M + (int64_t)blockIdx.y * rc * cb;
    for (int e = threadIdx.x; e < rc * cb; e += blockDim.x) Ms[e] = My[e];
    const int lda = rc + 1;
    for (int64_t i0 = (int64_t)blockIdx.x * kRows; i0 < n; i0 += (int64_t)gridDim.x * kRows) {
        const int rows = (int)min((int64_t)kRows, n - i0);
        __syncthreads();   // the previous chunk is no longer read (and Ms is loaded)
        for (int e = threadIdx.x; e < rows * rc; e += blockDim.x) {
            const int rr = e / rc, cc = e - rr * rc;
            As[rr * lda + cc] = Ab[(i0 + rr) * A.ld + a0 + cc];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < rows * cb; e += blockDim.x) {
            const int rr = e / cb, s = e - rr * cb;
            double x = 0.0;
            for (int r = 0; r < rc; ++r) x = fma(As[rr * lda + r], Ms[r * cb + s], x);
            double *bp = Bb + (i0 + rr) * B.ld + b0 + s;
            *bp = sub ? *bp - x : x;
        }
    }
}

// SVQB of the B x B Gram G_y, eight lanes per slot (four slots per warp):
// lane k of a slot holds column k of the scaled Gram and of the eigenvector
// matrix in registers, and the cyclic Jacobi rotations (p, q) exchange
// columns p and q by shuffles within the slot's lanes (a thread per slot held
// three B x B matrices and spilled them to local memory).  Writes the
// transform M_y (V = W M) and R (W = V R): into Rs_y on the first pass, and
// R2 * Rs_y into rec[lay[y] * rstride] on the second.  flags[lay[y]] |= 1
// when a direction was dropped.  B is a template parameter so that the
// columns stay in registers.
template <int B>
__global__ void __launch_bounds__(128) k_lsvqb(const double *__restrict__ G, int nslots, const int *__restrict__ lay,
                                               double *M, double *Rs, double *rec, int64_t rstride, int pass, int *flags)
{
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = gid >> 3;          // slot
    const int k = gid & 7;           // column of this lane
    const bool slot_ok = y < nslots;
    const bool col_ok = slot_ok && k < B;
    const unsigned full = 0xffffffffu;
    const int t = slot_ok ? lay[y] : 0;
    const double *Gy = G + (int64_t)(slot_ok ? y : 0) * B * B;
    double sc[B];
#pragma unroll
    for (int i = 0; i < B; ++i) {
        const double d = slot_ok ? Gy[i * B + i] : 0.0;
        sc[i] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
    }
    // column k of the scaled, symmetrised Gram and of U (identity)
    double g[B], u[B];
#pragma unroll
    for (int i = 0; i < B; ++i) {
        g[i] = col_ok ? 0.5 * (Gy[i * B + k] + Gy[k * B + i]) * sc[i] * sc[k] : 0.0;
        u[i] = (col_ok && i == k) ? 1.0 : 0.0;
    }
    const int base = threadIdx.x & ~7;   // first lane of the slot within the warp
    for (int sweep = 0; sweep < 30; ++sweep) {
        bool rotated = false;
#pragma unroll
        for (int p = 0; p < B - 1; ++p)
#pragma unroll
            for (int q = p + 1; q < B; ++q) {
                // g[p][q] lives in lane q (its element p), g[p][p] in lane p, g[q][q] in lane q
                const double apq = __shfl_sync(full, g[p], (base & 31) + q);
                const double app = __shfl_sync(full, g[p], (base & 31) + p);
                const double aqq = __shfl_sync(full, g[q], (base & 31) + q);
                // rotate while the pair is coupled beyond rounding: 1e-15 of
                // sqrt(app aqq) (a bound below the FP64 rounding level never
                // holds once rounding noise remains, and every call ran all 30
                // sweeps)
                const bool rot = !(fabs(apq) <= 1e-15 * sqrt(fabs(app * aqq)) + 1e-300);
                double c = 1.0, sn = 0.0;
                if (rot) {
                    rotated = true;
                    const double tau = (aqq - app) / (2.0 * apq);
                    const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    c = 1.0 / sqrt(1.0 + tt * tt);
                    sn = tt * c;
                }
                // rows p and q of every column (lane-local)
                {
                    const double gp = g[p], gq = g[q];
                    g[p] = c * gp - sn * gq;
                    g[q] = sn * gp + c * gq;
                }
                // columns p and q: lanes p and q take each other's column
                const int partner = (k == p) ? q : ((k == q) ? p : k);
#pragma unroll
                for (int i = 0; i < B; ++i) {
                    const double og = __shfl_sync(full, g[i], (base & 31) + partner);
                    const double ou = __shfl_sync(full, u[i], (base & 31) + partner);
                    if (k == p) {
                        g[i] = c * g[i] - sn * og;
                        u[i] = c * u[i] - sn * ou;
                    } else if (k == q) {
                        g[i] = sn * og + c * g[i];
                        u[i] = sn * ou + c * u[i];
                    }
                }
            }
        // every lane of a slot took the same decisions; the warp continues
        // while any of its slots rotated
        if (!__any_sync(full, rotated)) break;
    }
    // eigenvalue of column k: g[k]
    double lamk = 0.0;
#pragma unroll
    for (int i = 0; i < B; ++i)
        if (i == k) lamk = g[i];
    double lmax = col_ok ? lamk : 0.0;
    for (int o = 4; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(full, lmax, o));
    const bool keep = col_ok && lmax > 0.0 && lamk > 1e-20 * lmax;
    const double il = keep ? 1.0 / sqrt(lamk) : 0.0, sl = keep ? sqrt(lamk) : 0.0;
    if (col_ok) {
        double *My = M + (int64_t)y * B * B;
#pragma unroll
        for (int r = 0; r < B; ++r) My[r * B + k] = sc[r] * u[r] * il;
    }
    // row k of R: R[k][q] = sl_k u[q][k] / sc[q]
    double Rk[B];
#pragma unroll
    for (int q = 0; q < B; ++q) Rk[q] = (sc[q] > 0.0) ? sl * u[q] / sc[q] : 0.0;
    double *Ry = Rs + (int64_t)(slot_ok ? y : 0) * B * B;
    if (col_ok) {
        if (pass == 0) {
#pragma unroll
            for (int j = 0; j < B; ++j) Ry[k * B + j] = Rk[j];
        } else if (rec) {
            double *Rt = rec + (int64_t)t * rstride;
#pragma unroll
            for (int j = 0; j < B; ++j) {
                double x = 0.0;
#pragma unroll
                for (int q = 0; q < B; ++q) x = fma(Rk[q], Ry[q * B + j], x);
                Rt[k * B + j] = x;
            }
        }
    }
    const bool dropped = col_ok && !keep;
    if (dropped && flags) atomicOr(flags + t, 1);
}

// rec_t[r, s] += sum_q H2_y[r, q] Rs_y[q, s]   (r < rc): the second pass's
// coefficients mapped back to the product block
__global__ void k_lhacc(const double *__restrict__ H2, const double *__restrict__ Rs, int rc, int b,
                        const int *__restrict__ lay, double *rec, int64_t rstride, const int *__restrict__ gate)
{
    if (gate && *gate == 0) return;
    const int y = blockIdx.y;
    const double *H = H2 + (int64_t)y * rc * b, *R = Rs + (int64_t)y * b * b;
    double *out = rec + (int64_t)lay[y] * rstride;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rc * b; e += gridDim.x * blockDim.x) {
        const int r = e / b, s = e - r * b;
        double x = 0.0;
        for (int q = 0; q < b; ++q) x = fma(H[r * b + q], R[q * b + s], x);
        out[e] += x;
    }
}

// Three-term part of a block step: M_y[s, q] = R_t[q, s] for the record R_t
// (b x b, row-major) of the previous step, t = lay[y]: A Q_{j-1} has the
// component Q_j R, so A Q_j has the component Q_{j-1} R^T
__global__ void k_lthree(const double *__restrict__ rprev, int64_t rstride, const int *__restrict__ lay, int nslots,
                         int b, double *M)
{
    const int y = blockIdx.x;
    if (y >= nslots) return;
    const double *R = rprev + (int64_t)lay[y] * rstride;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        const int s = e / b, q = e - s * b;
        M[(int64_t)y * b * b + e] = R[q * b + s];
    }
}

// the coefficients the three-term part removed, added to this step's record
// (rows c - b .. c - 1: M_y = R^T when given; rows c .. c + b - 1: A_y)
__global__ void k_lrec_add(double *rec, int64_t rstride, const int *__restrict__ lay, int nslots, const double *M,
                           const double *__restrict__ A, int c, int b)
{
    const int y = blockIdx.x;
    if (y >= nslots) return;
    double *R = rec + (int64_t)lay[y] * rstride;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        const int s = e / b, q = e - s * b;
        if (M) R[(int64_t)(c - b + s) * b + q] += M[(int64_t)y * b * b + e];
        R[(int64_t)(c + s) * b + q] += A[(int64_t)y * b * b + e];
    }
}

// Second-pass criterion over all active layers: *flag = 1 when some column
// of some layer kept less than eta2 of its norm squared through the first
// Gram-Schmidt pass (G0: the block's Gram matrix before it, G after);
// *flag is cleared by the caller before
__global__ void k_ldgks(const double *__restrict__ G0, const double *__restrict__ G, int nslots, int b, double eta2,
                        int *flag)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nslots * b; e += gridDim.x * blockDim.x) {
        const int y = e / b, s = e - y * b;
        const double before = G0[(int64_t)y * b * b + s * b + s], after = G[(int64_t)y * b * b + s * b + s];
        if (after < eta2 * before) atomicOr(flag, 1);
    }
}

// SplitMix64 (Steele, Lea, Flood 2014) of a counter, mapped to (-1, 1)
__device__ __forceinline__ double lz_uniform(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z = z ^ (z >> 31);
    return ((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
}

// Q_t[i, c0 + s] = random, an independent stream per layer
__global__ void k_lrandom(LMat Q, int c0, int b, const int *__restrict__ lay, uint64_t seed, int64_t n)
{
    const int t = lay[blockIdx.y];
    double *Qt = Q.at(t);
    const uint64_t sd = seed ^ (0xD1B54A32D192ED03ULL * (uint64_t)(t + 1));
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * b; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / b;
        const int s = (int)(e - i * b);
        Qt[i * Q.ld + c0 + s] = lz_uniform(sd, (uint64_t)e);
    }
}

// B_t[i, b0 + s] = A_t[i, a0 + s], s < cols
__global__ void k_lcopy(LMat A, int a0, LMat B, int b0, int cols, const int *__restrict__ lay, int64_t n)
{
    const int t = lay[blockIdx.y];
    const double *At = A.at(t);
    double *Bt = B.at(t);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * cols;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / cols;
        const int s = (int)(e - i * cols);
        Bt[i * B.ld + b0 + s] = At[i * A.ld + a0 + s];
    }
}

// out[j * n + i] = Q_t[i, j] for j < k (column-major n x k)
__global__ void k_lcolmajor(LMat Q, int t, int k, int64_t n, double *out)
{
    const double *Qt = Q.at(t);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * k; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / n);
        const int64_t i = e - (int64_t)j * n;
        out[e] = Qt[i * Q.ld + j];
    }
}

// --------------------------------------------------------------------- host
namespace {

struct Solver {
    ml_plan_s *const *L;
    int T, k, b;
    int64_t n;
    int ncv = 0, ldq = 0, kkeep = 0, nsteps_max = 0;
    int nbx = 1;
    cudaStream_t st;
    DevBuf Q[2], Wb, part, hcur, Gs, Ms, Rs, Hrec, Rrec, Sd, layd, flags;
    DevBuf G0s, Mt, Ajs, dflag;         // block_step: Gram before the pass, R^T, A_j, second-pass flag
    DescSlot desc;
    int64_t hstride = 0, rstride = 0;   // per layer record strides (doubles)
    int nslots = 0;                     // active layers
    bool tensor = false;                // products of the basis on the tensor cores
    bool dword = false;                 // products of the basis in double-word FP32
    std::vector<int> lay;               // slot -> layer

    LMat q(int which) const { return LMat{Q[which].as<double>(), n * ldq, ldq}; }

    // CTAs per layer so that the launch (x nslots) fills one wave of resident
    // CTAs of `kernel` (a partial last wave leaves SMs idle), at most nbx
    template <typename K>
    int wave_x(K kernel, int threads, size_t smem) const
    {
        int r = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, kernel, threads, smem) != cudaSuccess || r <= 0) {
            cudaGetLastError();
            return nbx;
        }
        return std::max(1, std::min(nbx, sm_count() * r / std::max(1, nslots)));
    }
    LMat w() const { return LMat{Wb.as<double>(), n * b, b}; }

    ml_status upload_lay()
    {
        nslots = (int)lay.size();
        ML_CUDA(cudaMemcpyAsync(layd.p, lay.data(), lay.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        ML_CUDA(cudaStreamSynchronize(st));   // lay is host memory that changes later
        nbx = (int)std::max<int64_t>(1, std::min<int64_t>((n + kRows - 1) / kRows, (sm_count() * 8 + nslots - 1) / nslots));
        return ML_OK;
    }

    // out[y] (rc x cb) = A_t[:, a0:a0+rc]^T B_t[:, b0:b0+cb]; optionally recorded.
    // basis: A is the orthonormal basis and B a block of norm-bounded vectors
    // (|entries| < 2), so the product may run on the tensor cores (ozaki.cu)
    ml_status gram(LMat A, int a0, int rc, LMat B, int b0, int cb, double *out, double *rec, int64_t rs,
                   bool basis = false, const int *gate = nullptr, const char *family = "dots")
    {
        const int nout = rc * cb;
        if (nout > kGramOut) return fail(ML_ERR_ARG, "Gram block too large");
        // double-word products for every Gram of the double-word kind (any
        // magnitudes: the block's own Gram W^T W as well; the FP64 kernel's
        // 8 x 8 outputs left most of its threads idle at each chunk's barrier)
        int nb = nbx;
        const bool dw = dword && rc <= kMaxLd && cb <= kMaxBlk;
        if (dw) nb = wave_x(k_lgram_dw, 256, 0);
        if (dw) {
            ProfScope pr(family, st);
            k_lgram_dw<<<dim3(nb, nslots), 256, 0, st>>>(A, a0, rc, B, b0, cb, layd.as<int>(), n, part.as<double>(),
                                                         gate);
        } else if (basis && tensor && oz_gram_ok(rc, cb)) {
            ProfScope pr("dots", st);
            nb = oz_gram_blocks(nslots, n);
            ML_TRY(oz_gram(OzMat{A.base + a0, A.stride, A.ld, 1}, rc, OzMat{B.base + b0, B.stride, B.ld, 1}, cb,
                           layd.as<int>(), nslots, n, nb, part.as<double>(), st));
        } else {
            ProfScope pr(family, st);
            k_lgram<<<dim3(nbx, nslots), 256, 0, st>>>(A, a0, rc, B, b0, cb, layd.as<int>(), n, part.as<double>(),
                                                      gate);
        }
        {
            ProfScope pr("dots_reduce", st);
            k_lreduce<<<dim3((nout + 127) / 128, nslots), 128, 0, st>>>(part.as<double>(), nb, nout, layd.as<int>(),
                                                                       out, rec, rs, gate);
        }
        ML_CUDA(cudaGetLastError());
        return ML_OK;
    }

    // B_t[:, b0:b0+cb] (-)= A_t[:, a0:a0+rc] M_y (M any magnitude); B may be A.
    // Double-word kind: k_lgemm_dw for every product; basis (A the orthonormal
    // basis, entries below 2) lets the tensor-core kind take it
    ml_status gemm(LMat A, int a0, int rc, const double *M, LMat B, int b0, int cb, bool sub, bool basis = false,
                   const char *family = "update", const int *gate = nullptr)
    {
        ProfScope pr(family, st);
        if (dword && rc <= kMaxLd) {
            for (int j0 = 0; j0 < cb; j0 += kMaxBlk) {
                const int w = std::min(kMaxBlk, cb - j0);
                const size_t smem = ((size_t)rc * w + (size_t)kDwGemmRows * (rc + 1)) * sizeof(float2);
                k_lgemm_dw<<<dim3(wave_x(k_lgemm_dw, kDwGemmRows, smem), nslots), kDwGemmRows, smem, st>>>(
                    A, a0, rc, M + j0, cb, B, b0 + j0, w, layd.as<int>(), n, sub ? 1 : 0, gate);
            }
            ML_CUDA(cudaGetLastError());
            return ML_OK;
        }
        if (basis && tensor && oz_gemm_ok(rc))
            return oz_gemm(OzMat{A.base + a0, A.stride, A.ld, 1}, rc, M, cb, 1, (int64_t)rc * cb, cb,
                           OzOut{B.base + b0, B.stride, B.ld, 1}, layd.as<int>(), nslots, n, sub, st);
        const size_t smem = ((size_t)rc * cb + (size_t)kRows * (rc + 1)) * sizeof(double);
        k_lgemm<<<dim3(nbx, nslots), 256, smem, st>>>(A, a0, rc, M, B, b0, cb, layd.as<int>(), n, sub ? 1 : 0, gate);
        ML_CUDA(cudaGetLastError());
        return ML_OK;
    }

    ml_status svqb(int pass, double *rec)
    {
        ProfScope pr("svqb", st);
        const dim3 grid((nslots * 8 + 127) / 128);
        double *G = Gs.as<double>(), *Mp = Ms.as<double>(), *Rp = Rs.as<double>();
        const int *ly = layd.as<int>();
        int *fl = flags.as<int>();
        switch (b) {
#define ML_SVQB_CASE(BB) \
    case BB: k_lsvqb<BB><<<grid, 128, 0, st>>>(G, nslots, ly, Mp, Rp, rec, rstride, pass, fl); break;
            ML_SVQB_CASE(1)
            ML_SVQB_CASE(2)
            ML_SVQB_CASE(3)
            ML_SVQB_CASE(4)
            ML_SVQB_CASE(5)
            ML_SVQB_CASE(6)
            ML_SVQB_CASE(7)
            ML_SVQB_CASE(8)
#undef ML_SVQB_CASE
        default: return fail(ML_ERR_ARG, "block size out of range");
        }
        ML_CUDA(cudaGetLastError());
        return ML_OK;
    }

    // orthonormalise the block W (columns 0..b-1 of w()) against Q[:, 0:cq]
    // (cq > 0) and within itself; result into Q_dst[:, d0:d0+b].  hrec/rrec:
    // this step's records (hrec null: no Gram-Schmidt coefficients kept).
    ml_status orthonormalise(int cur, int cq, LMat dst, int d0, double *hrec, double *rrec)
    {
        const LMat Qc = q(cur), Wm = w();
        double *h = hcur.as<double>();
        if (cq > 0) {
            ML_TRY(gram(Qc, 0, cq, Wm, 0, b, h, hrec, hstride, true));
            ML_TRY(gemm(Qc, 0, cq, h, Wm, 0, b, true, true));
        }
        ML_TRY(gram(Wm, 0, b, Wm, 0, b, Gs.as<double>(), nullptr, 0));
        ML_TRY(svqb(0, nullptr));
        ML_TRY(gemm(Wm, 0, b, Ms.as<double>(), Wm, 0, b, false));
        if (cq > 0) {
            ML_TRY(gram(Qc, 0, cq, Wm, 0, b, h, nullptr, 0, true));
            ML_TRY(gemm(Qc, 0, cq, h, Wm, 0, b, true, true));
            if (hrec) {
                ProfScope pr("svqb", st);
                k_lhacc<<<dim3((cq * b + 127) / 128, nslots), 128, 0, st>>>(h, Rs.as<double>(), cq, b, layd.as<int>(),
                                                                           hrec, hstride, nullptr);
                ML_CUDA(cudaGetLastError());
            }
        }
        ML_TRY(gram(Wm, 0, b, Wm, 0, b, Gs.as<double>(), nullptr, 0));
        ML_TRY(svqb(1, rrec));
        ML_TRY(gemm(Wm, 0, b, Ms.as<double>(), dst, d0, b, false));
        return ML_OK;
    }

    // One block step for the block Q[:, c:c+b] (step j of the cycle), W = A Q_j
    // on entry; FP64-pipe or double-word products (the tensor-core kind uses
    // orthonormalise).  The three-term part first: W -= Q_{j-1} R^T (R the
    // previous step's record, j >= 1), A_j = Q_j^T W, W -= Q_j A_j.  Then one
    // Gram-Schmidt pass against Q[:, 0:c+b] and SVQB, and a second pass only
    // when some column of some layer lost more than half of its norm squared
    // in the first (the criterion of Daniel, Gragg, Kaufman and Stewart
    // 1976, decided on the device; the second pass's kernels return at once
    // otherwise), then SVQB into Q[:, c+b:c+2b].  The record holds the same
    // coefficients as orthonormalise's: the three-term part's are added back.
    ml_status block_step(int cur, int c, int j, double *hrec, double *rrec)
    {
        const LMat Qc = q(cur), Wm = w();
        const int cq = c + b;
        double *h = hcur.as<double>();
        int *fl = dflag.as<int>();
        const double *rprev = j >= 1 ? Rrec.as<double>() + (int64_t)(j - 1) * b * b : nullptr;
        if (rprev) {
            {
                ProfScope pr("vector", st);
                k_lthree<<<nslots, 64, 0, st>>>(rprev, rstride, layd.as<int>(), nslots, b, Mt.as<double>());
            }
            ML_TRY(gemm(Qc, c - b, b, Mt.as<double>(), Wm, 0, b, true, true));
        }
        ML_TRY(gram(Qc, c, b, Wm, 0, b, Ajs.as<double>(), nullptr, 0, true));
        ML_TRY(gemm(Qc, c, b, Ajs.as<double>(), Wm, 0, b, true, true));
        ML_TRY(gram(Wm, 0, b, Wm, 0, b, G0s.as<double>(), nullptr, 0));
        ML_TRY(gram(Qc, 0, cq, Wm, 0, b, h, hrec, hstride, true));
        ML_TRY(gemm(Qc, 0, cq, h, Wm, 0, b, true, true));
        {
            ProfScope pr("svqb", st);
            k_lrec_add<<<nslots, 64, 0, st>>>(hrec, hstride, layd.as<int>(), nslots, rprev ? Mt.as<double>() : nullptr,
                                             Ajs.as<double>(), c, b);
        }
        ML_TRY(gram(Wm, 0, b, Wm, 0, b, Gs.as<double>(), nullptr, 0));
        ML_TRY(svqb(0, nullptr));
        {
            ProfScope pr("svqb", st);
            ML_CUDA(cudaMemsetAsync(fl, 0, sizeof(int), st));
            k_ldgks<<<std::max(1, (nslots * b + 127) / 128), 128, 0, st>>>(G0s.as<double>(), Gs.as<double>(), nslots, b,
                                                                          0.5, fl);
        }
        ML_TRY(gemm(Wm, 0, b, Ms.as<double>(), Wm, 0, b, false));
        ML_TRY(gram(Qc, 0, cq, Wm, 0, b, h, nullptr, 0, true, fl, "dots2"));
        ML_TRY(gemm(Qc, 0, cq, h, Wm, 0, b, true, true, "update2", fl));
        if (hrec) {
            ProfScope pr("svqb", st);
            k_lhacc<<<dim3((cq * b + 127) / 128, nslots), 128, 0, st>>>(h, Rs.as<double>(), cq, b, layd.as<int>(), hrec,
                                                                       hstride, fl);
        }
        ML_CUDA(cudaGetLastError());
        ML_TRY(gram(Wm, 0, b, Wm, 0, b, Gs.as<double>(), nullptr, 0));
        ML_TRY(svqb(1, rrec));
        ML_TRY(gemm(Wm, 0, b, Ms.as<double>(), q(cur), cq, b, false));
        return ML_OK;
    }

    // W_t = A_t Q_t[:, c:c+b] for the active layers
    ml_status apply(int cur, int c)
    {
        std::vector<ml_plan_s *> pl(nslots);
        for (int y = 0; y < nslots; ++y) pl[y] = L[lay[y]];
        double *Qb = Q[cur].as<double>(), *Wp = Wb.as<double>();
        ApplyOpts o;
        o.normalized = true;
        if (nslots >= 2 && batchable_layers(pl.data(), nslots)) {
            std::vector<ApplyVec> vs(nslots);
            for (int c0 = 0, nv = 0; c0 < b; c0 += nv) {
                nv = 8;
                for (int y = 0; y < nslots; ++y) nv = std::min(nv, pass_width(pl[y], b - c0));
                for (int y = 0; y < nslots; ++y) {
                    const int t = lay[y];
                    vs[y] = ApplyVec{Qb + (int64_t)t * n * ldq + c + c0, ldq, Wp + (int64_t)t * n * b + c0, b, nv};
                }
                o.layer_vecs = vs.data();
                o.desc = &desc;
                ML_TRY(run_batch(pl.data(), nslots, vs[0], o, st));
            }
            return ML_OK;
        }
        for (int y = 0; y < nslots; ++y) {
            const int t = lay[y];
            for (int c0 = 0, nv = 0; c0 < b; c0 += nv) {
                nv = pass_width(pl[y], b - c0);
                ApplyVec v{Qb + (int64_t)t * n * ldq + c + c0, ldq, Wp + (int64_t)t * n * b + c0, b, nv};
                ML_TRY(apply_layer(pl[y], v, o, st));
            }
        }
        return ML_OK;
    }
};

}  // namespace

// returned by layers_impl when a tensor-core product met an operand beyond its
// fixed scale: the solve is repeated with the FP64-pipe products
constexpr int kRetryFp64 = 1000;

static ml_status layers_impl(ml_plan_s *const *L, int T, int k, double tol, int maxit, int b, int ncv_req,
                             uint64_t seed, double *evals, double *evecs_dev, int *nconv_out, cudaStream_t st,
                             bool tensor)
{
    Solver S;
    S.tensor = tensor;
    S.dword = !tensor && dense_products_kind() == 1;
    if (tensor) ML_TRY(oz_reset_error(st));
    S.L = L;
    S.T = T;
    S.k = k;
    S.b = b;
    S.n = L[0]->n;
    S.st = st;
    const int64_t n = S.n;
    const int target = ncv_req > 0 ? ncv_req - b : std::max(2 * k + 1, 20);
    int ncv = b * ((target + 2 * b - 1) / b);
    ncv = (int)std::min<int64_t>(ncv, (int64_t)b * ((n - b) / b));
    const int keep_goal = std::max(k + 1, (ncv + k) / 2);
    int kkeep = ncv - b * ((ncv - keep_goal + b - 1) / b);
    if (ncv + b > kMaxLd || (ncv + b) * b > kGramOut)
        return fail(ML_ERR_ARG, "k too large for the block size (basis beyond " + std::to_string(kMaxLd) + " columns)");
    if (kkeep < k + 1 || kkeep >= ncv) return fail(ML_ERR_ARG, "n too small for k and the block size");
    S.ncv = ncv;
    S.ldq = ncv + b;
    S.kkeep = kkeep;
    S.nsteps_max = ncv / b;
    S.hstride = (int64_t)S.nsteps_max * S.ldq * b;
    S.rstride = (int64_t)S.nsteps_max * b * b;
    const int ldq = S.ldq;
    for (int w = 0; w < 2; ++w) ML_TRY(S.Q[w].ensure((size_t)T * n * ldq * sizeof(double)));
    ML_TRY(S.Wb.ensure((size_t)T * n * b * sizeof(double)));
    const int64_t nbx_max = std::max<int64_t>(1, std::min<int64_t>((n + kRows - 1) / kRows, sm_count() * 8));
    ML_TRY(S.part.ensure((size_t)T * nbx_max * kGramOut * sizeof(double) + 64));
    ML_TRY(S.hcur.ensure((size_t)T * ldq * b * sizeof(double)));
    ML_TRY(S.Gs.ensure((size_t)T * b * b * sizeof(double)));
    ML_TRY(S.Ms.ensure((size_t)T * b * b * sizeof(double)));
    ML_TRY(S.Rs.ensure((size_t)T * b * b * sizeof(double)));
    ML_TRY(S.Hrec.ensure((size_t)T * S.hstride * sizeof(double)));
    ML_TRY(S.Rrec.ensure((size_t)T * S.rstride * sizeof(double)));
    ML_TRY(S.Sd.ensure((size_t)T * ncv * kkeep * sizeof(double)));
    ML_TRY(S.layd.ensure((size_t)T * sizeof(int)));
    ML_TRY(S.flags.ensure((size_t)T * sizeof(int)));
    ML_TRY(S.G0s.ensure((size_t)T * b * b * sizeof(double)));
    ML_TRY(S.Mt.ensure((size_t)T * b * b * sizeof(double)));
    ML_TRY(S.Ajs.ensure((size_t)T * b * b * sizeof(double)));
    ML_TRY(S.dflag.ensure(sizeof(int)));
    ML_CUDA(cudaMemsetAsync(S.flags.p, 0, (size_t)T * sizeof(int), st));
    {
        const size_t smax = ((size_t)kMaxLd * kMaxLd + (size_t)kRows * (kMaxLd + 1)) * sizeof(double);
        ML_CUDA(cudaFuncSetAttribute(k_lgemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
        const size_t sdw = ((size_t)kMaxLd * kMaxLd + (size_t)kDwGemmRows * (kMaxLd + 1)) * sizeof(float2);
        ML_CUDA(cudaFuncSetAttribute(k_lgemm_dw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sdw));
    }
    S.lay.resize(T);
    for (int t = 0; t < T; ++t) S.lay[t] = t;
    ML_TRY(S.upload_lay());

    // start blocks: random, orthonormalised
    int cur = 0;
    {
        ProfScope pr("vector", st);
        k_lrandom<<<dim3(std::max(1, S.nbx * 4), S.nslots), 256, 0, st>>>(S.w(), 0, b, S.layd.as<int>(), seed, n);
    }
    ML_CUDA(cudaGetLastError());
    ML_TRY(S.orthonormalise(cur, 0, S.q(cur), 0, nullptr, nullptr));

    std::vector<std::vector<double>> Tm(T, std::vector<double>((size_t)ncv * ncv, 0.0));
    // per layer, the basis columns (0..ncv+b-1, the last b the residual block)
    // that are zero because SVQB dropped their direction (a deflated block,
    // recognised by a zero row of the step's R): the Rayleigh-Ritz step
    // leaves them out, so that they give no spurious Ritz pairs
    std::vector<std::vector<char>> dead(T, std::vector<char>((size_t)ncv + b, 0));
    std::vector<int> nconv(T, 0), matvecs(T, 0);
    std::vector<char> done(T, 0);
    std::vector<double> hrec_h, rrec_h, theta, Sv;
    int kk = 0;
    while (S.nslots > 0) {
        const int nsteps = (ncv - kk) / b;
        for (int j = 0; j < nsteps; ++j) {
            const int c = kk + j * b;
            ML_TRY(S.apply(cur, c));
            double *hr = S.Hrec.as<double>() + (int64_t)j * ldq * b;
            double *rr = S.Rrec.as<double>() + (int64_t)j * b * b;
            if (tensor)
                ML_TRY(S.orthonormalise(cur, c + b, S.q(cur), c + b, hr, rr));
            else
                ML_TRY(S.block_step(cur, c, j, hr, rr));
        }
        for (int y = 0; y < S.nslots; ++y) matvecs[S.lay[y]] += nsteps * b;
        // records of the cycle to the host
        hrec_h.resize((size_t)T * S.hstride);
        rrec_h.resize((size_t)T * S.rstride);
        ML_CUDA(cudaMemcpyAsync(hrec_h.data(), S.Hrec.p, hrec_h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        ML_CUDA(cudaMemcpyAsync(rrec_h.data(), S.Rrec.p, rrec_h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        ML_CUDA(cudaStreamSynchronize(st));
        std::vector<double> Sh((size_t)S.nslots * ncv * kkeep, 0.0);
        std::vector<std::vector<double>> th_keep(S.nslots), coup(S.nslots);
        std::vector<int> finishing;
        for (int y = 0; y < S.nslots; ++y) {
            const int t = S.lay[y];
            std::vector<double> &Tt = Tm[t];
            const double *H = hrec_h.data() + (int64_t)t * S.hstride;
            const double *R = rrec_h.data() + (int64_t)t * S.rstride;
            for (int j = 0; j < nsteps; ++j) {
                const int c = kk + j * b;
                for (int s = 0; s < b; ++s) {
                    const int col = c + s;
                    for (int r = 0; r < c + b; ++r) {
                        double v = H[(int64_t)j * ldq * b + (int64_t)r * b + s];
                        if (r < kk && c != kk) v = 0.0;   // zero by the restart structure
                        Tt[(size_t)r * ncv + col] = v;
                        Tt[(size_t)col * ncv + r] = v;
                    }
                    if (j + 1 < nsteps)
                        for (int qq = 0; qq < b; ++qq) {
                            const double v = R[(int64_t)j * b * b + qq * b + s];
                            Tt[(size_t)(c + b + qq) * ncv + col] = v;
                            Tt[(size_t)col * ncv + c + b + qq] = v;
                        }
                }
            }
            const double *Rl = R + (int64_t)(nsteps - 1) * b * b;
            std::vector<char> &dd = dead[t];
            for (int j = 0; j < nsteps; ++j)
                for (int qq = 0; qq < b; ++qq) {
                    bool zero = true;
                    for (int s2 = 0; s2 < b; ++s2) zero = zero && R[(int64_t)j * b * b + qq * b + s2] == 0.0;
                    dd[(size_t)kk + (j + 1) * b + qq] = zero ? 1 : 0;
                }
            std::vector<int> live;
            for (int i = 0; i < ncv; ++i)
                if (!dd[i]) live.push_back(i);
            const int m = (int)live.size(), nd = ncv - m;   // theta[0..nd-1]: no Ritz pair
            if (m == ncv) {
                std::vector<double> a = Tt;
                sym_eig(ncv, a, theta, Sv);
            } else {
                std::vector<double> a((size_t)m * m), thc, Sc;
                for (int r = 0; r < m; ++r)
                    for (int c2 = 0; c2 < m; ++c2) a[(size_t)r * m + c2] = Tt[(size_t)live[r] * ncv + live[c2]];
                if (m > 0) sym_eig(m, a, thc, Sc);
                theta.assign(ncv, 0.0);
                Sv.assign((size_t)ncv * ncv, 0.0);
                for (int e = 0; e < m; ++e) {
                    theta[nd + e] = thc[e];
                    for (int r = 0; r < m; ++r) Sv[(size_t)live[r] * ncv + nd + e] = Sc[(size_t)r * m + e];
                }
            }
            double tmax = 0.0;
            for (int i = nd; i < ncv; ++i) tmax = std::max(tmax, std::fabs(theta[i]));
            // coupling of each Ritz vector to the residual block: Rl * S[last block, i]
            auto coupling = [&](int col, int qq) {
                double x = 0.0;
                for (int s = 0; s < b; ++s) x += Rl[qq * b + s] * Sv[(size_t)(ncv - b + s) * ncv + col];
                return x;
            };
            int nc = 0;
            for (int i = ncv - 1; i >= ncv - k && i >= nd; --i) {
                double r2 = 0.0;
                for (int qq = 0; qq < b; ++qq) {
                    const double x = coupling(i, qq);
                    r2 += x * x;
                }
                if (std::sqrt(r2) <= tol * std::max(tmax, 1e-300)) ++nc;
                else break;
            }
            nconv[t] = nc;
            const bool fin = nc >= k || matvecs[t] >= maxit;
            if (fin) finishing.push_back(y);
            th_keep[y].resize(kkeep);
            coup[y].assign((size_t)b * kkeep, 0.0);
            std::vector<char> nextdead((size_t)ncv + b, 0);
            for (int i = 0; i < kkeep; ++i) {
                const int col = ncv - 1 - i;   // descending theta
                nextdead[i] = col < nd ? 1 : 0;   // no Ritz pair: a zero column after the restart
                th_keep[y][i] = col < nd ? 0.0 : theta[col];
                for (int c2 = 0; c2 < ncv; ++c2) Sh[((size_t)y * ncv + c2) * kkeep + i] = Sv[(size_t)c2 * ncv + col];
                for (int qq = 0; qq < b; ++qq) coup[y][(size_t)qq * kkeep + i] = coupling(col, qq);
            }
            for (int qq = 0; qq < b; ++qq) nextdead[(size_t)kkeep + qq] = dd[(size_t)ncv + qq];
            dd.swap(nextdead);
            if (fin)
                for (int i = 0; i < k; ++i)
                    evals[(size_t)t * k + i] = ncv - 1 - i < nd ? std::nan("") : 1.0 - th_keep[y][i];
        }
        // Ritz vectors of every active layer -> the other basis buffer
        ML_CUDA(cudaMemcpyAsync(S.Sd.p, Sh.data(), Sh.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        ML_TRY(S.gemm(S.q(cur), 0, ncv, S.Sd.as<double>(), S.q(cur ^ 1), 0, kkeep, false, true, "ritz"));
        {
            ProfScope pr("ritz", st);
            k_lcopy<<<dim3(std::max(1, S.nbx * 4), S.nslots), 256, 0, st>>>(S.q(cur), ncv, S.q(cur ^ 1), kkeep, b,
                                                                             S.layd.as<int>(), n);
        }
        ML_CUDA(cudaGetLastError());
        for (int y : finishing) {
            const int t = S.lay[y];
            done[t] = 1;
            if (evecs_dev) {
                double *out = evecs_dev + (int64_t)t * n * k;
                {
                    ProfScope pr("vector", st);
                    k_lcolmajor<<<(int)std::min<int64_t>((n * k + 255) / 256, sm_count() * 16), 256, 0, st>>>(S.q(cur ^ 1), t,
                                                                                                      k, n, out);
                }
                ML_CUDA(cudaGetLastError());
                ML_TRY(sign_fix_cols(out, n, k, st));
            }
        }
        // restart the others: T = diag(theta_keep) with the residual coupling
        std::vector<int> next;
        for (int y = 0; y < S.nslots; ++y) {
            const int t = S.lay[y];
            if (done[t]) continue;
            next.push_back(t);
            std::vector<double> &Tt = Tm[t];
            std::fill(Tt.begin(), Tt.end(), 0.0);
            for (int i = 0; i < kkeep; ++i) {
                Tt[(size_t)i * ncv + i] = th_keep[y][i];
                for (int qq = 0; qq < b; ++qq) {
                    const double v = coup[y][(size_t)qq * kkeep + i];
                    Tt[(size_t)(kkeep + qq) * ncv + i] = v;
                    Tt[(size_t)i * ncv + kkeep + qq] = v;
                }
            }
        }
        cur ^= 1;
        kk = kkeep;
        if (next.size() != S.lay.size()) {
            S.lay = next;
            if (!S.lay.empty()) ML_TRY(S.upload_lay());
            else S.nslots = 0;
        }
    }
    ML_CUDA(cudaStreamSynchronize(st));
    if (tensor) {
        int flags = 0;
        ML_TRY(oz_read_error(&flags, st));
        if (flags & 2) return fail(ML_ERR_TIMEOUT, "tensor-core product: a bounded wait gave up");
        if (flags & 1) return (ml_status)kRetryFp64;
    }
    int all = 1;
    for (int t = 0; t < T; ++t) {
        if (nconv_out) nconv_out[t] = std::min(nconv[t], k);
        if (nconv[t] < k) all = 0;
    }
    if (all) return ML_OK;
    std::string msg = "block Lanczos stopped at maxit " + std::to_string(maxit) + " with fewer than " +
                      std::to_string(k) + " converged pairs on layer(s)";
    for (int t = 0; t < T; ++t)
        if (nconv[t] < k) msg += " " + std::to_string(t) + " (" + std::to_string(nconv[t]) + ")";
    set_error(msg);
    return ML_WARN_NOT_CONVERGED;
}

}  // namespace ml

extern "C" ml_status ml_lanczos_eigs_layers(const ml_plan_t *layers, int T, int k, double tol, int maxit, int block,
                                            int ncv, uint64_t seed, double *evals, double *evecs, int *nconv,
                                            void *stream)
{
    using namespace ml;
    if (!layers || T < 1) return fail(ML_ERR_ARG, "layers is null or T < 1");
    for (int t = 0; t < T; ++t)
        if (!layers[t]) return fail(ML_ERR_ARG, "null layer");
    const int64_t n = layers[0]->n;
    for (int t = 1; t < T; ++t)
        if (layers[t]->n != n) return fail(ML_ERR_ARG, "layers do not share n");
    if (block < 1 || block > kMaxBlk) return fail(ML_ERR_ARG, "block must be in [1, 8]");
    if (k < 1 || k > n / 2) return fail(ML_ERR_ARG, "k must be in [1, n/2]");
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
            ML_TRY(stage.ensure((size_t)T * n * k * sizeof(double)));
            evd = stage.as<double>();
            host_out = true;
        }
    }
    if (ncv < 0 || ncv > kMaxLd - block) return fail(ML_ERR_ARG, "ncv must be 0 (automatic) or at most 96 - block");
    ml_status s = layers_impl(layers, T, k, tol, maxit, block, ncv, seed, evals, evd, nconv, st, oz_enabled());
    if ((int)s == kRetryFp64) s = layers_impl(layers, T, k, tol, maxit, block, ncv, seed, evals, evd, nconv, st, false);
    if ((s == ML_OK || s == ML_WARN_NOT_CONVERGED) && host_out)
        ML_CUDA(cudaMemcpy(evecs, evd, (size_t)T * n * k * sizeof(double), cudaMemcpyDeviceToHost));
    return s;
}
