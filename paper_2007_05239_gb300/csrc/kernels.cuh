// Device kernels of one layer's fast summation (Alg. 1, Sec. 4), templated
// on the precision T of the window/grid arithmetic, the dimension D and the
// window half-width M.
//
// Data layout (all in the plan's sorted order, see plan.cu):
//   coords   T [n][D]    local grid coordinate u of each point; the first tap
//                        of dim a is f0 = floor(u_a) - M + 1 >= 0
//   perm     int [n]     sorted position -> input index
//   dinv     double [n]  D^{-1/2} in sorted order
//   grid     T [L2][L1][L0][nv]  active grid, dim 0 fastest, vectors innermost
//   scratch  T [nsub][Pt^D][nv]  one padded tile per subproblem
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ml {

// ------------------------------------------------------------ window
// Normalised Kaiser-Bessel window phi_n(t) = sinh(b s)/s / (sinh(b m)/m),
// s = sqrt(m^2 - t^2), t in [-m, m] (grid units).  norm2 = m e^{-bm}/(1-e^{-2bm}),
// so phi_n(t) = norm2 (e^{bs} - e^{-bs}) / s.
__device__ __forceinline__ float kb_weight(float t, float m2, float b, float norm2)
{
    const float s = sqrtf(fmaxf(m2 - t * t, 0.0f));
    const float bs = b * s;
    if (bs < 1e-3f) return norm2 * 2.0f * b * (1.0f + bs * bs * (1.0f / 6.0f));
    const float e = __expf(bs);
    return norm2 * (e - __frcp_rn(e)) / s;
}
__device__ __forceinline__ double kb_weight(double t, double m2, double b, double norm2)
{
    const double s = sqrt(fmax(m2 - t * t, 0.0));
    const double bs = b * s;
    if (bs < 1e-6) return norm2 * 2.0 * b * (1.0 + bs * bs * (1.0 / 6.0));
    const double e = exp(bs);
    return norm2 * (e - 1.0 / e) / s;
}

// round-to-nearest float -> int for |x| < 2^22 by the 1.5*2^23 shift
__device__ __forceinline__ int fixed_round(float x)
{
    return __float_as_int(x + 12582912.0f) - 0x4B400000;
}

// The 2M window weights of one dimension for a point with local coordinate x
// (relative to its bin origin): taps start at o = floor(x) - M + 1 and the
// weight of tap q is phi_n(frac(x) + M - 1 - q).
template <int M>
__device__ __forceinline__ int window_row(float x, float m2, float b, float norm2, float *w)
{
    const float fl = floorf(x);
    const float fr = x - fl;
#pragma unroll
    for (int q = 0; q < 2 * M; ++q) w[q] = kb_weight(fr + (float)(M - 1 - q), m2, b, norm2);
    return (int)fl - M + 1;
}
template <int M>
__device__ __forceinline__ int window_row(double x, double m2, double b, double norm2, double *w)
{
    const double fl = floor(x);
    const double fr = x - fl;
#pragma unroll
    for (int q = 0; q < 2 * M; ++q) w[q] = kb_weight(fr + (double)(M - 1 - q), m2, b, norm2);
    return (int)fl - M + 1;
}

struct SpreadArgs {
    const int *sub_bin, *sub_start, *sub_count;
    const int *perm;
    const void *coords;      // T [n][D]
    const double *dinv;      // null: no pre-scaling
    const double *X;         // null: all-ones input
    int ldx;
    int nv;
    int B, Pt;
    int nb0, nb1;
    float m2f, bf, normf;    // window constants (FP32 copies)
    double m2d, bd, normd;   // window constants (FP64)
    void *scratch;           // T [nsub][Pt^D][nv]
};

struct FoldArgs {
    const int *bin_sub;      // nbins + 1
    const void *scratch;
    void *grid;
    int nv, B, Pt, R;
    int nb0, nb1, nb2;
    int L0, L1, L2;
};

struct InterpArgs {
    const int *sub_bin, *sub_start, *sub_count;
    const int *perm;
    const void *coords;
    const double *dinv;      // pre/post scale (normalized) or null
    const double *X;         // input (for the self term and the shift), null = ones
    int ldx;
    double *Y;
    int ldy;
    int nv;
    int B, Pt;
    int nb0, nb1;
    int L0, L1, L2;
    float m2f, bf, normf;
    double m2d, bd, normd;
    const void *grid;        // T [L2][L1][L0][nv]
    double alpha, shift, self;
    int normalized, accumulate, sorted_out;
};

template <int D>
__device__ __forceinline__ void bin_coords(int bin, int nb0, int nb1, int bc[3])
{
    bc[0] = bin % nb0;
    bc[1] = (D >= 2) ? (bin / nb0) % nb1 : 0;
    bc[2] = (D >= 3) ? bin / (nb0 * nb1) : 0;
}

template <int D>
__device__ __forceinline__ int tile_cells(int Pt)
{
    return D == 1 ? Pt : (D == 2 ? Pt * Pt : Pt * Pt * Pt);
}

// ------------------------------------------------------------ block reductions
__device__ __forceinline__ float warp_sum(float v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Scale for the fixed-point tile of one vector: a power of two with
// scale * sum|u| <= 2^30 (no cell can overflow int32, every weight is <= 1)
// and scale * max|u| <= 2^21 (every single tap is < 2^22 for fixed_round).
__device__ __forceinline__ float fixed_scale(float sum_abs, float max_abs)
{
    if (!(sum_abs > 0.0f)) return 1.0f;
    const float lim = fminf(1073741824.0f / sum_abs, 2097152.0f / fmaxf(max_abs, 1e-30f));
    int e;
    frexpf(lim, &e);                    // lim = f * 2^e, f in [0.5, 1)
    return ldexpf(1.0f, e - 1);         // largest power of two <= lim
}

// ==================================================================== spread
// FP32 form: weights and taps in FP32; each tile cell accumulates integers
// (fixed point, per-subproblem power-of-two scale) with 32-bit shared-memory
// atomics, which are exact and order-independent.  The tile is written to
// the subproblem's scratch slot as FP32.
template <int D, int M, int NV>
__global__ void __launch_bounds__(256) k_spread_f32(const SpreadArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int *tile = reinterpret_cast<int *>(smem_raw);
    __shared__ float s_part[2][NV][8];
    __shared__ float s_scale[NV];
    const int sub = blockIdx.x;
    const int bin = a.sub_bin[sub], start = a.sub_start[sub], cnt = a.sub_count[sub];
    constexpr int nv = NV;
    const int tc = tile_cells<D>(a.Pt);
    for (int e = threadIdx.x; e < tc * nv; e += blockDim.x) tile[e] = 0;

    // per-vector sum and max of |u| over this subproblem's points
    float lsum[NV], lmax[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) lsum[c] = lmax[c] = 0.0f;
    for (int i = start + threadIdx.x; i < start + cnt; i += blockDim.x) {
        const int orig = a.perm[i];
        const double ds = a.dinv ? a.dinv[i] : 1.0;
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            const float u = fabsf((float)((a.X ? a.X[(int64_t)orig * a.ldx + c] : 1.0) * ds));
            lsum[c] += u;
            lmax[c] = fmaxf(lmax[c], u);
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        const float s = warp_sum(lsum[c]), mx = warp_max(lmax[c]);
        if (lane == 0) {
            s_part[0][c][warp] = s;
            s_part[1][c][warp] = mx;
        }
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        float s = 0.0f, mx = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            s += s_part[0][threadIdx.x][w];
            mx = fmaxf(mx, s_part[1][threadIdx.x][w]);
        }
        s_scale[threadIdx.x] = fixed_scale(s, mx);
    }
    __syncthreads();

    (void)bin;
    const float *coords = static_cast<const float *>(a.coords);
    for (int i = start + threadIdx.x; i < start + cnt; i += blockDim.x) {
        const int orig = a.perm[i];
        const double ds = a.dinv ? a.dinv[i] : 1.0;
        float u[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c)
            u[c] = (float)((a.X ? a.X[(int64_t)orig * a.ldx + c] : 1.0) * ds) * s_scale[c];
        float wx[2 * M], wy[2 * M], wz[2 * M];
        int o[3] = {0, 0, 0};
        o[0] = window_row<M>(coords[(int64_t)i * D], a.m2f, a.bf, a.normf, wx);
        if (D >= 2) o[1] = window_row<M>(coords[(int64_t)i * D + 1], a.m2f, a.bf, a.normf, wy);
        if (D >= 3) o[2] = window_row<M>(coords[(int64_t)i * D + 2], a.m2f, a.bf, a.normf, wz);
        const int ny = (D >= 2) ? 2 * M : 1, nz = (D >= 3) ? 2 * M : 1;
#pragma unroll 1
        for (int qz = 0; qz < nz; ++qz) {
#pragma unroll 1
            for (int qy = 0; qy < ny; ++qy) {
                const float wyz = (D >= 3 ? wz[qz] : 1.0f) * (D >= 2 ? wy[qy] : 1.0f);
                int *row = tile + (((o[2] + qz) * a.Pt + o[1] + qy) * a.Pt + o[0]) * nv;
#pragma unroll
                for (int qx = 0; qx < 2 * M; ++qx) {
                    const float wt = wyz * wx[qx];
#pragma unroll
                    for (int c = 0; c < NV; ++c) atomicAdd(row + qx * nv + c, fixed_round(u[c] * wt));
                }
            }
        }
    }
    __syncthreads();
    float *out = static_cast<float *>(a.scratch) + (int64_t)sub * tc * nv;
    for (int e = threadIdx.x; e < tc * nv; e += blockDim.x) out[e] = (float)tile[e] / s_scale[e % nv];
}

// FP64 form: weights, taps and the tile in FP64 (shared-memory FP64 atomics).
template <int D, int M, int NV>
__global__ void __launch_bounds__(256) k_spread_f64(const SpreadArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *tile = reinterpret_cast<double *>(smem_raw);
    const int sub = blockIdx.x;
    const int bin = a.sub_bin[sub], start = a.sub_start[sub], cnt = a.sub_count[sub];
    constexpr int nv = NV;
    const int tc = tile_cells<D>(a.Pt);
    for (int e = threadIdx.x; e < tc * nv; e += blockDim.x) tile[e] = 0.0;
    __syncthreads();
    (void)bin;
    const double *coords = static_cast<const double *>(a.coords);
    for (int i = start + threadIdx.x; i < start + cnt; i += blockDim.x) {
        const int orig = a.perm[i];
        const double ds = a.dinv ? a.dinv[i] : 1.0;
        double u[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) u[c] = (a.X ? a.X[(int64_t)orig * a.ldx + c] : 1.0) * ds;
        double wx[2 * M], wy[2 * M], wz[2 * M];
        int o[3] = {0, 0, 0};
        o[0] = window_row<M>(coords[(int64_t)i * D], a.m2d, a.bd, a.normd, wx);
        if (D >= 2) o[1] = window_row<M>(coords[(int64_t)i * D + 1], a.m2d, a.bd, a.normd, wy);
        if (D >= 3) o[2] = window_row<M>(coords[(int64_t)i * D + 2], a.m2d, a.bd, a.normd, wz);
        const int ny = (D >= 2) ? 2 * M : 1, nz = (D >= 3) ? 2 * M : 1;
#pragma unroll 1
        for (int qz = 0; qz < nz; ++qz) {
#pragma unroll 1
            for (int qy = 0; qy < ny; ++qy) {
                const double wyz = (D >= 3 ? wz[qz] : 1.0) * (D >= 2 ? wy[qy] : 1.0);
                double *row = tile + (((o[2] + qz) * a.Pt + o[1] + qy) * a.Pt + o[0]) * nv;
#pragma unroll
                for (int qx = 0; qx < 2 * M; ++qx) {
                    const double wt = wyz * wx[qx];
#pragma unroll
                    for (int c = 0; c < NV; ++c) atomicAdd(row + qx * nv + c, u[c] * wt);
                }
            }
        }
    }
    __syncthreads();
    double *out = static_cast<double *>(a.scratch) + (int64_t)sub * tc * nv;
    for (int e = threadIdx.x; e < tc * nv; e += blockDim.x) out[e] = tile[e];
}

// ==================================================================== fold
// One CTA per bin: each active-grid cell of the bin sums, in a fixed order,
// the tile values of every subproblem whose padded tile covers it (the bin
// itself and up to R bins below it per dim).  Deterministic, no atomics.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_fold(const FoldArgs a)
{
    const int bin = blockIdx.x;
    int bc[3];
    bin_coords<D>(bin, a.nb0, a.nb1, bc);
    const int B = a.B, Pt = a.Pt, nv = a.nv;
    const int tc = tile_cells<D>(Pt);
    const int cells = (D == 1 ? B : (D == 2 ? B * B : B * B * B));
    const T *scr = static_cast<const T *>(a.scratch);
    T *grid = static_cast<T *>(a.grid);
    for (int e = threadIdx.x; e < cells * nv; e += blockDim.x) {
        const int c = e % nv;
        const int cell = e / nv;
        const int cx = cell % B;
        const int cy = (D >= 2) ? (cell / B) % B : 0;
        const int cz = (D >= 3) ? cell / (B * B) : 0;
        const int gx = bc[0] * B + cx, gy = bc[1] * B + cy, gz = bc[2] * B + cz;
        if (gx >= a.L0 || gy >= a.L1 || gz >= a.L2) continue;
        T acc = 0;
        const int zlo = (D >= 3) ? max(0, bc[2] - a.R) : 0;
        const int ylo = (D >= 2) ? max(0, bc[1] - a.R) : 0;
        const int xlo = max(0, bc[0] - a.R);
        for (int nz = zlo; nz <= bc[2]; ++nz) {
            const int oz = gz - nz * B;
            if (oz >= Pt) continue;
            for (int ny = ylo; ny <= bc[1]; ++ny) {
                const int oy = gy - ny * B;
                if (oy >= Pt) continue;
                for (int nx = xlo; nx <= bc[0]; ++nx) {
                    const int ox = gx - nx * B;
                    if (ox >= Pt) continue;
                    const int nbin = (nz * a.nb1 + ny) * a.nb0 + nx;
                    const int s0 = a.bin_sub[nbin], s1 = a.bin_sub[nbin + 1];
                    const int64_t off = (int64_t)((oz * Pt + oy) * Pt + ox) * nv + c;
                    for (int s = s0; s < s1; ++s) acc += scr[(int64_t)s * tc * nv + off];
                }
            }
        }
        grid[((int64_t)(gz * a.L1 + gy) * a.L0 + gx) * nv + c] = acc;
    }
}

// ==================================================================== axis
// out[(a*Ko + k)*C + c] = sum_j M[k*J + j] * in[(a*J + j)*C + c]
// (one real trigonometric transform along the middle index).  Tiles of
// 32 k x 64 flattened (a, c) pairs; 256 threads, 8 outputs each.
template <typename T>
__global__ void __launch_bounds__(256) k_axis(const T *__restrict__ in, T *__restrict__ out,
                                              const T *__restrict__ M, int A, int J, int Ko, int C)
{
    __shared__ T Ms[32][33];
    __shared__ T Is[32][65];
    const int64_t P = (int64_t)A * C;
    const int64_t p0 = (int64_t)blockIdx.x * 64;
    const int k0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = 0;
    for (int j0 = 0; j0 < J; j0 += 32) {
        for (int e = threadIdx.x; e < 32 * 32; e += 256) {
            const int kk = e >> 5, jj = e & 31;
            Ms[jj][kk] = (k0 + kk < Ko && j0 + jj < J) ? M[(int64_t)(k0 + kk) * J + j0 + jj] : (T)0;
        }
        for (int e = threadIdx.x; e < 32 * 64; e += 256) {
            int jj, pp;
            if (C >= 16) { jj = e >> 6; pp = e & 63; }
            else { pp = e >> 5; jj = e & 31; }
            const int64_t p = p0 + pp;
            T v = 0;
            if (p < P && j0 + jj < J) {
                const int64_t aa = p / C;
                const int cc = (int)(p - aa * C);
                v = in[(aa * J + j0 + jj) * C + cc];
            }
            Is[jj][pp] = v;
        }
        __syncthreads();
#pragma unroll 8
        for (int jj = 0; jj < 32; ++jj) {
            const T m0 = Ms[jj][ty * 2], m1 = Ms[jj][ty * 2 + 1];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const T x = Is[jj][tx + 16 * q];
                acc[0][q] += m0 * x;
                acc[1][q] += m1 * x;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int k = k0 + ty * 2 + i;
        if (k >= Ko) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t p = p0 + tx + 16 * q;
            if (p >= P) continue;
            const int64_t aa = p / C;
            const int cc = (int)(p - aa * C);
            out[(aa * Ko + k) * C + cc] = acc[i][q];
        }
    }
}

template <typename T>
__global__ void k_mult(T *coef, const T *__restrict__ mult, int64_t slots, int nv)
{
    const int64_t tot = slots * nv;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x)
        coef[e] *= mult[e / nv];
}

// ==================================================================== interp
// One CTA per subproblem: the bin's padded tile of the convolved grid is
// loaded into shared memory, each point sums its (2M)^D taps, and the FP64
// epilogue forms  alpha * D^{-1/2} * (sum - K(0) u) (+ shift * x)  in input
// order (or the raw sum minus the self term in sorted order for degrees).
template <typename T, int D, int M, int NV>
__global__ void __launch_bounds__(256) k_interp(const InterpArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tile = reinterpret_cast<T *>(smem_raw);
    const int sub = blockIdx.x;
    const int bin = a.sub_bin[sub], start = a.sub_start[sub], cnt = a.sub_count[sub];
    constexpr int nv = NV;
    const int Pt = a.Pt;
    const int tc = tile_cells<D>(Pt);
    int bc[3];
    bin_coords<D>(bin, a.nb0, a.nb1, bc);
    const T *grid = static_cast<const T *>(a.grid);
    for (int e = threadIdx.x; e < tc * nv; e += blockDim.x) {
        const int c = e % nv;
        const int cell = e / nv;
        const int lx = cell % Pt;
        const int ly = (D >= 2) ? (cell / Pt) % Pt : 0;
        const int lz = (D >= 3) ? cell / (Pt * Pt) : 0;
        const int gx = bc[0] * a.B + lx, gy = bc[1] * a.B + ly, gz = bc[2] * a.B + lz;
        T v = 0;
        if (gx < a.L0 && gy < a.L1 && gz < a.L2) v = grid[((int64_t)(gz * a.L1 + gy) * a.L0 + gx) * nv + c];
        tile[e] = v;
    }
    __syncthreads();
    const T *coords = static_cast<const T *>(a.coords);
    for (int i = start + threadIdx.x; i < start + cnt; i += blockDim.x) {
        T wx[2 * M], wy[2 * M], wz[2 * M];
        int o[3] = {0, 0, 0};
        if (sizeof(T) == 4) {
            o[0] = window_row<M>((float)coords[(int64_t)i * D], a.m2f, a.bf, a.normf, (float *)wx);
            if (D >= 2) o[1] = window_row<M>((float)coords[(int64_t)i * D + 1], a.m2f, a.bf, a.normf, (float *)wy);
            if (D >= 3) o[2] = window_row<M>((float)coords[(int64_t)i * D + 2], a.m2f, a.bf, a.normf, (float *)wz);
        } else {
            o[0] = window_row<M>((double)coords[(int64_t)i * D], a.m2d, a.bd, a.normd, (double *)wx);
            if (D >= 2) o[1] = window_row<M>((double)coords[(int64_t)i * D + 1], a.m2d, a.bd, a.normd, (double *)wy);
            if (D >= 3) o[2] = window_row<M>((double)coords[(int64_t)i * D + 2], a.m2d, a.bd, a.normd, (double *)wz);
        }
        T acc[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) acc[c] = 0;
        const int ny = (D >= 2) ? 2 * M : 1, nz = (D >= 3) ? 2 * M : 1;
#pragma unroll 1
        for (int qz = 0; qz < nz; ++qz) {
            T pz[NV];
#pragma unroll
            for (int c = 0; c < NV; ++c) pz[c] = 0;
#pragma unroll 1
            for (int qy = 0; qy < ny; ++qy) {
                const T *row = tile + (((o[2] + qz) * Pt + o[1] + qy) * Pt + o[0]) * nv;
                T r[NV];
#pragma unroll
                for (int c = 0; c < NV; ++c) r[c] = 0;
#pragma unroll
                for (int qx = 0; qx < 2 * M; ++qx)
#pragma unroll
                    for (int c = 0; c < NV; ++c) r[c] += wx[qx] * row[qx * nv + c];
                const T wyq = (D >= 2) ? wy[qy] : (T)1;
#pragma unroll
                for (int c = 0; c < NV; ++c) pz[c] += wyq * r[c];
            }
            const T wzq = (D >= 3) ? wz[qz] : (T)1;
#pragma unroll
            for (int c = 0; c < NV; ++c) acc[c] += wzq * pz[c];
        }
        const int orig = a.perm[i];
        const double ds = a.dinv ? a.dinv[i] : 1.0;
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            const double x = a.X ? a.X[(int64_t)orig * a.ldx + c] : 1.0;
            const double u = x * ds;
            const double r = (double)acc[c] - a.self * u;
            if (a.sorted_out) {
                a.Y[(int64_t)i * a.ldy + c] = r;
            } else {
                double outv = a.alpha * ds * r + a.shift * x;
                double *yp = a.Y + (int64_t)orig * a.ldy + c;
                if (a.accumulate) outv += *yp;
                *yp = outv;
            }
        }
    }
}

}  // namespace ml
