// Device kernels of one layer's fast summation (Alg. 1, Sec. 4), templated
// on the precision T of the window/grid arithmetic, the dimension D and the
// window width W (taps per dimension).
//
// Data layout (all in the plan's sorted order, see plan.cu):
//   coords   T [n][D]    local grid coordinate u of each point; the first tap
//                        of dim a is floor(u_a - W/2) + 1 >= 0
//   perm     int [n]     sorted position -> input index
//   dinv     double [n]  D^{-1/2} in sorted order
//   grid     T [L2][L1][L0][nv]  active grid, dim 0 fastest, vectors innermost
//   scratch  T [nsub][Pt^D][nv]  one padded tile per subproblem
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ml {

// FP32 window weights by polynomials (plan-time fit, see window_row_poly):
// up to kPolyW taps per dimension, degree kPolyTerms - 1 in u, the even and
// odd coefficients of each of the first ceil(W/2) taps in a row of
// kPolyStride floats (16-byte aligned, zero padded; the other taps mirror them)
constexpr int kPolyW = 16;
constexpr int kPolyTerms = 10;
constexpr int kPolyStride = 12;
// shared memory for an FP32 spreading tile plus its row-product slots
constexpr size_t kRowSpreadBudget = 220 * 1024;


// ------------------------------------------------------------ window
// Normalised Kaiser-Bessel window phi_n(t) = sinh(b s)/s / (sinh(b m)/m),
// s = sqrt(m^2 - t^2), t in [-m, m] (grid units).  norm2 = m e^{-bm}/(1-e^{-2bm}),
// so phi_n(t) = norm2 (e^{bs} - e^{-bs}) / s.
// (the FP32 form evaluates it through plan-time polynomials, window_row_poly;
// the FP64 form tabulates it at plan time with this FP64 version)
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

// ------------------------------------------------------------ double-word
// The FP64 form runs its taps on the FP32 pipes (GB300 issues FP64 at about
// 1/60 of the FP32 rate).  A value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2 (about 48 significant bits).  Products use
// the FMA-based exact product (p + e = a*b exactly for floats a, b); sums the
// exact two-sum of Knuth (the "double-word" algorithms of Dekker 1971 and
// Joldes, Muller and Popescu 2017; the dot-product accumulation follows
// Dot2 of Ogita, Rump and Oishi 2005).  The _rn intrinsics keep the compiler
// from contracting these steps into FMAs.
__device__ __forceinline__ float2 dw_split(double x)
{
    const float hi = __double2float_rn(x);
    return make_float2(hi, __double2float_rn(x - (double)hi));
}
__device__ __forceinline__ double dw_value(float2 x)
{
    return (double)x.x + (double)x.y;
}
// x * y with a relative error of a few units of 2^-48
__device__ __forceinline__ float2 dw_mul(float2 x, float2 y)
{
    const float ph = __fmul_rn(x.x, y.x);
    float pl = fmaf(x.x, y.x, -ph);
    pl = fmaf(x.x, y.y, pl);
    pl = fmaf(x.y, y.x, pl);
    const float h = __fadd_rn(ph, pl);
    return make_float2(h, __fsub_rn(pl, __fsub_rn(h, ph)));
}
// s += g * w with s left unnormalised (s.y collects the rounding errors of
// the running sum and of the products; renormalise with dw_norm)
__device__ __forceinline__ void dw_fma_acc(float2 &s, float2 g, float2 w)
{
    const float p = __fmul_rn(g.x, w.x);
    float e = fmaf(g.x, w.x, -p);
    e = fmaf(g.x, w.y, e);
    e = fmaf(g.y, w.x, e);
    const float t = __fadd_rn(s.x, p);
    const float bb = __fsub_rn(t, s.x);
    const float err = __fadd_rn(__fsub_rn(s.x, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    s.y = __fadd_rn(s.y, __fadd_rn(err, e));
    s.x = t;
}
// s += x (x a double-word value), s left unnormalised
__device__ __forceinline__ void dw_acc(float2 &s, float2 x)
{
    const float t = __fadd_rn(s.x, x.x);
    const float bb = __fsub_rn(t, s.x);
    const float err = __fadd_rn(__fsub_rn(s.x, __fsub_rn(t, bb)), __fsub_rn(x.x, bb));
    s.y = __fadd_rn(s.y, __fadd_rn(err, x.y));
    s.x = t;
}
__device__ __forceinline__ float2 dw_norm(float2 s)
{
    const float h = __fadd_rn(s.x, s.y);
    return make_float2(h, __fsub_rn(s.y, __fsub_rn(h, s.x)));
}
// Fixed point of one tap p + e (p the rounded product, e its error) for
// |p| < 2^22: hi = round(p), lo = round((p - hi + e) * 2^20); the tap is
// hi + lo * 2^-20 to within 2^-21 + 2^-25.
__device__ __forceinline__ void fixed_split(float p, float e, int &hi, int &lo)
{
    const float t = __fadd_rn(p, 12582912.0f);
    hi = __float_as_int(t) - 0x4B400000;
    const float r = __fadd_rn(__fsub_rn(p, __fsub_rn(t, 12582912.0f)), e);
    lo = __float_as_int(fmaf(r, 1048576.0f, 12582912.0f)) - 0x4B400000;
}

// The W window weights of one dimension for a point with local coordinate x
// (relative to its bin origin): the taps are the W cells nearest to x, the
// first at o = floor(x - W/2) + 1, and the weight of tap q is
// phi_n(x - o - q), |x - o - q| <= W/2.  FP32 form, from polynomials fitted
// at plan time: with
// f = (x - W/2) - floor(x - W/2) in [0, 1) and u = f - 1/2, tap q has weight
// phi_n(W/2 - 1 - q + f) ~ p_q(u), a polynomial of degree 9 (Chebyshev
// interpolation of the window on each unit interval; the fit error is below
// 1e-7 of the window's peak for every W and oversampling the plans allow,
// checked at plan time).  The window is even, so tap W-1-q sees the mirror
// image of tap q: p_{W-1-q}(u) = p_q(-u).  Writing p_q(u) = E_q(u^2) +
// u O_q(u^2), the pair costs two Horner chains of degree 4 in u^2 and two
// FMAs (the middle tap of an odd W is even: E only) -- 25 FMAs for W = 5 in
// place of 45 for ten-term Horner per tap, and no exponential, square root or
// reciprocal on the special-function unit (whose fast exponential errs by
// about 1e-6 near the window's centre).  Row q < ceil(W/2) of c holds
// e_0..e_4 (coefficients of u^0, u^2, .., u^8), then o_0..o_4 (u^1, u^3, ..,
// u^9), then two zeros.  c: kernel parameters (single-layer launches) or a
// shared copy.
template <int W>
__device__ __forceinline__ int window_row_poly(float x, const float *__restrict__ c, float *w)
{
    const float xs = x - 0.5f * (float)W;
    const float fl = floorf(xs);
    const float u = (xs - fl) - 0.5f;
    const float u2 = u * u;
#pragma unroll
    for (int q = 0; q < (W + 1) / 2; ++q) {
        const float4 *row = reinterpret_cast<const float4 *>(c + q * kPolyStride);
        const float4 c0 = row[0], c1 = row[1], c2 = row[2];
        float e = fmaf(c1.x, u2, c0.w);
        e = fmaf(e, u2, c0.z);
        e = fmaf(e, u2, c0.y);
        e = fmaf(e, u2, c0.x);
        if (2 * q + 1 == W) {
            w[q] = e;
        } else {
            float o = fmaf(c2.y, u2, c2.x);
            o = fmaf(o, u2, c1.w);
            o = fmaf(o, u2, c1.z);
            o = fmaf(o, u2, c1.y);
            w[q] = fmaf(u, o, e);
            w[W - 1 - q] = fmaf(-u, o, e);
        }
    }
    return (int)fl + 1;
}
static_assert(kPolyTerms == 10 && kPolyStride == 12, "window_row_poly evaluates degree 9 from 12-float rows");

// coefficients of a batched launch's layer copied to shared memory (the
// caller synchronises before they are read)
__device__ __forceinline__ void stage_window_poly(const float *__restrict__ src, float *dst, int W)
{
    for (int e = threadIdx.x; e < (W + 1) / 2 * kPolyStride; e += blockDim.x) dst[e] = src[e];
}


struct SpreadArgs {
    const int *sub_bin, *sub_start, *sub_count;
    const int *perm;
    const int *sidx;         // null, or the spreading order of the sorted positions (one-tile FP32 layers)
    const void *coords;      // T [n][D]
    const float2 *wts;       // FP64 form: window weights [n][D][W] as double-word pairs
    const int *offs;         // FP64 form: first tap per dim, packed o0 | o1 << 10 | o2 << 20
    const double *dinv;      // null: no pre-scaling
    const double *X;         // null: all-ones input
    int ldx;
    int nv;
    int B, Pt;
    int nb0, nb1;
    float m2f, bf, normf;    // window constants (FP32 copies)
    double m2d, bd, normd;   // window constants (FP64)
    void *scratch;           // T [nsub][Pt^D][nv]
    int sub_max;             // largest subproblem (smem staging size)
    int nsub;                // subproblems (batched launches)
    int rows_off;            // FP32, D = 3: byte offset of the row-product slots in dynamic shared
                             // memory (RowSpread), 0 = not used
    int stage_off;           // FP32: byte offset of the staged points (sub_max x nv values u, then,
                             // with sidx, sub_max sorted indices) in dynamic shared memory, 0 = not staged
    int4 *sub_box;           // FP32: null (whole tiles written), or per subproblem the box of tile
                             // cells its taps reach (pack_box); only that box of its tile is written
    alignas(16) float kbp[kPolyW * kPolyStride];   // FP32 window polynomials (window_row_poly)
};

// most subproblem tiles per group of k_group_sum_box
constexpr int kGroupSubsMax = 64;

// Box of tile cells [lo_a, hi_a) per axis a, packed lo | hi << 16 per int
// (tile edges are below 2^16); an empty box has hi = lo on an axis
__device__ __forceinline__ int4 pack_box(const int lo[3], const int hi[3])
{
    return make_int4(lo[0] | (hi[0] << 16), lo[1] | (hi[1] << 16), lo[2] | (hi[2] << 16), 0);
}

// Sum of the tiles of each group of consecutive subproblems of one bin
// (fixed order): gtile[g] = sum_{s in group g} scratch[s].  CTA b handles
// group b / chunks and the tile chunk b % chunks (flattened so that the
// group count is not limited by gridDim.y).
template <typename T>
__global__ void __launch_bounds__(256) k_group_sum(const T *__restrict__ scratch, const int *__restrict__ grp_sub,
                                                  int64_t tile_elems, int chunks, T *gtile)
{
    const int g = blockIdx.x / chunks;
    const int ch = blockIdx.x - g * chunks;
    const int s0 = grp_sub[g], s1 = grp_sub[g + 1];
    for (int64_t e = ch * (int64_t)blockDim.x + threadIdx.x; e < tile_elems; e += (int64_t)chunks * blockDim.x) {
        T acc = 0;
        for (int s = s0; s < s1; ++s) acc += scratch[(int64_t)s * tile_elems + e];
        gtile[(int64_t)g * tile_elems + e] = acc;
    }
}

struct GroupArgs {
    const void *scratch;
    const int *grp_sub;
    int64_t tile_elems;
    void *gtile;
    int ngroups;
};

// batched: blockIdx.y is the layer, blockIdx.x = group * chunks + chunk
template <typename T>
__global__ void __launch_bounds__(256) k_group_sum_batch(const GroupArgs *__restrict__ args, int chunks)
{
    const GroupArgs a = args[blockIdx.y];
    const int g = blockIdx.x / chunks;
    const int ch = blockIdx.x - g * chunks;
    if (g >= a.ngroups) return;
    const T *scratch = static_cast<const T *>(a.scratch);
    T *gtile = static_cast<T *>(a.gtile);
    const int s0 = a.grp_sub[g], s1 = a.grp_sub[g + 1];
    for (int64_t e = ch * (int64_t)blockDim.x + threadIdx.x; e < a.tile_elems; e += (int64_t)chunks * blockDim.x) {
        T acc = 0;
        for (int s = s0; s < s1; ++s) acc += scratch[(int64_t)s * a.tile_elems + e];
        gtile[(int64_t)g * a.tile_elems + e] = acc;
    }
}

struct FoldArgs {
    int nbins;               // bins (batched launches)
    const int *bin_sub;      // nbins + 1 (first tile of each bin: subproblem or group)
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
    const float2 *wts;       // FP64 form: window weights [n][D][W] as double-word pairs
    const int *offs;         // FP64 form: packed first taps
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
    int sorted_final;        // the finished value at the sorted position (no accumulation)
    int nsub;                // subproblems (batched launches)
    alignas(16) float kbp[kPolyW * kPolyStride];   // FP32 window polynomials (window_row_poly)
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

// Division by a divisor that is fixed for a whole block: q = x / d by one
// multiply-high with m = floor((2^32 - 1) / d) + 1.  Exact for d >= 2 and
// 0 <= x < 2^32 / d: m d = 2^32 + e with 0 <= e < d, so x m / 2^32 exceeds
// x / d by x e / (d 2^32) < 1 / d, which cannot reach the next multiple of
// 1/d above x / d.  d = 1 returns x.
struct FastDiv {
    uint32_t d, m;
    __device__ __forceinline__ explicit FastDiv(int div) : d((uint32_t)div), m(0xFFFFFFFFu / (uint32_t)div + 1u) {}
    __device__ __forceinline__ int div(int x) const { return d == 1u ? x : (int)__umulhi((uint32_t)x, m); }
};

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
// Shared-memory tiles are vector-major: tile[c * tc + cell], so that the NV
// values of one tap fall in different banks.

// Sum over the warp of 32 values per lane: after five exchange rounds lane l
// holds the sum of every lane's v[l] (a fixed order: deterministic).
__device__ __forceinline__ float warp_transpose_sum32(float (&v)[32], int lane)
{
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const int h = 16 >> r;
        const bool up = (lane & h) != 0;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const float send = up ? v[k] : v[k + h];
            const float keep = up ? v[k + h] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, h);
        }
    }
    return v[0];
}

// The warp's 32 points share their first tap o: every tap t (and vector c) is
// summed over the warp in chunks of 32 taps, and lane l adds the sum of tap
// 32 j + l of chunk j, rounded to the fixed-point integer (the scaled sum of
// a subproblem stays below 2^30), with one atomic.  Lanes past the end of the
// subproblem carry u = 0.
template <int D, int W, int NV>
__device__ __forceinline__ void warp_spread_sum(int *tile, int tc, int Pt, const int (&o)[3], const float (&u)[NV],
                                                const float (&wx)[W], const float (&wy)[W], const float (&wz)[W],
                                                int lane)
{
    constexpr int ny = (D >= 2) ? W : 1, nz = (D >= 3) ? W : 1;
    constexpr int NT = W * ny * nz;
    float wzy[nz * ny];
#pragma unroll
    for (int qz = 0; qz < nz; ++qz)
#pragma unroll
        for (int qy = 0; qy < ny; ++qy) wzy[qz * ny + qy] = (D >= 3 ? wz[qz] : 1.0f) * (D >= 2 ? wy[qy] : 1.0f);
#pragma unroll 1
    for (int c = 0; c < NV; ++c) {
        float uc = u[0];
#pragma unroll
        for (int k = 1; k < NV; ++k)
            if (c == k) uc = u[k];
        float uw[W];
#pragma unroll
        for (int qx = 0; qx < W; ++qx) uw[qx] = uc * wx[qx];
#pragma unroll
        for (int j = 0; j < (NT + 31) / 32; ++j) {
            float v[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const int t = 32 * j + k;
                v[k] = t < NT ? wzy[t / W] * uw[t % W] : 0.0f;
            }
            const float sum = warp_transpose_sum32(v, lane);
            const int t = 32 * j + lane;
            if (t < NT) {
                const int qx = t % W, qy = (t / W) % ny, qz = t / (W * ny);
                atomicAdd(tile + c * tc + ((o[2] + qz) * Pt + o[1] + qy) * Pt + o[0] + qx, __float2int_rn(sum));
            }
        }
    }
}

// Row-product spreading (D = 3).  When the warp's 32 points share their first
// tap o, the tap sums S_c[qz][qy][qx] = sum_p u_pc wz_p[qz] wy_p[qy] wx_p[qx]
// are products of small matrices: lane l owns the rows r = l, l + 32, ...
// (r = qz W + qy) and adds, for p = 0..31 in order, wx_p[qx] times
// (u_pc (wy_p[qy] wz_p[qz])) to its accumulators (W per vector c).  Each lane
// first writes its point's slot in the warp's shared region: wx and u (read
// by all lanes alike: broadcasts, 16 bytes at a time), then wy and wz (W
// distinct words each).  One atomic per row, qx and vector, with the sum
// rounded to the fixed-point integer (the scaled sum of a subproblem stays
// below 2^30).  The arithmetic per vector does not depend on the number of
// vectors in the pass, so passes of any width give the same bits.  About 11
// instructions per point and row group for one vector, against a transpose
// of the 32 lanes' tap values (5 exchange rounds per 32 taps) in
// warp_spread_sum.  (Storing the W^2 products wy wz instead would save one
// load and one multiply per point but nearly double the slots, which then
// cost a resident block per SM.)
__host__ __device__ constexpr int row_slot_head(int W, int NV) { return (W + NV + 3) / 4 * 4; }
// floats per point, padded to 4 (mod 8) so that the lanes' 16-byte slot
// stores fall on distinct bank groups
__host__ __device__ constexpr int pad_slot(int f) { return ((f + 3) / 4 * 4) % 8 == 0 ? (f + 3) / 4 * 4 + 4 : (f + 3) / 4 * 4; }
__host__ __device__ constexpr int row_slot_floats(int W, int NV) { return pad_slot(row_slot_head(W, NV) + 2 * W); }
// d = 2 (warp_spread_taps): wx, wy, padding, u
__host__ __device__ constexpr int tap_slot_u0(int W) { return (2 * W + 3) / 4 * 4; }
__host__ __device__ constexpr int tap_slot_floats(int W, int NV) { return pad_slot(tap_slot_u0(W) + NV); }
// whether warps whose points share a first tap use the shared slots (d = 3:
// row products, d = 2: one tap per lane), and the bytes of the slots of a
// 256-thread block (8 warps of 32 points)
__host__ __device__ constexpr bool warp_slots_on(int D, int W) { return (D == 3 && W <= 8) || (D == 2 && W * W <= 64); }
__host__ __device__ constexpr size_t warp_slot_bytes(int D, int W, int NV)
{
    return !warp_slots_on(D, W) ? 0
                                : (size_t)8 * 32 * (D == 3 ? row_slot_floats(W, NV) : tap_slot_floats(W, NV)) * sizeof(float);
}
template <int D, int W, int NV>
struct RowSpread {
    static constexpr bool on = warp_slots_on(D, W);
    static constexpr int S = D == 3 ? row_slot_floats(W, NV) : tap_slot_floats(W, NV);
    static constexpr int warp_floats = 32 * S;
    static constexpr size_t smem = warp_slot_bytes(D, W, NV);
};

template <int W, int NV>
__device__ __forceinline__ void warp_spread_rows(int *tile, int tc, int Pt, const int (&o)[3], const float (&u)[NV],
                                                 const float (&wx)[W], const float (&wy)[W], const float (&wz)[W],
                                                 float *slots, int lane)
{
    constexpr int S = row_slot_floats(W, NV);
    constexpr int H = row_slot_head(W, NV);     // wx, u, padding; then wy, wz
    constexpr int R = W * W;
    {
        float v[S];
#pragma unroll
        for (int q = 0; q < W; ++q) v[q] = wx[q];
#pragma unroll
        for (int c = 0; c < NV; ++c) v[W + c] = u[c];
#pragma unroll
        for (int q = W + NV; q < H; ++q) v[q] = 0.0f;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            v[H + q] = wy[q];
            v[H + W + q] = wz[q];
        }
#pragma unroll
        for (int q = H + 2 * W; q < S; ++q) v[q] = 0.0f;
        float4 *dst = reinterpret_cast<float4 *>(slots + lane * S);
#pragma unroll
        for (int k = 0; k < S / 4; ++k) dst[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    }
    __syncwarp();
#pragma unroll 1
    for (int r0 = 0; r0 < R; r0 += 32) {
        const int r = r0 + lane;
        const int rr = r < R ? r : R - 1;
        const int qz = rr / W, qy = rr - qz * W;
        float acc[NV][W];
#pragma unroll
        for (int c = 0; c < NV; ++c)
#pragma unroll
            for (int qx = 0; qx < W; ++qx) acc[c][qx] = 0.0f;
#pragma unroll 4
        for (int p = 0; p < 32; ++p) {
            const float *sp = slots + p * S;
            float h[H];
#pragma unroll
            for (int k = 0; k < H; k += 4) {
                const float4 t = *reinterpret_cast<const float4 *>(sp + k);
                h[k] = t.x;
                h[k + 1] = t.y;
                h[k + 2] = t.z;
                h[k + 3] = t.w;
            }
            const float b = sp[H + qy] * sp[H + W + qz];
#pragma unroll
            for (int c = 0; c < NV; ++c) {
                const float ub = h[W + c] * b;
#pragma unroll
                for (int qx = 0; qx < W; ++qx) acc[c][qx] = fmaf(h[qx], ub, acc[c][qx]);
            }
        }
        if (r < R) {
            int *row = tile + ((o[2] + qz) * Pt + o[1] + qy) * Pt + o[0];
#pragma unroll
            for (int c = 0; c < NV; ++c)
#pragma unroll
                for (int qx = 0; qx < W; ++qx) atomicAdd(row + c * tc + qx, __float2int_rn(acc[c][qx]));
        }
    }
    __syncwarp();   // the slots are rewritten by the next group
}

// d = 2 counterpart of warp_spread_rows: the warp's 32 points share their
// first tap, lane l owns the taps t = l, l + 32, ... (t = qy W + qx) and
// adds, for p = 0..31 in order, u_pc (wx_p[qx] wy_p[qy]) to its
// accumulator of vector c.  The slots hold wx and wy (W distinct words each)
// and u (broadcast, 16 bytes at a time).  One atomic per tap and vector;
// the arithmetic per vector does not depend on the pass width.
template <int W, int NV>
__device__ __forceinline__ void warp_spread_taps(int *tile, int tc, int Pt, const int (&o)[3], const float (&u)[NV],
                                                 const float (&wx)[W], const float (&wy)[W], float *slots, int lane)
{
    constexpr int S = tap_slot_floats(W, NV);
    constexpr int U0 = tap_slot_u0(W);
    constexpr int NT = W * W;
    constexpr int NU = (NV + 3) / 4 * 4;
    {
        float v[S];
#pragma unroll
        for (int q = 0; q < W; ++q) {
            v[q] = wx[q];
            v[W + q] = wy[q];
        }
#pragma unroll
        for (int q = 2 * W; q < U0; ++q) v[q] = 0.0f;
#pragma unroll
        for (int c = 0; c < NV; ++c) v[U0 + c] = u[c];
#pragma unroll
        for (int q = U0 + NV; q < S; ++q) v[q] = 0.0f;
        float4 *dst = reinterpret_cast<float4 *>(slots + lane * S);
#pragma unroll
        for (int k = 0; k < S / 4; ++k) dst[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    }
    __syncwarp();
#pragma unroll 1
    for (int t0 = 0; t0 < NT; t0 += 32) {
        const int t = t0 + lane;
        const int tt = t < NT ? t : NT - 1;
        const int qy = tt / W, qx = tt - qy * W;
        float acc[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) acc[c] = 0.0f;
#pragma unroll 4
        for (int p = 0; p < 32; ++p) {
            const float *sp = slots + p * S;
            const float b = sp[qx] * sp[W + qy];
            float uu[NU];
#pragma unroll
            for (int k = 0; k < NU; k += 4) {
                const float4 q4 = *reinterpret_cast<const float4 *>(sp + U0 + k);
                uu[k] = q4.x;
                uu[k + 1] = q4.y;
                uu[k + 2] = q4.z;
                uu[k + 3] = q4.w;
            }
#pragma unroll
            for (int c = 0; c < NV; ++c) acc[c] = fmaf(uu[c], b, acc[c]);
        }
        if (t < NT) {
            int *cell = tile + (o[1] + qy) * Pt + o[0] + qx;
#pragma unroll
            for (int c = 0; c < NV; ++c) atomicAdd(cell + c * tc, __float2int_rn(acc[c]));
        }
    }
    __syncwarp();   // the slots are rewritten by the next group
}

// FP32 form: one thread per point.  Weights and taps in FP32; each tile cell
// accumulates integers (fixed point, per-subproblem power-of-two scale) with
// 32-bit shared-memory atomics, which are exact and order-independent.  Each
// lane walks its (qz, qy) rows starting at a lane-dependent offset, so lanes
// whose points share a cell (clustered data) hit different addresses.
template <int D, int W, int NV>
__device__ __forceinline__ void spread_f32_block(const SpreadArgs &a, const int sub, const float *kb)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int *tile = reinterpret_cast<int *>(smem_raw);
    __shared__ float s_part[2][NV][8];
    __shared__ float s_scale[NV];
    __shared__ int s_box[6];            // min first tap per axis, then max
    const int start = a.sub_start[sub], cnt = a.sub_count[sub];
    const int tc = tile_cells<D>(a.Pt);
    for (int e = threadIdx.x; e < tc * NV; e += blockDim.x) tile[e] = 0;
    if (threadIdx.x < 6) s_box[threadIdx.x] = threadIdx.x < 3 ? 0x7FFFFFFF : -1;
    int omin[3] = {0x7FFFFFFF, 0x7FFFFFFF, 0x7FFFFFFF}, omax[3] = {-1, -1, -1};

    // per-vector sum and max of |u| over this subproblem's points, u =
    // D^{-1/2} x in FP32; with staging, each point's sorted index and u go to
    // shared memory for the spreading pass.  Four points per thread are in
    // flight at once (the index, permutation and input loads form a chain).
    float *st_u = a.stage_off > 0 ? reinterpret_cast<float *>(smem_raw + a.stage_off) : nullptr;
    int *st_i = (st_u && a.sidx) ? reinterpret_cast<int *>(st_u + a.sub_max * NV) : nullptr;
    float lsum[NV], lmax[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) lsum[c] = lmax[c] = 0.0f;
    for (int l0 = threadIdx.x; l0 < cnt; l0 += 4 * blockDim.x) {
        int ii[4], orig[4];
        double ds[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int l = min(l0 + k * (int)blockDim.x, cnt - 1);
            ii[k] = a.sidx ? a.sidx[start + l] : start + l;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            orig[k] = a.perm[ii[k]];
            ds[k] = a.dinv ? a.dinv[ii[k]] : 1.0;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int l = l0 + k * (int)blockDim.x;
            float uk[NV];
#pragma unroll
            for (int c = 0; c < NV; ++c) uk[c] = (float)((a.X ? a.X[(int64_t)orig[k] * a.ldx + c] : 1.0) * ds[k]);
            if (l < cnt) {
#pragma unroll
                for (int c = 0; c < NV; ++c) {
                    const float au = fabsf(uk[c]);
                    lsum[c] += au;
                    lmax[c] = fmaxf(lmax[c], au);
                }
                if (st_u) {
#pragma unroll
                    for (int c = 0; c < NV; ++c) st_u[l * NV + c] = uk[c];
                    if (st_i) st_i[l] = ii[k];
                }
            }
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        const float sm = warp_sum(lsum[c]), mx = warp_max(lmax[c]);
        if (lane == 0) {
            s_part[0][c][warp] = sm;
            s_part[1][c][warp] = mx;
        }
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        float sm = 0.0f, mx = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            sm += s_part[0][threadIdx.x][w];
            mx = fmaxf(mx, s_part[1][threadIdx.x][w]);
        }
        s_scale[threadIdx.x] = fixed_scale(sm, mx);
    }
    __syncthreads();

    constexpr int ny = (D >= 2) ? W : 1, nz = (D >= 3) ? W : 1;
    constexpr int NT = W * ny * nz;                 // taps per point
    constexpr bool kWarpSum = NT <= 512;
    // full unrolling only for the small windows the throughput cases use
    constexpr int UZ = (NV == 1 && W <= 8) ? nz : 1;
    constexpr int UY = (W <= 8) ? ny : 1;
    const int ry = (D == 2) ? lane % ny : (D == 3 ? (lane / nz) % ny : 0);
    const int rz = (D == 3) ? lane % nz : 0;
    const float *coords = static_cast<const float *>(a.coords);
    const int Pt = a.Pt;
    float *slots = nullptr;
    if constexpr (RowSpread<D, W, NV>::on) {
        if (a.rows_off > 0)
            slots = reinterpret_cast<float *>(smem_raw + a.rows_off) + warp * RowSpread<D, W, NV>::warp_floats;
    }
    // a warp takes 32 consecutive points (sorted by cell); when all of them
    // have the same first tap, their taps are summed across the warp and
    // each lane adds one sum per 32 taps (warp_spread_sum), else every lane
    // adds its own point's taps
    for (int g0 = (threadIdx.x & ~31); g0 < cnt; g0 += blockDim.x) {
        const bool valid = g0 + lane < cnt;
        const int l = min(g0 + lane, cnt - 1);
        int i;
        float u[NV];
        if (st_u) {
            i = st_i ? st_i[l] : start + l;
#pragma unroll
            for (int c = 0; c < NV; ++c) u[c] = valid ? st_u[l * NV + c] * s_scale[c] : 0.0f;
        } else {
            i = a.sidx ? a.sidx[start + l] : start + l;
            const int orig = a.perm[i];
            const double ds = a.dinv ? a.dinv[i] : 1.0;
#pragma unroll
            for (int c = 0; c < NV; ++c)
                u[c] = valid ? (float)((a.X ? a.X[(int64_t)orig * a.ldx + c] : 1.0) * ds) * s_scale[c] : 0.0f;
        }
        float wx[W], wy[W], wz[W];
        int o[3] = {0, 0, 0};
        o[0] = window_row_poly<W>(coords[(int64_t)i * D], kb, wx);
        if (D >= 2) o[1] = window_row_poly<W>(coords[(int64_t)i * D + 1], kb, wy);
        if (D >= 3) o[2] = window_row_poly<W>(coords[(int64_t)i * D + 2], kb, wz);
        if (valid) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                omin[k] = min(omin[k], o[k]);
                omax[k] = max(omax[k], o[k]);
            }
        }
        const int key = o[0] | (o[1] << 10) | (o[2] << 20);
        const int key0 = __shfl_sync(0xffffffffu, key, 0);
        if (kWarpSum && __all_sync(0xffffffffu, !valid || key == key0)) {
            if constexpr (RowSpread<D, W, NV>::on) {
                if (slots) {
                    if constexpr (D == 3) warp_spread_rows<W, NV>(tile, tc, Pt, o, u, wx, wy, wz, slots, lane);
                    else warp_spread_taps<W, NV>(tile, tc, Pt, o, u, wx, wy, slots, lane);
                    continue;
                }
            }
            warp_spread_sum<D, W, NV>(tile, tc, Pt, o, u, wx, wy, wz, lane);
            continue;
        }
        if (!valid) continue;
        // rotated copies: row q of this lane is row (q + r) mod n of the point
        float wyr[ny], wzr[nz];
#pragma unroll
        for (int q = 0; q < ny; ++q) {
            int src = q + ry;
            src -= (src >= ny) ? ny : 0;
            float v = 1.0f;
#pragma unroll
            for (int k = 0; k < ny; ++k)
                if (D >= 2 && k == src) v = wy[k];
            wyr[q] = v;
        }
#pragma unroll
        for (int q = 0; q < nz; ++q) {
            int src = q + rz;
            src -= (src >= nz) ? nz : 0;
            float v = 1.0f;
#pragma unroll
            for (int k = 0; k < nz; ++k)
                if (D >= 3 && k == src) v = wz[k];
            wzr[q] = v;
        }
#pragma unroll UZ
        for (int qz0 = 0; qz0 < nz; ++qz0) {
            int qz = qz0 + rz;
            qz -= (qz >= nz) ? nz : 0;
#pragma unroll UY
            for (int qy0 = 0; qy0 < ny; ++qy0) {
                int qy = qy0 + ry;
                qy -= (qy >= ny) ? ny : 0;
                const float wyz = wzr[qz0] * wyr[qy0];
                int *row = tile + ((o[2] + qz) * Pt + o[1] + qy) * Pt + o[0];
#pragma unroll
                for (int qx = 0; qx < W; ++qx) {
                    const float wt = wyz * wx[qx];
#pragma unroll
                    for (int c = 0; c < NV; ++c) atomicAdd(row + c * tc + qx, fixed_round(u[c] * wt));
                }
            }
        }
    }
    if (a.sub_box) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            omin[k] = __reduce_min_sync(0xffffffffu, omin[k]);
            omax[k] = __reduce_max_sync(0xffffffffu, omax[k]);
        }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                atomicMin(&s_box[k], omin[k]);
                atomicMax(&s_box[3 + k], omax[k]);
            }
        }
    }
    __syncthreads();
    // the scales are powers of two: multiplying by the reciprocal is exact
    float inv_scale[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) inv_scale[c] = 1.0f / s_scale[c];
    float *out = static_cast<float *>(a.scratch) + (int64_t)sub * tc * NV;
    if (!a.sub_box) {
        for (int e = threadIdx.x; e < tc * NV; e += blockDim.x) {
            const int c = e % NV, cell = e / NV;
            float is = inv_scale[0];
#pragma unroll
            for (int k = 1; k < NV; ++k)
                if (c == k) is = inv_scale[k];
            out[e] = (float)tile[c * tc + cell] * is;
        }
        return;
    }
    // only the box of cells the taps reached: (hi_y - lo_y) (hi_z - lo_z) rows
    // of hi_x - lo_x cells, each row contiguous in the cell-major output
    int lo[3], hi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const bool used = k < D && s_box[k] <= s_box[3 + k];
        lo[k] = used ? s_box[k] : 0;
        hi[k] = used ? s_box[3 + k] + W : (k < D ? 0 : 1);
    }
    if (threadIdx.x == 0) a.sub_box[sub] = pack_box(lo, hi);
    const int span = (hi[0] - lo[0]) * NV, by = hi[1] - lo[1];
    const int rows = by * (hi[2] - lo[2]);
    if (span <= 0 || rows <= 0) return;
    const FastDiv dspan(span), dby(by);
    for (int e = threadIdx.x; e < rows * span; e += blockDim.x) {
        const int r = dspan.div(e);
        const int j = e - r * span;
        const int rz = dby.div(r);
        const int cell0 = ((lo[2] + rz) * Pt + lo[1] + r - rz * by) * Pt + lo[0];
        const int cj = j / NV, c = j - cj * NV;
        float is = inv_scale[0];
#pragma unroll
        for (int k = 1; k < NV; ++k)
            if (c == k) is = inv_scale[k];
        const int cell = cell0 + cj;
        out[cell * NV + c] = (float)tile[c * tc + cell] * is;
    }
}

template <int D, int W, int NV>
__global__ void __launch_bounds__(256) k_spread_f32(const SpreadArgs a)
{
    spread_f32_block<D, W, NV>(a, blockIdx.x, a.kbp);
}

// all layers of a batch in one launch: blockIdx.y is the layer
template <int D, int W, int NV>
__global__ void __launch_bounds__(256) k_spread_f32_batch(const SpreadArgs *__restrict__ args)
{
    const SpreadArgs a = args[blockIdx.y];
    if ((int)blockIdx.x >= a.nsub) return;
    __shared__ __align__(16) float s_kb[kPolyW * kPolyStride];
    stage_window_poly(args[blockIdx.y].kbp, s_kb, W);   // read after the block's first barrier
    spread_f32_block<D, W, NV>(a, blockIdx.x, s_kb);
}

// FP64 form: one shared tile per CTA, taps in double-word arithmetic on the
// FP32 pipes, accumulated exactly as integers with 32-bit shared-memory
// atomics (order-free, deterministic).
//  - the subproblem's inputs u = D^{-1/2} x are staged (FP64) and each vector
//    gets a power-of-two scale with every tap < 2^21 and scale * sum|u| <= 2^30
//    (fixed_scale); a tap p + e then goes to its cell as hi = round(p) and
//    lo = round((p - hi + e) * 2^20) (fixed_split), so each cell keeps
//    |sum hi| < 2^31 and |sum lo| <= 1024 * 0.75 * 2^20 (a subproblem has at
//    most 1024 points);
//  - work items are (point, slab) pairs, the slab being the point's qz (d = 3)
//    or qy (d = 2) plane of taps, numbered point-major and dealt to
//    consecutive threads: the lanes that share a point write to different
//    planes (distinct cells and banks, no same-address serialisation), and an
//    item forms u * w_z (* w_y per row) once per row and one exact product
//    with w_x per tap;
//  - hi and lo live in separate planes so that each atomic spans all banks.
// The tile is converted to FP64 exactly (hi + lo * 2^-20 has <= 51 bits).
template <int D, int W, int NV>
__global__ void __launch_bounds__(256) k_spread_f64(const SpreadArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float s_part[2][NV][8];
    __shared__ float s_scale[NV];
    const int sub = blockIdx.x;
    const int start = a.sub_start[sub], cnt = a.sub_count[sub];
    const int tc = tile_cells<D>(a.Pt);
    const int Pt = a.Pt;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *thi = reinterpret_cast<int *>(smem_raw);                          // [NV][tc]
    int *tlo = thi + (int64_t)NV * tc;                                     // [NV][tc]
    double *su = reinterpret_cast<double *>(tlo + (int64_t)NV * tc);       // [sub_max][NV]
    for (int e = threadIdx.x; e < 2 * tc * NV; e += blockDim.x) thi[e] = 0;
    float lsum[NV], lmax[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) lsum[c] = lmax[c] = 0.0f;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int j = start + i;
        const int orig = a.perm[j];
        const double ds = a.dinv ? a.dinv[j] : 1.0;
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            const double u = (a.X ? a.X[(int64_t)orig * a.ldx + c] : 1.0) * ds;
            su[i * NV + c] = u;
            const float au = fminf((float)fabs(u), 1e30f);
            lsum[c] += au;
            lmax[c] = fmaxf(lmax[c], au);
        }
    }
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        const float sm = warp_sum(lsum[c]), mx = warp_max(lmax[c]);
        if (lane == 0) {
            s_part[0][c][warp] = sm;
            s_part[1][c][warp] = mx;
        }
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        float sm = 0.0f, mx = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            sm += s_part[0][threadIdx.x][w];
            mx = fmaxf(mx, s_part[1][threadIdx.x][w]);
        }
        s_scale[threadIdx.x] = fixed_scale(sm, mx);
    }
    __syncthreads();
    constexpr int NW = D * W;
    constexpr int NI = (D >= 2) ? W : 1;       // items per point: its qz (d = 3) or qy (d = 2) slabs
    constexpr int ny = (D >= 3) ? W : 1;       // rows per item
    constexpr int UY = (W <= 8) ? ny : 1;
    const int nitems = cnt * NI;
    for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
        const int pl = it / NI;
        const int o = it - pl * NI;
        const int64_t j = start + pl;
        const float2 *wp = a.wts + j * NW;
        float2 wx[W];
#pragma unroll
        for (int q = 0; q < W; ++q) wx[q] = wp[q];
        // u times the item's slab weight (w_z of qz = o in d = 3, w_y of qy = o in d = 2)
        float2 us[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            const float2 u = dw_split(su[pl * NV + c] * (double)s_scale[c]);
            us[c] = (D >= 2) ? dw_mul(u, wp[(D - 1) * W + o]) : u;
        }
        const int off = a.offs[j];
        const int o0 = off & 1023, o1 = (off >> 10) & 1023, o2 = off >> 20;
        const int base = (D == 1) ? o0 : ((D == 2) ? (o1 + o) * Pt + o0 : ((o2 + o) * Pt + o1) * Pt + o0);
#pragma unroll UY
        for (int qy = 0; qy < ny; ++qy) {
            float2 ar[NV];
            if (D >= 3) {
                const float2 wy = wp[W + qy];
#pragma unroll
                for (int c = 0; c < NV; ++c) ar[c] = dw_mul(us[c], wy);
            } else {
#pragma unroll
                for (int c = 0; c < NV; ++c) ar[c] = us[c];
            }
            const int row = base + qy * Pt;
#pragma unroll
            for (int qx = 0; qx < W; ++qx) {
#pragma unroll
                for (int c = 0; c < NV; ++c) {
                    // exact product ar * w_x as p + e
                    const float p = __fmul_rn(ar[c].x, wx[qx].x);
                    float e = fmaf(ar[c].x, wx[qx].x, -p);
                    e = fmaf(ar[c].x, wx[qx].y, e);
                    e = fmaf(ar[c].y, wx[qx].x, e);
                    int hi, lo;
                    fixed_split(p, e, hi, lo);
                    atomicAdd(thi + c * tc + row + qx, hi);
                    atomicAdd(tlo + c * tc + row + qx, lo);
                }
            }
        }
    }
    __syncthreads();
    double *out = static_cast<double *>(a.scratch) + (int64_t)sub * tc * NV;
    for (int e = threadIdx.x; e < tc * NV; e += blockDim.x) {
        const int c = e % NV, cell = e / NV;
        // hi + lo * 2^-20 has at most 51 significant bits: exact in FP64
        out[e] = fma((double)tlo[c * tc + cell], 0x1p-20, (double)thi[c * tc + cell]) *
                 (double)(1.0f / s_scale[c]);
    }
}
// ==================================================================== fold
// One CTA per bin: each active-grid cell of the bin sums, in a fixed order,
// the tile values of every subproblem whose padded tile covers it (the bin
// itself and up to R bins below it per dim).  Deterministic, no atomics.
// The FP64 form writes the grid as double-word pairs (TO = float2) for the
// transforms that follow.
__device__ __forceinline__ void grid_store(double *out, int64_t i, double v)
{
    out[i] = v;
}
__device__ __forceinline__ void grid_store(float *out, int64_t i, float v)
{
    out[i] = v;
}
__device__ __forceinline__ void grid_store(float2 *out, int64_t i, double v)
{
    out[i] = dw_split(v);
}

// FP32 tiles with boxes (the spreading wrote only the box of cells its
// points reach): CTA (g, z) forms z-plane z of group g's tile (the whole tile
// for d < 3), one element per thread, by adding the subproblem tiles of the
// group in order (the same sums as k_group_sum, which adds the zeros outside
// the boxes too) and reading only the tiles whose box holds the element.  One
// warp first lists, in group order, the tiles whose box reaches plane z.
// Every element of the group tile is written.  At most kGroupSubsMax tiles per group.
template <int D>
__global__ void __launch_bounds__(512) k_group_sum_box(const float *__restrict__ scratch, const int *__restrict__ grp_sub,
                                                      const int4 *__restrict__ sub_box, int Pt, int nv, float *gtile)
{
    __shared__ int4 s_box[kGroupSubsMax];   // x0, x extent, y0, y extent of the listed tiles
    __shared__ int s_off[kGroupSubsMax];    // their element offsets from the group's first tile
    __shared__ int s_n;
    const int g = blockIdx.x;
    const int z = (D == 3) ? (int)blockIdx.y : 0;
    const int s0 = grp_sub[g], ns = min(grp_sub[g + 1] - s0, kGroupSubsMax);
    const int te = tile_cells<D>(Pt) * nv;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int cnt = 0;
        for (int k0 = 0; k0 < ns; k0 += 32) {
            const int k = k0 + lane;
            int4 b = make_int4(0, 0, 0, 0);
            bool in = false;
            if (k < ns) {
                b = sub_box[s0 + k];
                in = (unsigned)(z - (b.z & 0xFFFF)) < (unsigned)((b.z >> 16) - (b.z & 0xFFFF));
            }
            const unsigned m = __ballot_sync(0xffffffffu, in);
            if (in) {
                const int pos = cnt + __popc(m & ((1u << lane) - 1u));
                s_box[pos] = make_int4(b.x & 0xFFFF, (b.x >> 16) - (b.x & 0xFFFF), b.y & 0xFFFF,
                                       (b.y >> 16) - (b.y & 0xFFFF));
                s_off[pos] = k * te;
            }
            cnt += __popc(m);
        }
        if (lane == 0) s_n = cnt;
    }
    __syncthreads();
    const int nk = s_n;
    const int pc = (D == 1) ? Pt : Pt * Pt;           // cells of one plane
    const int64_t base = (int64_t)z * pc * nv;        // first element of the plane
    const float *src0 = scratch + (int64_t)s0 * te + base;
    for (int e = threadIdx.x; e < pc * nv; e += blockDim.x) {
        const int cell = e / nv;
        const int y = (D >= 2) ? cell / Pt : 0, x = cell - y * Pt;
        float acc = 0.0f;
#pragma unroll 4
        for (int j = 0; j < nk; ++j) {
            const int4 b = s_box[j];
            if ((unsigned)(x - b.x) < (unsigned)b.y && (unsigned)(y - b.z) < (unsigned)b.w) acc += src0[s_off[j] + e];
        }
        gtile[(int64_t)g * te + base + e] = acc;
    }
}





// (the cells of a bin are shared by `chunks` CTAs: chunk ch takes elements
// ch * blockDim.x + tid, stepping by chunks * blockDim.x)
template <typename T, int D, typename TO = T>
__device__ __forceinline__ void fold_block(const FoldArgs &a, const int bin, const int ch, const int chunks)
{
    int bc[3];
    bin_coords<D>(bin, a.nb0, a.nb1, bc);
    const int B = a.B, Pt = a.Pt, nv = a.nv;
    const int tc = tile_cells<D>(Pt);
    const int cells = (D == 1 ? B : (D == 2 ? B * B : B * B * B));
    const T *scr = static_cast<const T *>(a.scratch);
    TO *grid = static_cast<TO *>(a.grid);
    const FastDiv dv(nv), db(B);   // e < B^3 nv, so e * nv < 2^32 and cell * B < 2^32
    for (int e = ch * blockDim.x + threadIdx.x; e < cells * nv; e += chunks * blockDim.x) {
        const int cell = dv.div(e);
        const int c = e - cell * nv;
        const int q1 = db.div(cell);
        const int cx = cell - q1 * B;
        const int cz = (D >= 3) ? db.div(q1) : 0;
        const int cy = (D >= 2) ? q1 - cz * B : 0;
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
        grid_store(grid, ((int64_t)(gz * a.L1 + gy) * a.L0 + gx) * nv + c, acc);
    }
}

template <typename T, int D, typename TO = T>
__global__ void __launch_bounds__(256) k_fold(const FoldArgs a, int chunks)
{
    fold_block<T, D, TO>(a, blockIdx.x / chunks, blockIdx.x % chunks, chunks);
}

template <typename T, int D>
__global__ void __launch_bounds__(256) k_fold_batch(const FoldArgs *__restrict__ args, int chunks)
{
    const FoldArgs a = args[blockIdx.y];
    if ((int)blockIdx.x >= a.nbins * chunks) return;
    fold_block<T, D>(a, blockIdx.x / chunks, blockIdx.x % chunks, chunks);
}

// CTAs per bin for the fold: enough for about two CTAs per SM in all
inline int fold_chunks(int64_t bins, int64_t cells_nv, int sms)
{
    const int64_t by_work = (cells_nv + 255) / 256;
    const int64_t by_fill = (2 * (int64_t)sms + bins - 1) / std::max<int64_t>(bins, 1);
    return (int)std::max<int64_t>(1, std::min(by_work, by_fill));
}

// ==================================================================== axis
// out[(a*Ko + k)*C + c] = sum_j M[k*J + j] * in[(a*J + j)*C + c]
// (one real trigonometric transform along the middle index).  Tiles of
// 32 k x 64 flattened (a, c) pairs; 256 threads, 8 outputs each.
template <typename T, int KT = 32, int PT = 64>
__device__ __forceinline__ void axis_block(const T *__restrict__ in, T *__restrict__ out, const T *__restrict__ M,
                                           int A, int J, int Ko, int C, int bx, int by)
{
    // tiles of KT k x PT flattened (a, c) pairs; 16 threads along p and KT/2
    // along k, each thread 2 k x PT/16 p outputs (KT * 8 threads)
    constexpr int NQ = PT / 16;
    __shared__ T Ms[32][KT + 1];
    __shared__ T Is[32][PT + 1];
    const int64_t P = (int64_t)A * C;
    const int64_t p0 = (int64_t)bx * PT;
    const int k0 = by * KT;
    const int nthr = KT * 8;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[2][NQ];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[i][q] = 0;
    for (int j0 = 0; j0 < J; j0 += 32) {
        for (int e = threadIdx.x; e < 32 * KT; e += nthr) {
            const int kk = e >> 5, jj = e & 31;
            Ms[jj][kk] = (k0 + kk < Ko && j0 + jj < J) ? M[(int64_t)(k0 + kk) * J + j0 + jj] : (T)0;
        }
        for (int e = threadIdx.x; e < 32 * PT; e += nthr) {
            int jj, pp;
            if (C >= 16) { jj = e / PT; pp = e % PT; }
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
            for (int q = 0; q < NQ; ++q) {
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
        for (int q = 0; q < NQ; ++q) {
            const int64_t p = p0 + tx + 16 * q;
            if (p >= P) continue;
            const int64_t aa = p / C;
            const int cc = (int)(p - aa * C);
            out[(aa * Ko + k) * C + cc] = acc[i][q];
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_axis(const T *__restrict__ in, T *__restrict__ out,
                                              const T *__restrict__ M, int A, int J, int Ko, int C)
{
    axis_block<T>(in, out, M, A, J, Ko, C, blockIdx.x, blockIdx.y);
}

// the same with tiles of 16 k x 32 p (128 threads), for transforms whose
// 32 x 64 tiles would occupy only a few SMs
template <typename T>
__global__ void __launch_bounds__(128) k_axis_small(const T *__restrict__ in, T *__restrict__ out,
                                                    const T *__restrict__ M, int A, int J, int Ko, int C)
{
    axis_block<T, 16, 32>(in, out, M, A, J, Ko, C, blockIdx.x, blockIdx.y);
}

// FP64 form: the same transform in double-word arithmetic (grid, matrix and
// result as hi/lo pairs).  One thread per output, p = (a, c) fastest so that
// a warp mostly shares the row k of M; two compensated accumulators over
// even and odd j, renormalised every 8 terms.
template <typename F2>
__global__ void __launch_bounds__(128) k_axis_dw(const F2 *__restrict__ in, F2 *__restrict__ out,
                                                 const F2 *__restrict__ M, int A, int J, int Ko, int C)
{
    const int64_t P = (int64_t)A * C;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P * Ko) return;
    const int k = (int)(t / P);
    const int64_t p = t - (int64_t)k * P;
    const int64_t aa = p / C;
    const int cc = (int)(p - aa * C);
    const F2 *col = in + aa * J * C + cc;
    const F2 *row = M + (int64_t)k * J;
    float2 s0 = make_float2(0.0f, 0.0f), s1 = s0;
    int j = 0;
    for (; j + 1 < J; j += 2) {
        dw_fma_acc(s0, col[(int64_t)j * C], row[j]);
        dw_fma_acc(s1, col[(int64_t)(j + 1) * C], row[j + 1]);
        if ((j & 15) == 14) {
            s0 = dw_norm(s0);
            s1 = dw_norm(s1);
        }
    }
    if (j < J) dw_fma_acc(s0, col[(int64_t)j * C], row[j]);
    s0 = dw_norm(s0);
    dw_acc(s0, dw_norm(s1));
    out[(aa * Ko + k) * C + cc] = dw_norm(s0);
}

struct AxisArgs {
    const void *in;
    void *out;
    const void *M;
    int A, J, Ko, C;
};

template <typename T>
__global__ void __launch_bounds__(256) k_axis_batch(const AxisArgs *__restrict__ args)
{
    const AxisArgs a = args[blockIdx.z];
    if ((int64_t)blockIdx.x * 64 >= (int64_t)a.A * a.C || (int)blockIdx.y * 32 >= a.Ko) return;
    axis_block<T>(static_cast<const T *>(a.in), static_cast<T *>(a.out), static_cast<const T *>(a.M), a.A, a.J, a.Ko,
                  a.C, blockIdx.x, blockIdx.y);
}

struct MultArgs {
    void *coef;
    const void *mult;
    int64_t slots;
};

template <typename T>
__global__ void k_mult_batch(const MultArgs *__restrict__ args, int nv)
{
    const MultArgs a = args[blockIdx.y];
    T *coef = static_cast<T *>(a.coef);
    const T *mult = static_cast<const T *>(a.mult);
    const int64_t tot = a.slots * nv;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x)
        coef[e] *= mult[e / nv];
}

template <typename F2>
__global__ void k_mult_dw(F2 *coef, const F2 *__restrict__ mult, int64_t slots, int nv)
{
    const int64_t tot = slots * nv;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x)
        coef[e] = dw_mul(coef[e], mult[e / nv]);
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
// loaded into shared memory (vector-major), each point sums its (2M)^D taps,
// and the FP64 epilogue forms  alpha * D^{-1/2} * (sum - K(0) u) (+ shift * x)
// in input order (or the raw sum minus the self term in sorted order, for
// the degrees).
template <typename T, int NV>
__device__ __forceinline__ void load_interp_tile(const InterpArgs &a, int D, const int bc[3], int tc, T *tile)
{
    const T *grid = static_cast<const T *>(a.grid);
    const int Pt = a.Pt;
    const FastDiv dp(Pt);     // tile cells < Pt^3, so cell * Pt < 2^32
    for (int e = threadIdx.x; e < tc * NV; e += blockDim.x) {
        const int c = e % NV;
        const int cell = e / NV;
        const int q1 = dp.div(cell);
        const int lx = cell - q1 * Pt;
        const int lz = (D >= 3) ? dp.div(q1) : 0;
        const int ly = (D >= 2) ? q1 - lz * Pt : 0;
        const int gx = bc[0] * a.B + lx, gy = bc[1] * a.B + ly, gz = bc[2] * a.B + lz;
        T v{};
        if (gx < a.L0 && gy < a.L1 && gz < a.L2) v = grid[((int64_t)(gz * a.L1 + gy) * a.L0 + gx) * NV + c];
        tile[c * tc + cell] = v;
    }
}

// FP32 form: the epilogue runs in FP32 (the value carries FP32 accuracy);
// only the accumulation into the FP64 output is done in FP64.
__device__ __forceinline__ void interp_epilogue_f32(const InterpArgs &a, int i, int c, float acc)
{
    const int orig = a.perm[i];
    const float ds = a.dinv ? (float)a.dinv[i] : 1.0f;
    const float x = a.X ? (float)a.X[(int64_t)orig * a.ldx + c] : 1.0f;
    const float r = acc - (float)a.self * (x * ds);
    if (a.sorted_out) {
        a.Y[(int64_t)i * a.ldy + c] = (double)r;
    } else {
        double outv = (double)((float)a.alpha * ds * r);
        if (a.shift != 0.0) outv += a.shift * (a.X ? a.X[(int64_t)orig * a.ldx + c] : 1.0);
        double *yp = a.Y + (int64_t)(a.sorted_final ? i : orig) * a.ldy + c;
        if (a.accumulate && !a.sorted_final) outv += *yp;
        *yp = outv;
    }
}

// interp_epilogue_f32 split into its loads and its arithmetic (same results)
template <int NV>
struct EpilogueIn {
    int orig;
    float ds;
    double x[NV], yold[NV];
    __device__ __forceinline__ void load(const InterpArgs &a, int i)
    {
        orig = a.perm[i];
        ds = a.dinv ? (float)a.dinv[i] : 1.0f;
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            x[c] = a.X ? a.X[(int64_t)orig * a.ldx + c] : 1.0;
            yold[c] = (!a.sorted_out && !a.sorted_final && a.accumulate) ? a.Y[(int64_t)orig * a.ldy + c] : 0.0;
        }
    }
    __device__ __forceinline__ void finish(const InterpArgs &a, int i, int c, float acc) const
    {
        const float r = acc - (float)a.self * ((float)x[c] * ds);
        if (a.sorted_out) {
            a.Y[(int64_t)i * a.ldy + c] = (double)r;
        } else {
            double outv = (double)((float)a.alpha * ds * r);
            if (a.shift != 0.0) outv += a.shift * x[c];
            if (a.accumulate && !a.sorted_final) outv += yold[c];
            a.Y[(int64_t)(a.sorted_final ? i : orig) * a.ldy + c] = outv;
        }
    }
};

__device__ __forceinline__ void interp_epilogue(const InterpArgs &a, int i, int c, double acc)
{
    const int orig = a.perm[i];
    const double ds = a.dinv ? a.dinv[i] : 1.0;
    const double x = a.X ? a.X[(int64_t)orig * a.ldx + c] : 1.0;
    const double r = acc - a.self * (x * ds);
    if (a.sorted_out) {
        a.Y[(int64_t)i * a.ldy + c] = r;
    } else {
        double outv = a.alpha * ds * r + a.shift * x;
        double *yp = a.Y + (int64_t)(a.sorted_final ? i : orig) * a.ldy + c;
        if (a.accumulate && !a.sorted_final) outv += *yp;
        *yp = outv;
    }
}

// FP32 form: one thread per point.
template <int D, int W, int NV>
__device__ __forceinline__ void interp_f32_block(const InterpArgs &a, const int sub, const float *kb)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *tile = reinterpret_cast<float *>(smem_raw);
    const int bin = a.sub_bin[sub], start = a.sub_start[sub], cnt = a.sub_count[sub];
    const int Pt = a.Pt;
    const int tc = tile_cells<D>(Pt);
    int bc[3];
    bin_coords<D>(bin, a.nb0, a.nb1, bc);
    load_interp_tile<float, NV>(a, D, bc, tc, tile);
    if (threadIdx.x < 2) tile[tc * NV + threadIdx.x] = 0.0f;   // read with zero weights only
    __syncthreads();
    const float *coords = static_cast<const float *>(a.coords);
    constexpr int ny = (D >= 2) ? W : 1, nz = (D >= 3) ? W : 1;
    constexpr int UY = (W <= 8) ? ny : 1;       // unroll the rows of small windows
    constexpr int UZ = (NV == 1 && W <= 8) ? nz : 1;
    // an even tile edge makes every row start even up to the first tap's
    // parity: each row is then read as NP aligned float pairs from the even
    // index at or below its first tap, with the weights shifted by that
    // parity (zero weights before or after the W taps, 2 NP - W of them; the
    // zero-weight terms add nothing, so the sums are those of the W taps in the
    // same order)
    constexpr int NP = W / 2 + 1;
    const bool paired = (Pt & 1) == 0;
    // one or two vectors: the epilogue's loads (permutation, D^{-1/2}, input,
    // the previous output when accumulating) are issued before the taps, so
    // that their latency hides behind the tap sums
    constexpr bool kPrefetch = NV <= 2;
    for (int i = start + threadIdx.x; i < start + cnt; i += blockDim.x) {
        EpilogueIn<NV> ein;
        if constexpr (kPrefetch) ein.load(a, i);
        float wx[W], wy[W], wz[W];
        int o[3] = {0, 0, 0};
        o[0] = window_row_poly<W>(coords[(int64_t)i * D], kb, wx);
        if (D >= 2) o[1] = window_row_poly<W>(coords[(int64_t)i * D + 1], kb, wy);
        if (D >= 3) o[2] = window_row_poly<W>(coords[(int64_t)i * D + 2], kb, wz);
        float acc[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) acc[c] = 0.0f;
        if (paired) {
            const int odd = o[0] & 1;
            float wp[2 * NP];
#pragma unroll
            for (int k = 0; k < 2 * NP; ++k) {
                const float we = k < W ? wx[k < W ? k : 0] : 0.0f;
                const float wo = (k >= 1 && k <= W) ? wx[k >= 1 && k <= W ? k - 1 : 0] : 0.0f;
                wp[k] = odd ? wo : we;
            }
#pragma unroll UZ
            for (int qz = 0; qz < nz; ++qz) {
                float pz[NV];
#pragma unroll
                for (int c = 0; c < NV; ++c) pz[c] = 0.0f;
#pragma unroll UY
                for (int qy = 0; qy < ny; ++qy) {
                    const float *row = tile + ((o[2] + qz) * Pt + o[1] + qy) * Pt + o[0] - odd;
                    float r[NV];
#pragma unroll
                    for (int c = 0; c < NV; ++c) r[c] = 0.0f;
#pragma unroll
                    for (int kk = 0; kk < NP; ++kk)
#pragma unroll
                        for (int c = 0; c < NV; ++c) {
                            const float2 v = *reinterpret_cast<const float2 *>(row + c * tc + 2 * kk);
                            r[c] = fmaf(wp[2 * kk], v.x, r[c]);
                            r[c] = fmaf(wp[2 * kk + 1], v.y, r[c]);
                        }
                    const float wyq = (D >= 2) ? wy[qy] : 1.0f;
#pragma unroll
                    for (int c = 0; c < NV; ++c) pz[c] = fmaf(wyq, r[c], pz[c]);
                }
                const float wzq = (D >= 3) ? wz[qz] : 1.0f;
#pragma unroll
                for (int c = 0; c < NV; ++c) acc[c] = fmaf(wzq, pz[c], acc[c]);
            }
        } else {
#pragma unroll UZ
            for (int qz = 0; qz < nz; ++qz) {
                float pz[NV];
#pragma unroll
                for (int c = 0; c < NV; ++c) pz[c] = 0.0f;
#pragma unroll UY
                for (int qy = 0; qy < ny; ++qy) {
                    const float *row = tile + ((o[2] + qz) * Pt + o[1] + qy) * Pt + o[0];
                    float r[NV];
#pragma unroll
                    for (int c = 0; c < NV; ++c) r[c] = 0.0f;
#pragma unroll
                    for (int qx = 0; qx < W; ++qx)
#pragma unroll
                        for (int c = 0; c < NV; ++c) r[c] = fmaf(wx[qx], row[c * tc + qx], r[c]);
                    const float wyq = (D >= 2) ? wy[qy] : 1.0f;
#pragma unroll
                    for (int c = 0; c < NV; ++c) pz[c] = fmaf(wyq, r[c], pz[c]);
                }
                const float wzq = (D >= 3) ? wz[qz] : 1.0f;
#pragma unroll
                for (int c = 0; c < NV; ++c) acc[c] = fmaf(wzq, pz[c], acc[c]);
            }
        }
        if constexpr (kPrefetch) {
#pragma unroll
            for (int c = 0; c < NV; ++c) ein.finish(a, i, c, acc[c]);
        } else {
#pragma unroll
            for (int c = 0; c < NV; ++c) interp_epilogue_f32(a, i, c, acc[c]);
        }
    }
}

template <int D, int W, int NV>
__global__ void __launch_bounds__(256) k_interp_f32(const InterpArgs a)
{
    interp_f32_block<D, W, NV>(a, blockIdx.x, a.kbp);
}

// one vector and a narrow window: 32 registers (eight CTAs per SM, every warp
// slot) without spills; the epilogue's gathers want the warps
template <int D, int W>
__global__ void __launch_bounds__(256, 8) k_interp_f32_1v(const InterpArgs a)
{
    interp_f32_block<D, W, 1>(a, blockIdx.x, a.kbp);
}

// all layers of a batch in one launch, each writing its own output block:
// blockIdx.y is the layer
template <int D, int W, int NV>
__global__ void __launch_bounds__(256) k_interp_f32_batch(const InterpArgs *__restrict__ args)
{
    const InterpArgs a = args[blockIdx.y];
    if ((int)blockIdx.x >= a.nsub) return;
    __shared__ __align__(16) float s_kb[kPolyW * kPolyStride];
    stage_window_poly(args[blockIdx.y].kbp, s_kb, W);   // read after the block's first barrier
    interp_f32_block<D, W, NV>(a, blockIdx.x, s_kb);
}

// FP64 form: one thread per point, on the FP32 pipes.  The grid arrives as
// double-word pairs (written by the last backward transform), the weights
// from the plan's double-word table; each row sum over qx is a compensated
// dot product (dw_fma_acc), weighted by w_y and w_z in double-word products,
// and the point's value enters the FP64 epilogue as hi + lo.
template <int D, int W, int NV>
__global__ void __launch_bounds__(256) k_interp_f64(const InterpArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *tile = reinterpret_cast<float2 *>(smem_raw);
    const int sub = blockIdx.x;
    const int bin = a.sub_bin[sub], start = a.sub_start[sub], cnt = a.sub_count[sub];
    const int Pt = a.Pt;
    const int tc = tile_cells<D>(Pt);
    int bc[3];
    bin_coords<D>(bin, a.nb0, a.nb1, bc);
    load_interp_tile<float2, NV>(a, D, bc, tc, tile);
    __syncthreads();
    constexpr int NW = D * W;
    constexpr int ny = (D >= 2) ? W : 1, nz = (D >= 3) ? W : 1;
    constexpr int UY = (W <= 8) ? ny : 1;      // rows of one qz unrolled; qz not (code size)
    const float2 zero2 = make_float2(0.0f, 0.0f);
    for (int i = start + threadIdx.x; i < start + cnt; i += blockDim.x) {
        const float2 *wp = a.wts + (int64_t)i * NW;
        float2 wx[W], wy[W];
#pragma unroll
        for (int q = 0; q < W; ++q) {
            wx[q] = wp[q];
            wy[q] = (D >= 2) ? wp[W + q] : zero2;
        }
        const int off = a.offs[i];
        const int o0 = off & 1023, o1 = (off >> 10) & 1023, o2 = off >> 20;
        float2 acc[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) acc[c] = zero2;
#pragma unroll 1
        for (int qz = 0; qz < nz; ++qz) {
            const float2 wz = (D >= 3) ? wp[2 * W + qz] : zero2;
            float2 pz[NV];
#pragma unroll
            for (int c = 0; c < NV; ++c) pz[c] = zero2;
#pragma unroll UY
            for (int qy = 0; qy < ny; ++qy) {
                const float2 *row = tile + ((o2 + qz) * Pt + o1 + qy) * Pt + o0;
                float2 r[NV];
#pragma unroll
                for (int c = 0; c < NV; ++c) r[c] = zero2;
#pragma unroll
                for (int qx = 0; qx < W; ++qx)
#pragma unroll
                    for (int c = 0; c < NV; ++c) dw_fma_acc(r[c], row[c * tc + qx], wx[qx]);
#pragma unroll
                for (int c = 0; c < NV; ++c) {
                    if (D >= 2) dw_acc(pz[c], dw_mul(dw_norm(r[c]), wy[qy]));
                    else pz[c] = r[c];
                }
            }
#pragma unroll
            for (int c = 0; c < NV; ++c) {
                if (D >= 3) dw_acc(acc[c], dw_mul(dw_norm(pz[c]), wz));
                else acc[c] = pz[c];
            }
        }
#pragma unroll
        for (int c = 0; c < NV; ++c) interp_epilogue(a, i, c, dw_value(acc[c]));
    }
}

// FP32 form, all layers of a batch whose grids are single tiles and whose
// points are in input order (identity permutation, same subproblem split):
// one CTA per subproblem walks the layers, loading each layer's grid into
// shared memory in turn, and sums the layer terms
//   alpha * D_t^{-1/2} (W~_t u_t - u_t),  u_t = D_t^{-1/2} x
// in registers, so the output is written once, without atomics, in a fixed
// order.  Up to kBatchPts points per thread.
constexpr int kBatchPts = 4;

// Layer groups: CTA (sub, g) sums the layers g*LG .. min(T, (g+1)*LG) - 1; with
// more than one group each writes FP32 partial sums part[g][i][c] that
// k_sum_parts adds up in group order.
template <int D, int W, int NV>
__global__ void __launch_bounds__(256) k_interp_f32_sum(const InterpArgs *__restrict__ args, int T, int LG,
                                                        float *__restrict__ part, int64_t n)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) float s_kb[kPolyW * kPolyStride];
    float *tile = reinterpret_cast<float *>(smem_raw);
    const int sub = blockIdx.x;
    const int g = blockIdx.y;
    const int t0 = g * LG, t1 = min(T, t0 + LG);
    const InterpArgs a0 = args[0];
    const int start = a0.sub_start[sub], cnt = a0.sub_count[sub];
    constexpr int ny = (D >= 2) ? W : 1, nz = (D >= 3) ? W : 1;
    constexpr int UY = (W <= 8) ? ny : 1;
    constexpr int UZ = (NV == 1 && W <= 8) ? nz : 1;
    float tot[kBatchPts][NV];
#pragma unroll
    for (int k = 0; k < kBatchPts; ++k)
#pragma unroll
        for (int c = 0; c < NV; ++c) tot[k][c] = 0.0f;
    for (int t = t0; t < t1; ++t) {
        const InterpArgs a = args[t];
        const int Pt = a.Pt;
        const int tc = tile_cells<D>(Pt);
        const int bc[3] = {0, 0, 0};
        __syncthreads();                       // previous layer's tile no longer read
        load_interp_tile<float, NV>(a, D, bc, tc, tile);
        stage_window_poly(args[t].kbp, s_kb, W);
        __syncthreads();
        const float *coords = static_cast<const float *>(a.coords);
#pragma unroll
        for (int k = 0; k < kBatchPts; ++k) {
            const int li = threadIdx.x + k * blockDim.x;
            if (li >= cnt) break;
            const int i = start + li;
            float wx[W], wy[W], wz[W];
            int o[3] = {0, 0, 0};
            o[0] = window_row_poly<W>(coords[(int64_t)i * D], s_kb, wx);
            if (D >= 2) o[1] = window_row_poly<W>(coords[(int64_t)i * D + 1], s_kb, wy);
            if (D >= 3) o[2] = window_row_poly<W>(coords[(int64_t)i * D + 2], s_kb, wz);
            float acc[NV];
#pragma unroll
            for (int c = 0; c < NV; ++c) acc[c] = 0.0f;
#pragma unroll UZ
            for (int qz = 0; qz < nz; ++qz) {
                float pz[NV];
#pragma unroll
                for (int c = 0; c < NV; ++c) pz[c] = 0.0f;
#pragma unroll UY
                for (int qy = 0; qy < ny; ++qy) {
                    const float *row = tile + ((o[2] + qz) * Pt + o[1] + qy) * Pt + o[0];
                    float r[NV];
#pragma unroll
                    for (int c = 0; c < NV; ++c) r[c] = 0.0f;
#pragma unroll
                    for (int qx = 0; qx < W; ++qx)
#pragma unroll
                        for (int c = 0; c < NV; ++c) r[c] = fmaf(wx[qx], row[c * tc + qx], r[c]);
                    const float wyq = (D >= 2) ? wy[qy] : 1.0f;
#pragma unroll
                    for (int c = 0; c < NV; ++c) pz[c] = fmaf(wyq, r[c], pz[c]);
                }
                const float wzq = (D >= 3) ? wz[qz] : 1.0f;
#pragma unroll
                for (int c = 0; c < NV; ++c) acc[c] = fmaf(wzq, pz[c], acc[c]);
            }
            const float ds = a.dinv ? (float)a.dinv[i] : 1.0f;
#pragma unroll
            for (int c = 0; c < NV; ++c) {
                const float x = a.X ? (float)a.X[(int64_t)i * a.ldx + c] : 1.0f;
                tot[k][c] += (float)a.alpha * ds * (acc[c] - (float)a.self * (x * ds));
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kBatchPts; ++k) {
        const int li = threadIdx.x + k * blockDim.x;
        if (li >= cnt) break;
        const int i = start + li;
        if (part) {
#pragma unroll
            for (int c = 0; c < NV; ++c) part[((int64_t)g * n + i) * NV + c] = tot[k][c];
        } else {
#pragma unroll
            for (int c = 0; c < NV; ++c) a0.Y[(int64_t)i * a0.ldy + c] = (double)tot[k][c];
        }
    }
}

// Y[i, c] = sum over the G layer groups of part[g][i][c], in group order
template <int NV>
__global__ void k_sum_parts(const float *__restrict__ part, int G, int64_t n, double *Y, int ldy)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * NV; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / NV;
        const int c = (int)(e - i * NV);
        double s = 0.0;
        for (int g = 0; g < G; ++g) s += (double)part[(int64_t)g * n * NV + e];
        Y[i * ldy + c] = s;
    }
}

}  // namespace ml
