// FP64-exact dense products of the Lanczos solvers on the fp16 tensor cores
// (tcgen05), by splitting every FP64 operand into 8-bit slices (the error-free
// splitting of Ozaki, Ogita, Oishi and Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59 (2012)).
//
// A value v with |v| < 2^(e+1) is written as the 64-bit fixed-point integer
// F = round(|v| 2^(63-e)) and its eight bytes d_1 (most significant) .. d_8:
//     v = sign(v) 2^e sum_{a=1..8} d_a 2^(1-8a)   (error <= 2^(e-64)).
// Every slice value is an integer 0..255 with its sign, exact in fp16, and a
// product of two slices is below 2^16; so a tensor-core dot product of up to
// 256 slice pairs (accumulated in FP32) is an exact integer below 2^24.  The
// product of two split matrices is the sum over slice pairs (a, b) of
// 2^(2-8(a+b)) D_ab; the pairs with a + b <= 10 are kept (a dropped pair
// weighs below 2^-70 per term), summed as integers, and converted to FP64
// once.  Eight slices (64 bits) leave a value of magnitude 2^-12 relative to
// its scale (a unit vector of 10^7 entries) with 52 significant bits.
//
// Two products of the Lanczos solvers take this path (Sec. 3: the block
// Gram-Schmidt reorthogonalisation and the Ritz vectors), each over a basis
// Q whose columns are orthonormal, so |Q_ij| <= 1 and the basis uses the
// fixed scale e = 0 (|v| < 2; a larger value sets the error flag):
//   gram:  G = A^T B   (A: n x rc basis columns, B: n x cb block of any
//                       norm, one exponent per column of B over the rows of
//                       a thread block; rc <= 48, cb <= 8), K = n accumulated
//                       in chunks of 64 rows, drained to 64-bit integers
//                       every 256 rows;
//   gemm:  Y (-)= A M  (A: n x rc, M: rc x cb small, any magnitude: one
//                       exponent per column of M), 128 rows per tile.
//
// Layout of the slices in shared memory: K-major fp16 core matrices
// (tc05.cuh), core matrix (row group g, K group k) at byte
// (g * KG + k) * 128 with KG = K / 8 groups along K.
#include <cuda_runtime.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <string>

#include "ml_internal.h"
#include "tc05.cuh"

namespace ml {

// error flags: 1 = an operand beyond the fixed scale, 2 = a bounded wait gave up
static __device__ int g_oz_err;

namespace {

constexpr int kOzThreads = 512;   // 16 warps
constexpr int kOzSlices = 8;
constexpr int kGramKC = 32;       // rows per chunk (K of one round of MMAs)
constexpr int kGramDrain = 8;     // chunks per integer drain (256 rows)
constexpr long kOzWait = 1L << 26;
constexpr int kOzMaxRc = 48;      // basis columns of one product

// F = round(|v| 2^(63 + eoff)) as (hi, lo) words for |v| 2^eoff < 2, from the
// bits of v with 64-bit shifts (no FP64 arithmetic); the sign bit in neg
__device__ __forceinline__ void oz_fixed(double v, int eoff, uint32_t &hi, uint32_t &lo, uint32_t &neg, int &ovf)
{
    const uint32_t whi = (uint32_t)__double2hiint(v), wlo = (uint32_t)__double2loint(v);
    neg = whi >> 31;
    const int E = (int)((whi >> 20) & 0x7FF);
    const unsigned long long M = (((unsigned long long)((whi & 0xFFFFFu) | 0x100000u) << 32) | wlo) << 11;
    const int r = 1023 - E - eoff;       // F = M 2^-r
    unsigned long long F = M;
    if (r > 0) F = r >= 64 ? 0ull : (((M >> (r - 1)) + 1ull) >> 1);
    if (r < 0) {
        ovf = 1;
        F = ~0ull;
    }
    if (E == 0) F = 0;                   // zero or subnormal: below the last slice
    lo = (uint32_t)F;
    hi = (uint32_t)(F >> 32);
}

// slice a (1..8) of two values as an fp16 pair: the bytes d of F0 and F1
// placed under the exponent of 1024 (fp16 0x6400 | d = 1024 + d), then
// (1024 + d) s - 1024 s = +-d exactly; s = +-1 per half from the sign bits
__device__ __forceinline__ uint32_t oz_pair(uint32_t w0, uint32_t w1, int byte, __half2 sgn, __half2 nb)
{
    const uint32_t t = __byte_perm(w0, w1, (uint32_t)byte | ((uint32_t)(byte + 4) << 8));
    const uint32_t x = (t & 0x00FF00FFu) | 0x64006400u;
    const __half2 h = __hfma2(*reinterpret_cast<const __half2 *>(&x), sgn, nb);
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ void oz_signs(uint32_t neg0, uint32_t neg1, __half2 &sgn, __half2 &nb)
{
    const __half s0 = neg0 ? __float2half(-1.0f) : __float2half(1.0f);
    const __half s1 = neg1 ? __float2half(-1.0f) : __float2half(1.0f);
    const __half b0 = neg0 ? __float2half(1024.0f) : __float2half(-1024.0f);
    const __half b1 = neg1 ? __float2half(1024.0f) : __float2half(-1024.0f);
    sgn = __halves2half2(s0, s1);
    nb = __halves2half2(b0, b1);
}

// the eight fp16 slice pairs of two values into eight words at addr + (a - 1) * sstride
__device__ __forceinline__ void oz_store_pairs(double v0, double v1, int eoff, unsigned char *addr, uint32_t sstride,
                                               int &ovf)
{
    uint32_t h0, l0, n0, h1, l1, n1;
    oz_fixed(v0, eoff, h0, l0, n0, ovf);
    oz_fixed(v1, eoff, h1, l1, n1, ovf);
    __half2 sgn, nb;
    oz_signs(n0, n1, sgn, nb);
#pragma unroll
    for (int a = 1; a <= 4; ++a)
        *reinterpret_cast<uint32_t *>(addr + (a - 1) * sstride) = oz_pair(h0, h1, 4 - a, sgn, nb);
#pragma unroll
    for (int a = 5; a <= 8; ++a)
        *reinterpret_cast<uint32_t *>(addr + (a - 1) * sstride) = oz_pair(l0, l1, 8 - a, sgn, nb);
}

// slice a of one value as a signed float (small matrices)
__device__ __forceinline__ float oz_slice1(double v, int eoff, int a, int &ovf)
{
    uint32_t h, l, ng;
    oz_fixed(v, eoff, h, l, ng, ovf);
    const uint32_t w = a <= 4 ? h : l;
    const int byte = a <= 4 ? 4 - a : 8 - a;
    const float d = (float)((w >> (8 * byte)) & 0xFFu);
    return ng ? -d : d;
}

// byte offset of element (row, k) in a K-major core-matrix operand with KG K-groups
__device__ __forceinline__ uint32_t core_off(int row, int k, int KG)
{
    return (uint32_t)(((row >> 3) * KG + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// ------------------------------------------------------------------ gram
// part[(y * gridDim.x + x) * rc * cb + c * cb + j] = sum over this CTA's rows i of A_t[i, c] B_t[i, j]
// Â (M operand): rows (a, c) = a * RCP + c, RCP = rc rounded up to 8, MT tiles of 128 rows
// B̂ (N operand): rows (b, j) = b * 8 + j, 64 rows
// 12 warps: all of them turn chunks of 32 rows into slices (each warp a few
// 8 x 8 "units", the next chunk's values loaded ahead in registers); one
// thread issues the MMAs; at a drain, warp (q, g) reads TMEM lanes 32 q.. of
// tile g, i.e. one row (a, c) of Â per thread.  Two CTAs share an SM.
constexpr int kGramThreads = 384;
constexpr int kGramUPW = 3;          // units per warp and chunk (up to 28 units)

__global__ void __launch_bounds__(kGramThreads, 2) k_oz_gram(OzMat A, int rc, OzMat B, int cb,
                                                             const int *__restrict__ lay, int64_t n,
                                                             int64_t rows_per_cta, double *part)
{
    extern __shared__ __align__(1024) unsigned char oz_smem[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tslot;
    __shared__ int bexp[8];
    const int RCP = (rc + 7) & ~7;
    const int MT = (kOzSlices * RCP + 127) / 128;
    const uint32_t a_bytes = (uint32_t)MT * 128 * kGramKC * 2, b_bytes = 64u * kGramKC * 2;
    const uint32_t stage_bytes = a_bytes + b_bytes;
    const uint32_t ncols = MT <= 1 ? 64 : (MT <= 2 ? 128 : 256);
    const int t = lay[blockIdx.y];
    const double *Ab = A.base + (int64_t)t * A.lstride, *Bb = B.base + (int64_t)t * B.lstride;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t r1 = min(n, r0 + rows_per_cta);
    const int nchunks = r1 > r0 ? (int)((r1 - r0 + kGramKC - 1) / kGramKC) : 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rr = lane >> 2, ww = lane & 3;
    constexpr int KG = kGramKC / 8;
    constexpr int NW = kGramThreads / 32;

    // zero both stages (rows never written stay zero), barriers, TMEM
    for (uint32_t e = threadIdx.x; e < 2 * stage_bytes / 16; e += blockDim.x)
        reinterpret_cast<uint4 *>(oz_smem)[e] = make_uint4(0, 0, 0, 0);
    // B's columns get their own scale over this block's rows (B may be a
    // vector of any norm, e.g. the residual after a first projection): slices
    // of B_ij 2^(1 - f_j) with |B_ij| < 2^f_j, and the partial Gram times 2^(f_j - 1)
    if (threadIdx.x < 8) bexp[threadIdx.x] = -100000;
    if (threadIdx.x == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
    }
    if (warp == 0) tc::tmem_alloc(&tslot, ncols);
    __syncthreads();
    {
        int mx[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) mx[j] = -100000;
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x)
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < cb) {
                    const double v = Bb[i * B.rs + (int64_t)j * B.cs];
                    if (v != 0.0) {
                        int ex;
                        frexp(v, &ex);
                        mx[j] = max(mx[j], ex);
                    }
                }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            int m = mx[j];
            for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0 && j < cb && m > -100000) atomicMax(&bexp[j], m);
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tslot;

    // this thread's units: u = warp + NW * k; unit -> (is B, column group, K group)
    const int ua = (RCP / 8) * KG, units = ua + KG;
    // per unit: the element pointer of its first row, the row step, the
    // exponent offset of its column (B) and its slice-1 address in a stage
    const double *uptr[kGramUPW];
    int64_t ustep[kGramUPW];
    int ueoff[kGramUPW], urow[kGramUPW];
    uint32_t uoff[kGramUPW], ustride[kGramUPW];
    bool uon[kGramUPW];
#pragma unroll
    for (int k = 0; k < kGramUPW; ++k) {
        const int u = warp + NW * k;
        const bool isb = u >= ua;
        const int uu = isb ? u - ua : u;
        const int cg = uu / KG, kg = uu - cg * KG;
        const int col = cg * 8 + rr;
        const OzMat &X = isb ? B : A;
        uon[k] = u < units && col < (isb ? cb : rc);
        uptr[k] = (isb ? Bb : Ab) + (r0 + kg * 8 + 2 * ww) * X.rs + (int64_t)col * X.cs;
        ustep[k] = X.rs;
        urow[k] = kg * 8 + 2 * ww;                                   // row within a chunk
        ueoff[k] = (isb && col < cb) ? 1 - (bexp[col] > -100000 ? bexp[col] : 0) : 0;
        uoff[k] = (isb ? a_bytes : 0u) + core_off(col, kg * 8 + 2 * ww, KG);
        ustride[k] = (uint32_t)(isb ? 8 : RCP) * KG * 16;            // bytes between slices
        if (u >= units) uoff[k] = 0xFFFFFFFFu;                       // no unit
    }
    auto load = [&](int ch, double (&v)[kGramUPW][2]) {
#pragma unroll
        for (int k = 0; k < kGramUPW; ++k) {
            const int64_t i = r0 + (int64_t)ch * kGramKC + urow[k];
            const double *p = uptr[k] + (int64_t)ch * kGramKC * ustep[k];
            v[k][0] = (uon[k] && ch < nchunks && i < r1) ? p[0] : 0.0;
            v[k][1] = (uon[k] && ch < nchunks && i + 1 < r1) ? p[ustep[k]] : 0.0;
        }
    };

    // drain bookkeeping: thread -> (tile g, TMEM lane 32 q + lane) -> Â row (a, c)
    const int q = warp & 3, g = warp >> 2;
    const int arow = g * 128 + q * 32 + lane;
    const int a_idx = arow / RCP, c_own = arow - a_idx * RCP;
    const bool own = g < MT && a_idx < kOzSlices && c_own < rc;
    long long hi_acc[8], lo_acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) hi_acc[j] = lo_acc[j] = 0;

    int ovf = 0;
    bool ok = true;
    int last = -1;                                  // last chunk whose MMAs were committed
    double vnext[kGramUPW][2];
    load(0, vnext);
    for (int ch = 0; ch < nchunks && ok; ++ch) {
        const int s = ch & 1;
        double vcur[kGramUPW][2];
#pragma unroll
        for (int k = 0; k < kGramUPW; ++k) {
            vcur[k][0] = vnext[k][0];
            vcur[k][1] = vnext[k][1];
        }
        load(ch + 1, vnext);                        // in flight while this chunk is sliced
        if (ch >= 2) ok = tc::mbar_wait(&mbar[s], ((ch - 2) >> 1) & 1, kOzWait);   // stage s free
        ok = __syncthreads_and(ok);
        if (!ok) break;
        unsigned char *sa = oz_smem + s * stage_bytes, *sb = sa + a_bytes;
#pragma unroll
        for (int k = 0; k < kGramUPW; ++k)
            if (uoff[k] != 0xFFFFFFFFu)
                oz_store_pairs(vcur[k][0], vcur[k][1], ueoff[k], sa + uoff[k], ustride[k], ovf);
        tc::fence_proxy_async();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        const bool first = (ch % kGramDrain) == 0;
        if (threadIdx.x == 0) {
            const uint32_t idesc = tc::idesc_f16(128, 64);
            const uint32_t abase = tc::smem_addr(sa), bbase = tc::smem_addr(sb);
            for (int mt = 0; mt < MT; ++mt)
                for (int ks = 0; ks < kGramKC / 16; ++ks) {
                    const uint64_t ad = tc::desc_kmajor(abase + mt * 16 * KG * 128 + ks * 256, 128, KG * 128);
                    const uint64_t bd = tc::desc_kmajor(bbase + ks * 256, 128, KG * 128);
                    tc::mma_f16(tmem + mt * 64, ad, bd, idesc, !(first && ks == 0));
                }
            tc::commit(&mbar[s]);
        }
        last = ch;
        const bool drain = (ch % kGramDrain) == kGramDrain - 1 || ch == nchunks - 1;
        if (drain) {
            ok = tc::mbar_wait(&mbar[s], (ch >> 1) & 1, kOzWait);
            ok = __syncthreads_and(ok);
            if (!ok) break;
            tc::fence_after();
            if (g < MT) {
                const int a = a_idx + 1;
#pragma unroll
                for (int bi = 0; bi < kOzSlices; ++bi) {
                    uint32_t r[8];
                    tc::tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + g * 64 + bi * 8, r);
                    tc::tmem_ld_wait();
                    const int b = bi + 1;
                    if (own && a + b <= 10) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const long long d = (long long)__float2int_rn(__uint_as_float(r[j]));
                            if (b <= 4) hi_acc[j] += d * (1LL << (8 * (4 - b)));
                            else lo_acc[j] += d * (1LL << (8 * (8 - b)));
                        }
                    }
                }
            }
            tc::fence_before();
            __syncthreads();
            tc::fence_after();
        }
    }
    if (ovf) atomicOr(&g_oz_err, 1);
    if (!ok) {
        atomicOr(&g_oz_err, 2);
        if (last >= 0) tc::mbar_wait(&mbar[last & 1], (last >> 1) & 1, kOzWait);   // MMAs in flight
    }
    // sum_b 2^(-8b) D_ab = hi 2^-32 + lo 2^-64; weight 2^(2-8a) for slice a of A
    __syncthreads();
    double *red = reinterpret_cast<double *>(oz_smem);     // [8][RCP][8]
    if (own && ok) {
        const int a = a_idx + 1;
        const double wh = ldexp(1.0, 2 - 8 * a - 32), wl = ldexp(1.0, 2 - 8 * a - 64);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            red[(a_idx * RCP + c_own) * 8 + j] = fma((double)hi_acc[j], wh, (double)lo_acc[j] * wl);
    }
    __syncthreads();
    const int nout = rc * cb;
    for (int e = threadIdx.x; e < nout; e += blockDim.x) {
        const int c = e / cb, j = e - c * cb;
        double sacc = 0.0;
        if (ok)
            for (int ai = 0; ai < kOzSlices; ++ai) sacc += red[(ai * RCP + c) * 8 + j];
        const int ex = bexp[j] > -100000 ? bexp[j] : 0;
        part[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * nout + e] = ldexp(sacc, ex - 1);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// ------------------------------------------------------------------ gemm
__device__ __forceinline__ void tmem_ld2(uint32_t taddr, uint32_t &r0, uint32_t &r1)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(taddr));
}

// exact integer value of an FP32 holding an integer of magnitude < 2^22
__device__ __forceinline__ int small_int(uint32_t fbits)
{
    return __float_as_int(__uint_as_float(fbits) + 12582912.0f) - 0x4B400000;
}

// Y_t[i, j] (-)= sum_{r < rc} A_t[i, r] M_y[r, j], j < cb, for 128-row tiles
// bx, bx + gridDim.x, ...; M_y[r, j] = M[y * mslot + r * mrs + j * mcs] (y the slot).
// Â_a (M operand, one per slice a): 128 rows x K16 (rc rounded up to 16);
// M̂ (N operand): rows (b, j) = b * 8 + j, 64 rows, K16 columns; one TMEM
// accumulator of 64 columns per slice a of A.
__global__ void __launch_bounds__(kOzThreads, 1) k_oz_gemm(OzMat A, int rc, const double *__restrict__ M, int64_t mrs,
                                                           int64_t mcs, int64_t mslot, int cb, OzOut Y,
                                                           const int *__restrict__ lay, int64_t n, int sub)
{
    extern __shared__ __align__(1024) unsigned char oz_smem[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tslot;
    __shared__ int mexp[8];
    const int K16 = (rc + 15) & ~15;
    const int KG = K16 / 8;
    const uint32_t slice_bytes = 128u * K16 * 2, stage_bytes = kOzSlices * slice_bytes;
    const uint32_t mhat_bytes = 64u * K16 * 2;
    unsigned char *mhat = oz_smem + 2 * stage_bytes;
    const uint32_t ncols = 512;
    const int y = blockIdx.y, t = lay[y];
    const double *Ab = A.base + (int64_t)t * A.lstride;
    double *Yb = Y.base + (int64_t)t * Y.lstride;
    const double *My = M + (int64_t)y * mslot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rr = lane >> 2, ww = lane & 3;
    const int64_t ntiles = (n + 127) / 128;

    // M̂: per-column exponents, then the slices of M 2^(1 - e_j) (|.| < 2)
    for (uint32_t e = threadIdx.x; e < mhat_bytes / 16; e += blockDim.x)
        reinterpret_cast<uint4 *>(mhat)[e] = make_uint4(0, 0, 0, 0);
    if (threadIdx.x < 8) mexp[threadIdx.x] = -100000;
    if (threadIdx.x == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
    }
    if (warp == 0) tc::tmem_alloc(&tslot, ncols);
    __syncthreads();
    for (int e = threadIdx.x; e < rc * cb; e += blockDim.x) {
        const int r = e / cb, j = e - r * cb;
        const double v = My[r * mrs + j * mcs];
        if (v != 0.0) {
            int ex;
            frexp(v, &ex);
            atomicMax(&mexp[j], ex);
        }
    }
    __syncthreads();
    int ovf = 0;
    for (int e = threadIdx.x; e < rc * cb; e += blockDim.x) {
        const int r = e / cb, j = e - r * cb;
        const int ex = mexp[j] < -50000 ? 0 : mexp[j];
        const double mv = My[r * mrs + j * mcs];
#pragma unroll
        for (int b = 1; b <= kOzSlices; ++b)
            *reinterpret_cast<__half *>(mhat + core_off((b - 1) * 8 + j, r, KG)) =
                __float2half_rn(oz_slice1(mv, 1 - ex, b, ovf));
    }

    // this thread's units of a tile: u = warp + 16 k -> (row group, K group)
    constexpr int kUPW = 6;                         // K16 <= 48: at most 6 K groups
    auto load = [&](int64_t tile, double (&v)[kUPW][2]) {
        const int64_t i0 = tile * 128;
#pragma unroll
        for (int k = 0; k < kUPW; ++k) {
            const int u = warp + 16 * k;
            const int rg = u / KG, kg = u - rg * KG;
            const int64_t i = i0 + rg * 8 + rr;
            const int k0 = kg * 8 + 2 * ww;
#pragma unroll
            for (int e = 0; e < 2; ++e)
                v[k][e] = (k < KG && tile < ntiles && k0 + e < rc && i < n) ? Ab[i * A.rs + (int64_t)(k0 + e) * A.cs]
                                                                             : 0.0;
        }
    };
    auto slice = [&](const double (&v)[kUPW][2], unsigned char *stage) {
#pragma unroll
        for (int k = 0; k < kUPW; ++k) {
            if (k >= KG) break;
            const int u = warp + 16 * k;
            const int rg = u / KG, kg = u - rg * KG;
            oz_store_pairs(v[k][0], v[k][1], 0, stage + core_off(rg * 8 + rr, kg * 8 + 2 * ww, KG), slice_bytes, ovf);
        }
        tc::fence_proxy_async();
    };
    auto issue = [&](unsigned char *stage, uint64_t *bar) {
        const uint32_t idesc = tc::idesc_f16(128, 64);
        const uint32_t sbase = tc::smem_addr(stage), mbase = tc::smem_addr(mhat);
        for (int a = 0; a < kOzSlices; ++a)
            for (int ks = 0; ks < K16 / 16; ++ks) {
                const uint64_t ad = tc::desc_kmajor(sbase + a * slice_bytes + ks * 256, 128, KG * 128);
                const uint64_t bd = tc::desc_kmajor(mbase + ks * 256, 128, KG * 128);
                tc::mma_f16(tslot + a * 64, ad, bd, idesc, ks > 0);
            }
        tc::commit(bar);
    };

    bool ok = true;
    int64_t tile = blockIdx.x;
    int idx = 0, last = -1;
    double v[kUPW][2];
    load(tile, v);
    if (tile < ntiles) slice(v, oz_smem);
    load(tile + gridDim.x, v);                      // the next tile's values, in flight
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tslot;
    if (tile < ntiles && threadIdx.x == 0) issue(oz_smem, &mbar[0]);
    if (tile < ntiles) last = 0;
    const int q = warp & 3, g = warp >> 2;
    for (; tile < ntiles; tile += gridDim.x, ++idx) {
        const int64_t next = tile + gridDim.x;
        if (next < ntiles) slice(v, oz_smem + ((idx + 1) & 1) * stage_bytes);
        load(next + gridDim.x, v);                  // two tiles ahead
        ok = tc::mbar_wait(&mbar[idx & 1], (idx >> 1) & 1, kOzWait);
        ok = __syncthreads_and(ok);
        if (!ok) break;
        tc::fence_after();
        // drain: TMEM lane 32 q + lane = row, outputs j = 2 g, 2 g + 1; the
        // pairs of slices (a, b) with a + b = d summed per diagonal d = 2..10
        int S[2][11];
#pragma unroll
        for (int jj = 0; jj < 2; ++jj)
#pragma unroll
            for (int e = 0; e < 11; ++e) S[jj][e] = 0;
#pragma unroll
        for (int a = 1; a <= kOzSlices; ++a) {
            uint32_t d[8][2];
#pragma unroll
            for (int b = 1; b <= kOzSlices; ++b)
                if (a + b <= 10)
                    tmem_ld2(tmem + ((uint32_t)(q * 32) << 16) + (a - 1) * 64 + (b - 1) * 8 + 2 * g, d[b - 1][0],
                             d[b - 1][1]);
            tc::tmem_ld_wait();
#pragma unroll
            for (int b = 1; b <= kOzSlices; ++b)
                if (a + b <= 10) {
                    S[0][a + b] += small_int(d[b - 1][0]);
                    S[1][a + b] += small_int(d[b - 1][1]);
                }
        }
        const int64_t i = tile * 128 + q * 32 + lane;
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
            const int j = 2 * g + jj;
            const int *Sd = S[jj];
            // sum_d 2^(-8d) S_d = hi 2^-40 + lo 2^-80
            const long long hi = (long long)Sd[2] * 16777216 + (long long)Sd[3] * 65536 + (long long)Sd[4] * 256 + Sd[5];
            const long long lo = (long long)Sd[6] * 4294967296LL + (long long)Sd[7] * 16777216 +
                                 (long long)Sd[8] * 65536 + (long long)Sd[9] * 256 + Sd[10];
            if (j < cb && i < n) {
                const int ex = mexp[j] < -50000 ? 0 : mexp[j];
                const double val = fma((double)hi, ldexp(1.0, ex + 1 - 40), (double)lo * ldexp(1.0, ex + 1 - 80));
                double *yp = Yb + i * Y.rs + (int64_t)j * Y.cs;
                *yp = sub ? *yp - val : val;
            }
        }
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (next < ntiles) {
            if (threadIdx.x == 0) issue(oz_smem + ((idx + 1) & 1) * stage_bytes, &mbar[(idx + 1) & 1]);
            last = idx + 1;
        }
    }
    if (ovf) atomicOr(&g_oz_err, 1);
    if (!ok) {
        atomicOr(&g_oz_err, 2);
        if (last >= 0) tc::mbar_wait(&mbar[last & 1], (last >> 1) & 1, kOzWait);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

}  // namespace

// ------------------------------------------------------------------ host
// The solvers' products of the basis: 0 on the FP64 pipe, 1 in double-word
// arithmetic on the FP32 pipes (the default), 2 on the tensor cores through
// the slices above.  On GB300 the tensor-core path is not faster for these
// shapes (a basis of <= 48 columns against blocks of <= 8 vectors): forming
// the eight slices of every FP64 element costs more issue slots than the
// FP64 multiply-adds it replaces.
static std::atomic<int> g_dense_kind{1};

int dense_products_kind() { return g_dense_kind.load(std::memory_order_relaxed); }
bool oz_enabled() { return dense_products_kind() == 2; }

bool oz_gram_ok(int rc, int cb) { return rc >= 1 && rc <= kOzMaxRc && cb >= 1 && cb <= 8; }
bool oz_gemm_ok(int rc) { return rc >= 1 && rc <= kOzMaxRc; }

// at least 80 KB, so that at most two Gram CTAs share an SM (two TMEM
// allocations of up to 256 columns each)
static size_t gram_smem(int rc)
{
    const int RCP = (rc + 7) & ~7, MT = (kOzSlices * RCP + 127) / 128;
    return std::max<size_t>(2 * ((size_t)MT * 128 * kGramKC * 2 + 64 * kGramKC * 2), (size_t)80 << 10);
}
static size_t gemm_smem(int rc)
{
    const int K16 = (rc + 15) & ~15;
    return 2 * (size_t)kOzSlices * 128 * K16 * 2 + 64 * (size_t)K16 * 2;
}

static ml_status oz_attrs()
{
    static int done[64] = {0};
    int dev = 0;
    ML_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && done[dev]) return ML_OK;
    ML_CUDA(cudaFuncSetAttribute(k_oz_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_smem(kOzMaxRc)));
    ML_CUDA(cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem(kOzMaxRc)));
    if (dev >= 0 && dev < 64) done[dev] = 1;
    return ML_OK;
}

int oz_gram_blocks(int nslots, int64_t n)
{
    const int64_t per = std::max<int64_t>(1, 2 * sm_count() / std::max(1, nslots));
    return (int)std::max<int64_t>(1, std::min<int64_t>(per, (n + 255) / 256));
}

ml_status oz_gram(OzMat A, int rc, OzMat B, int cb, const int *lay, int nslots, int64_t n, int nbx, double *part,
                  cudaStream_t st)
{
    if (!oz_gram_ok(rc, cb)) return fail(ML_ERR_ARG, "tensor-core Gram: sizes out of range");
    ML_TRY(oz_attrs());
    int64_t rows = (n + nbx - 1) / nbx;
    rows = (rows + kGramKC - 1) / kGramKC * kGramKC;
    // 64-bit drain sums stay below 2^62 for up to 2^21 rows per block
    if (rows > (int64_t)1 << 21) return fail(ML_ERR_ARG, "tensor-core Gram: more than 2^21 rows per block");
    k_oz_gram<<<dim3(nbx, nslots), kGramThreads, gram_smem(rc), st>>>(A, rc, B, cb, lay, n, rows, part);
    ML_CUDA(cudaGetLastError());
    return ML_OK;
}

ml_status oz_gemm(OzMat A, int rc, const double *M, int64_t mrs, int64_t mcs, int64_t mslot, int cb, OzOut Y,
                  const int *lay, int nslots, int64_t n, bool sub, cudaStream_t st)
{
    if (!oz_gemm_ok(rc) || cb < 1) return fail(ML_ERR_ARG, "tensor-core product: sizes out of range");
    ML_TRY(oz_attrs());
    const int64_t ntiles = (n + 127) / 128;
    const int nbx = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (sm_count() + nslots - 1) / nslots));
    for (int j0 = 0; j0 < cb; j0 += 8) {
        OzOut Yj = Y;
        Yj.base += (int64_t)j0 * Y.cs;
        k_oz_gemm<<<dim3(nbx, nslots), kOzThreads, gemm_smem(rc), st>>>(A, rc, M + j0 * mcs, mrs, mcs, mslot,
                                                                        std::min(8, cb - j0), Yj, lay, n, sub ? 1 : 0);
        ML_CUDA(cudaGetLastError());
    }
    return ML_OK;
}

ml_status oz_reset_error(cudaStream_t st)
{
    const int zero = 0;
    ML_CUDA(cudaMemcpyToSymbolAsync(g_oz_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
    return ML_OK;
}

// reads the flags (synchronises the stream): 0, or 1 (an operand beyond the
// fixed scale) | 2 (a bounded wait gave up)
ml_status oz_read_error(int *flags, cudaStream_t st)
{
    ML_CUDA(cudaMemcpyFromSymbolAsync(flags, g_oz_err, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
    ML_CUDA(cudaStreamSynchronize(st));
    return ML_OK;
}

}  // namespace ml

extern "C" ml_status ml_set_dense_products(int kind)
{
    if (kind < 0 || kind > 2) return ml::fail(ML_ERR_ARG, "kind must be 0 (FP64), 1 (double-word) or 2 (tensor cores)");
    ml::g_dense_kind.store(kind);
    return ML_OK;
}

namespace ml {
namespace {
__global__ void k_oz_reduce(const double *__restrict__ part, int nbx, int nout, double *out)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nout; e += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int x = 0; x < nbx; ++x) acc += part[(int64_t)x * nout + e];
        out[e] = acc;
    }
}
}  // namespace

static ml_status oz_finish(cudaStream_t st)
{
    int flags = 0;
    ML_TRY(oz_read_error(&flags, st));
    if (flags & 2) return fail(ML_ERR_TIMEOUT, "tensor-core product: a bounded wait gave up");
    if (flags & 1) return fail(ML_ERR_DOMAIN, "tensor-core product: an element of the tall operands has |v| >= 2");
    return ML_OK;
}
}  // namespace ml

extern "C" ml_status ml_block_gram(const double *A, int64_t n, int rc, int64_t lda, const double *B, int cb,
                                   int64_t ldb, double *G, void *stream)
{
    using namespace ml;
    if (!A || !B || !G || n < 1 || rc < 1 || rc > kOzMaxRc || cb < 1 || cb > 8 || lda < rc || ldb < cb)
        return fail(ML_ERR_ARG, "ml_block_gram: null pointer or size out of range (rc <= 48, cb <= 8)");
    cudaStream_t st = (cudaStream_t)stream;
    const int nbx = oz_gram_blocks(1, n);
    DevBuf part, lay;
    ML_TRY(part.ensure((size_t)nbx * rc * cb * sizeof(double)));
    ML_TRY(lay.ensure(sizeof(int)));
    ML_CUDA(cudaMemsetAsync(lay.p, 0, sizeof(int), st));
    ML_TRY(oz_reset_error(st));
    ML_TRY(oz_gram(OzMat{A, 0, lda, 1}, rc, OzMat{B, 0, ldb, 1}, cb, lay.as<int>(), 1, n, nbx, part.as<double>(),
                   st));
    k_oz_reduce<<<(rc * cb + 127) / 128, 128, 0, st>>>(part.as<double>(), nbx, rc * cb, G);
    ML_CUDA(cudaGetLastError());
    return oz_finish(st);
}

extern "C" ml_status ml_block_update(const double *A, int64_t n, int rc, int64_t lda, const double *M, int cb,
                                     double *Y, int64_t ldy, int sub, void *stream)
{
    using namespace ml;
    if (!A || !M || !Y || n < 1 || rc < 1 || rc > kOzMaxRc || cb < 1 || lda < rc || ldy < cb)
        return fail(ML_ERR_ARG, "ml_block_update: null pointer or size out of range (rc <= 48)");
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf lay;
    ML_TRY(lay.ensure(sizeof(int)));
    ML_CUDA(cudaMemsetAsync(lay.p, 0, sizeof(int), st));
    ML_TRY(oz_reset_error(st));
    ML_TRY(oz_gemm(OzMat{A, 0, lda, 1}, rc, M, cb, 1, 0, cb, OzOut{Y, 0, ldy, 1}, lay.as<int>(), 1, n, sub != 0,
                   st));
    return oz_finish(st);
}
