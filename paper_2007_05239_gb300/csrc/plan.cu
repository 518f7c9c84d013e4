// ml_fastsum_plan and friends: one layer's set-up for Alg. 1 (Sec. 4) and its
// degrees (Sec. 2).  Device work: bounding box, grid coordinates, a stable
// LSD radix sort of the points by spreading bin, bin counts; host work (FP64):
// domain scaling, parameter choice, Fourier tables.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "ml_internal.h"

namespace ml {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

ml_status fail(ml_status st, const std::string &msg)
{
    g_err = msg;
    return st;
}

ml_status cuda_fail(cudaError_t e, const char *what, const char *file, int line)
{
    char buf[512];
    snprintf(buf, sizeof(buf), "CUDA error %s (%s) in %s at %s:%d", cudaGetErrorName(e),
             cudaGetErrorString(e), what, file, line);
    g_err = buf;
    return e == cudaErrorMemoryAllocation ? ML_ERR_OOM : ML_ERR_CUDA;
}

int sm_count()
{
    static std::atomic<int> cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 1;
    }
    int c = cached[dev].load(std::memory_order_relaxed);
    if (c <= 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            return 1;
        }
        cached[dev].store(v, std::memory_order_relaxed);   // every writer stores the same value
        c = v;
    }
    return c;
}

namespace {
constexpr size_t kCacheMin = (size_t)1 << 20;
constexpr size_t kCacheCap = (size_t)64 << 30;   // per device
std::mutex g_cache_mu;
std::map<int, std::multimap<size_t, void *>> g_cache;
std::map<int, size_t> g_cache_bytes;
}  // namespace

ml_status DevBuf::ensure(size_t nbytes)
{
    if (nbytes <= bytes && p) return ML_OK;
    release();
    if (nbytes == 0) return ML_OK;
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) {
        cudaGetLastError();
        d = -1;
    }
    if (nbytes >= kCacheMin && d >= 0) {
        // the smallest cached block of at least nbytes and at most 5/4 of it
        std::lock_guard<std::mutex> lk(g_cache_mu);
        auto &m = g_cache[d];
        auto it = m.lower_bound(nbytes);
        if (it != m.end() && it->first <= nbytes + nbytes / 4) {
            p = it->second;
            bytes = it->first;
            dev = d;
            g_cache_bytes[d] -= bytes;
            m.erase(it);
            return ML_OK;
        }
    }
    cudaError_t e = cudaMalloc(&p, nbytes);
    if (e != cudaSuccess) {
        p = nullptr;
        bytes = 0;
        return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
    }
    bytes = nbytes;
    dev = d;
    return ML_OK;
}

void DevBuf::release()
{
    if (!p) return;
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess) {
        cudaGetLastError();
        d = -1;
    }
    if (bytes >= kCacheMin && d >= 0 && d == dev) {
        // no work may still use the block when it is handed out again
        if (cudaDeviceSynchronize() == cudaSuccess) {
            std::lock_guard<std::mutex> lk(g_cache_mu);
            if (g_cache_bytes[d] + bytes <= kCacheCap) {
                g_cache[d].insert({bytes, p});
                g_cache_bytes[d] += bytes;
                p = nullptr;
                bytes = 0;
                return;
            }
        } else {
            cudaGetLastError();
        }
    }
    cudaFree(p);
    p = nullptr;
    bytes = 0;
}

namespace {
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;   // null entry: the device has no pools

cudaMemPool_t scratch_pool(int dev)
{
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) return it->second;
    cudaMemPool_t pool = nullptr;
    int ok = 0;
    if (cudaDeviceGetAttribute(&ok, cudaDevAttrMemoryPoolsSupported, dev) == cudaSuccess && ok) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;   // keep freed memory in the pool
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        } else {
            pool = nullptr;
        }
    }
    cudaGetLastError();
    g_pools[dev] = pool;
    return pool;
}
}  // namespace

ml_status StreamBuf::ensure(size_t nbytes)
{
    if (nbytes <= bytes && p) return ML_OK;
    release();
    if (nbytes == 0) return ML_OK;
    int d = 0;
    ML_CUDA(cudaGetDevice(&d));
    cudaMemPool_t pool = scratch_pool(d);
    cudaError_t e;
    if (pool) {
        e = cudaMallocFromPoolAsync(&p, nbytes, pool, st);
        pooled = true;
    } else {
        e = cudaMalloc(&p, nbytes);
        pooled = false;
    }
    if (e != cudaSuccess) {
        p = nullptr;
        bytes = 0;
        return cuda_fail(e, "scratch allocation", __FILE__, __LINE__);
    }
    bytes = nbytes;
    return ML_OK;
}

void StreamBuf::release()
{
    if (!p) return;
    if (pooled) cudaFreeAsync(p, st);
    else cudaFree(p);
    p = nullptr;
    bytes = 0;
}

// frees every cached block of the current device
ml_status release_cached()
{
    int d = 0;
    ML_CUDA(cudaGetDevice(&d));
    ML_CUDA(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (auto &kv : g_cache[d]) cudaFree(kv.second);
    g_cache[d].clear();
    g_cache_bytes[d] = 0;
    if (cudaMemPool_t pool = scratch_pool(d)) ML_CUDA(cudaMemPoolTrimTo(pool, 0));
    return ML_OK;
}

// ------------------------------------------------------------- reductions
__global__ void k_bbox(const double *__restrict__ X, int64_t n, int d, double *part)
{
    // part[block][2*a] = min, part[block][2*a+1] = max
    __shared__ double smin[3][256], smax[3][256];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < d; ++a) {
            const double x = X[i * d + a];
            lo[a] = fmin(lo[a], x);
            hi[a] = fmax(hi[a], x);
        }
    for (int a = 0; a < 3; ++a) {
        smin[a][threadIdx.x] = lo[a];
        smax[a][threadIdx.x] = hi[a];
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int a = 0; a < 3; ++a) {
                smin[a][threadIdx.x] = fmin(smin[a][threadIdx.x], smin[a][threadIdx.x + s]);
                smax[a][threadIdx.x] = fmax(smax[a][threadIdx.x], smax[a][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int a = 0; a < 3; ++a) {
            part[blockIdx.x * 6 + 2 * a] = smin[a][0];
            part[blockIdx.x * 6 + 2 * a + 1] = smax[a][0];
        }
}

// max_i ||x_i - c||^2 per block
__global__ void k_maxrad(const double *__restrict__ X, int64_t n, int d, double c0, double c1, double c2, double *part)
{
    __shared__ double s[256];
    const double c[3] = {c0, c1, c2};
    double m = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double r2 = 0.0;
        for (int a = 0; a < d; ++a) {
            const double t = X[i * d + a] - c[a];
            r2 += t * t;
        }
        m = fmax(m, r2);
    }
    s[threadIdx.x] = m;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + k]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

struct TorusMap {
    double c[3];
    double s;      // scale into the Alg. 1 domain
    int n_os, W, d;
};

// U_a = n_os (s (x_a - c_a) + 1/2): torus grid coordinate; F_a = floor(U_a - W/2) + 1
// is the first of the W taps.  Per-block min/max of F_a.
__global__ void k_first_tap_range(const double *__restrict__ X, int64_t n, TorusMap tm, long long *part)
{
    __shared__ long long smin[3][256], smax[3][256];
    long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < tm.d; ++a) {
            const double U = tm.n_os * (tm.s * (X[i * tm.d + a] - tm.c[a]) + 0.5);
            const long long F = (long long)floor(U - 0.5 * tm.W) + 1;
            lo[a] = min(lo[a], F);
            hi[a] = max(hi[a], F);
        }
    for (int a = 0; a < 3; ++a) {
        smin[a][threadIdx.x] = lo[a];
        smax[a][threadIdx.x] = hi[a];
    }
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k)
            for (int a = 0; a < 3; ++a) {
                smin[a][threadIdx.x] = min(smin[a][threadIdx.x], smin[a][threadIdx.x + k]);
                smax[a][threadIdx.x] = max(smax[a][threadIdx.x], smax[a][threadIdx.x + k]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int a = 0; a < 3; ++a) {
            part[blockIdx.x * 6 + 2 * a] = smin[a][0];
            part[blockIdx.x * 6 + 2 * a + 1] = smax[a][0];
        }
}

// local coordinate relative to the point's bin origin, and the sort key:
// bin * cells + the first-tap cell within the bin (cells = B^d), so that the
// points of a bin are ordered by cell and the points a warp spreads together
// usually share their taps (cells = 1: by bin only)
struct KeyArgs {
    TorusMap tm;
    int s0[3];
    int B;
    int nb0, nb1;
    uint32_t cells;
};

__global__ void k_keys(const double *__restrict__ X, int64_t n, KeyArgs ka, double *urel, uint32_t *keys, int *idx)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int bcoord[3] = {0, 0, 0}, ccoord[3] = {0, 0, 0};
        for (int a = 0; a < ka.tm.d; ++a) {
            const double U = ka.tm.n_os * (ka.tm.s * (X[i * ka.tm.d + a] - ka.tm.c[a]) + 0.5);
            const double u = U - ka.s0[a];                        // local active-grid coordinate
            const long long f0 = (long long)floor(u - 0.5 * ka.tm.W) + 1;  // >= 0 by construction of s0
            const int b = (int)(f0 / ka.B);
            bcoord[a] = b;
            ccoord[a] = (int)(f0 - (long long)b * ka.B);
            urel[i * ka.tm.d + a] = u - (double)b * ka.B;
        }
        const uint32_t bin = (uint32_t)((bcoord[2] * ka.nb1 + bcoord[1]) * ka.nb0 + bcoord[0]);
        const uint32_t cell = ka.cells > 1 ? (uint32_t)((ccoord[2] * ka.B + ccoord[1]) * ka.B + ccoord[0]) : 0u;
        keys[i] = bin * ka.cells + cell;
        idx[i] = (int)i;
    }
}

template <typename T>
__global__ void k_gather_coords(const double *__restrict__ urel, const int *__restrict__ perm, int64_t n, int d, T *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t src = perm[i];
        for (int a = 0; a < d; ++a) out[i * d + a] = (T)urel[src * d + a];
    }
}

// First sorted position of every bin (bin = key / cells, keys ascending):
// starts[b] for b in 0..nbins, starts[nbins] = n.  Position i writes the
// starts of the bins from just after its predecessor's bin up to its own, so
// every entry (empty bins included) is written exactly once: no atomics
// (a global atomic count on a few dozen bins serialised on their addresses).
__global__ void k_bin_starts(const uint32_t *__restrict__ keys, int64_t n, uint32_t cells, int nbins, int *starts)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
        const int b = i < n ? (int)(keys[i] / cells) : nbins;
        const int bp = i > 0 ? (int)(keys[i - 1] / cells) : -1;
        for (int bb = bp + 1; bb <= b; ++bb) starts[bb] = (int)i;
    }
}

// FP64 window weights of every point (plan time), stored as double-word
// pairs: wts[i][a][q] = phi_n(x - o - q),
// o = floor(x - W/2) + 1 the first tap
__global__ void k_window_table_f64(const double *__restrict__ coords, int64_t n, int d, int W, double h2, double b,
                                   double norm2, float2 *wts)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * d * W;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(e % W);
        const int64_t ia = e / W;   // point * d + dim
        const double x = coords[ia];
        const double fl = floor(x - 0.5 * W);
        wts[e] = dw_split(kb_weight(x - fl - 1.0 - (double)q, h2, b, norm2));
    }
}


// packed first tap of every point: o_a = floor(u_a - W/2) + 1 in [0, B]
__global__ void k_first_taps(const double *__restrict__ coords, int64_t n, int d, int W, int *offs)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int packed = 0;
        for (int a = 0; a < d; ++a) packed |= ((int)floor(coords[i * d + a] - 0.5 * W) + 1) << (10 * a);
        offs[i] = packed;
    }
}

// ------------------------------------------------------------ radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_TILE = 4096;

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint32_t *__restrict__ keys, int64_t n, int shift,
                                                        uint32_t *hist, int nblk)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int e = threadIdx.x; e < RS_TILE; e += RS_THREADS) {
        const int64_t i = base + e;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of `total` entries in place, in three launches: per-chunk
// sums (one CTA per chunk of `chunk` entries, coalesced), a scan of the chunk
// sums in one CTA, and the chunks' own scans from their offsets (tiles of
// 1024 entries, Hillis-Steele in shared memory).  Integer sums: exact.
constexpr int RS_SCAN_THREADS = 1024;

__device__ __forceinline__ uint32_t block_sum_u32(uint32_t v)
{
    __shared__ uint32_t red[RS_SCAN_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    uint32_t t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    __syncthreads();
    return t;
}

// inclusive scan of one value per thread over the block (blockDim.x = 1024)
__device__ __forceinline__ uint32_t block_incl_scan_u32(uint32_t v)
{
    __shared__ uint32_t wsum[RS_SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        if (lane < (int)(blockDim.x >> 5)) wsum[lane] = w;
    }
    __syncthreads();
    const uint32_t r = v + (warp > 0 ? wsum[warp - 1] : 0u);
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(RS_SCAN_THREADS) k_scan_sums(const uint32_t *__restrict__ a, int64_t total,
                                                               int64_t chunk, uint32_t *sums)
{
    const int64_t lo = (int64_t)blockIdx.x * chunk, hi = min(total, lo + chunk);
    uint32_t s = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += a[i];
    s = block_sum_u32(s);
    if (threadIdx.x == 0) sums[blockIdx.x] = s;
}

// exclusive scan of the g <= 1024 chunk sums, in place
__global__ void __launch_bounds__(RS_SCAN_THREADS) k_scan_top(uint32_t *sums, int g)
{
    const uint32_t v = (int)threadIdx.x < g ? sums[threadIdx.x] : 0u;
    const uint32_t incl = block_incl_scan_u32(v);
    if ((int)threadIdx.x < g) sums[threadIdx.x] = incl - v;
}

__global__ void __launch_bounds__(RS_SCAN_THREADS) k_scan_apply(uint32_t *a, int64_t total, int64_t chunk,
                                                                const uint32_t *__restrict__ sums)
{
    const int64_t lo = (int64_t)blockIdx.x * chunk, hi = min(total, lo + chunk);
    uint32_t run = sums[blockIdx.x];
    for (int64_t t0 = lo; t0 < hi; t0 += blockDim.x) {
        const int64_t i = t0 + threadIdx.x;
        const uint32_t v = i < hi ? a[i] : 0u;
        const uint32_t incl = block_incl_scan_u32(v);
        if (i < hi) a[i] = run + incl - v;
        // the tile's total, from the last thread's inclusive value
        __shared__ uint32_t tile_total;
        if (threadIdx.x == blockDim.x - 1) tile_total = incl;
        __syncthreads();
        run += tile_total;
        __syncthreads();
    }
}

static ml_status exclusive_scan(uint32_t *a, int64_t total, StreamBuf &sums, cudaStream_t st)
{
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(RS_SCAN_THREADS, (total + 4095) / 4096));
    const int64_t chunk = (total + g - 1) / g;
    ML_TRY(sums.ensure((size_t)g * sizeof(uint32_t)));
    k_scan_sums<<<g, RS_SCAN_THREADS, 0, st>>>(a, total, chunk, sums.as<uint32_t>());
    k_scan_top<<<1, RS_SCAN_THREADS, 0, st>>>(sums.as<uint32_t>(), g);
    k_scan_apply<<<g, RS_SCAN_THREADS, 0, st>>>(a, total, chunk, sums.as<uint32_t>());
    return ML_OK;
}

// Stable scatter: items of a block are ranked in input order, 256 per round;
// within a round the rank of an item among equal digits is (count in earlier
// warps) + (count in earlier lanes), the latter from __match_any_sync.
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint32_t *__restrict__ kin, const int *__restrict__ vin,
                                                           uint32_t *kout, int *vout, int64_t n, int shift,
                                                           const uint32_t *__restrict__ scanned, int nblk)
{
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcnt[RS_THREADS / 32][256];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    base[tid] = scanned[(int64_t)tid * nblk + blockIdx.x];
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < RS_TILE / RS_THREADS; ++r) {
        const int64_t item = (int64_t)blockIdx.x * RS_TILE + (int64_t)r * RS_THREADS + tid;
        const bool valid = item < n;
        const uint32_t key = valid ? kin[item] : 0u;
        const uint32_t digit = valid ? ((key >> shift) & 255u) : 256u;
        for (int w = 0; w < RS_THREADS / 32; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        const unsigned mask = __match_any_sync(0xffffffffu, digit);
        const uint32_t lrank = __popc(mask & lt_mask);
        if (valid && lrank == 0) wcnt[warp][digit] = __popc(mask);
        __syncthreads();
        uint32_t run = 0;
        for (int w = 0; w < RS_THREADS / 32; ++w) {
            const uint32_t t = wcnt[w][tid];
            wcnt[w][tid] = run;
            run += t;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = base[digit] + wcnt[warp][digit] + lrank;
            kout[pos] = key;
            vout[pos] = vin[item];
        }
        __syncthreads();
        base[tid] += run;
        __syncthreads();
    }
}

ml_status radix_sort(uint32_t *keys, int *vals, uint32_t *keys2, int *vals2, int64_t n, int bits,
                     cudaStream_t st, int **result_vals)
{
    const int nblk = (int)((n + RS_TILE - 1) / RS_TILE);
    StreamBuf hist(st), sums(st);
    ML_TRY(hist.ensure((size_t)256 * nblk * sizeof(uint32_t)));
    uint32_t *ka = keys, *kb = keys2;
    int *va = vals, *vb = vals2;
    for (int shift = 0; shift < bits; shift += 8) {
        { ProfScope pr_("plan", st);
        k_rs_hist<<<nblk, RS_THREADS, 0, st>>>(ka, n, shift, hist.as<uint32_t>(), nblk);
        }
        { ProfScope pr_("plan", st);
        ML_TRY(exclusive_scan(hist.as<uint32_t>(), (int64_t)256 * nblk, sums, st));
        }
        { ProfScope pr_("plan", st);
        k_rs_scatter<<<nblk, RS_THREADS, 0, st>>>(ka, va, kb, vb, n, shift, hist.as<uint32_t>(), nblk);
        }
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    ML_CUDA(cudaGetLastError());
    ML_CUDA(cudaStreamSynchronize(st));
    hist.release();
    *result_vals = va;
    return ML_OK;
}

// iperm[perm[s]] = s
__global__ void k_invert_perm(const int *__restrict__ perm, int64_t n, int *iperm)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
        iperm[perm[s]] = (int)s;
}

__global__ void k_copy_int(const int *src, int *dst, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// D^{-1/2} and a validity flag (degree not positive or not finite)
// D^{-1/2}, the validity flag, and per-block (min, max) of the degrees in
// range[2 * blockIdx.x] (blockDim.x = 256)
__global__ void k_dinv(const double *__restrict__ deg, int64_t n, double *dinv, int *bad, double *range)
{
    __shared__ double smin[256], smax[256];
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = deg[i];
        lo = fmin(lo, v);
        hi = fmax(hi, v);
        if (!(v > 0.0) || !isfinite(v)) {
            atomicExch(bad, 1);
            dinv[i] = 0.0;
        } else {
            dinv[i] = 1.0 / sqrt(v);
        }
    }
    smin[threadIdx.x] = lo;
    smax[threadIdx.x] = hi;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) {
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + k]);
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + k]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        range[2 * blockIdx.x] = smin[0];
        range[2 * blockIdx.x + 1] = smax[0];
    }
}

static int grid_for(int64_t n, int threads = 256);

// bounding box of n x d points (device), synchronises the stream
ml_status bounding_box(const double *points, int64_t n, int d, cudaStream_t st, double lo[3], double hi[3])
{
    const int nblk = grid_for(n);
    StreamBuf part(st);
    ML_TRY(part.ensure((size_t)nblk * 6 * sizeof(double)));
    {
        ProfScope pr_("plan", st);
        k_bbox<<<nblk, 256, 0, st>>>(points, n, d, part.as<double>());
    }
    ML_CUDA(cudaGetLastError());
    std::vector<double> hp((size_t)nblk * 6);
    ML_CUDA(cudaMemcpyAsync(hp.data(), part.p, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    ML_CUDA(cudaStreamSynchronize(st));
    for (int a = 0; a < 3; ++a) {
        lo[a] = 0.0;
        hi[a] = 0.0;
    }
    for (int a = 0; a < d; ++a) {
        lo[a] = INFINITY;
        hi[a] = -INFINITY;
        for (int b = 0; b < nblk; ++b) {
            lo[a] = std::min(lo[a], hp[b * 6 + 2 * a]);
            hi[a] = std::max(hi[a], hp[b * 6 + 2 * a + 1]);
        }
    }
    return ML_OK;
}

static int grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, sm_count() * 16));
}

// ---------------------------------------------------------- window polynomials
// phi_n(t) = norm (e^{bs} - e^{-bs}) / s, s = sqrt(h^2 - t^2), in FP64
static double kb_phi(double t, double h, double b, double norm)
{
    const double s = std::sqrt(std::max(h * h - t * t, 0.0)), bs = b * s;
    if (bs < 1e-4) return norm * 2.0 * b * (1.0 + bs * bs / 6.0);
    return norm * 2.0 * std::sinh(bs) / s;
}

// FP32 form: for every tap q < ceil(W/2) the polynomial of degree 9 in
// u = f - 1/2 that interpolates phi_n(W/2 - 1 - q + f), f in [0, 1), at the 10
// Chebyshev points of the unit interval (monomial coefficients from the
// Vandermonde system, Gaussian elimination with partial pivoting in FP64).
// The window is even, so tap W-1-q is the same polynomial at -u and is not
// fitted; the middle tap of an odd W keeps its even coefficients only (its
// odd ones are rounding noise).  Stored per row: the even coefficients, then
// the odd ones (window_row_poly).  The window is a function of
// s^2 = h^2 - t^2 whose series has only positive terms (an entire function
// of t), so the interpolant converges fast: the check on 2001 points of every
// tap, mirrored ones included, with the coefficients rounded to FP32, must
// stay below 1e-7 of the window's peak.
static ml_status fit_window_poly(ml_plan_s *p)
{
    constexpr int K = kPolyTerms;
    static_assert(sizeof(p->kbp) == sizeof(float) * kPolyW * kPolyStride, "window polynomial table size");
    static_assert(K == 10 && kPolyStride >= K, "five even and five odd coefficients per row");
    const int W = p->W;
    if (W > 16) return fail(ML_ERR_ARG, "FP32 window wider than 16 taps");
    const double h = 0.5 * W, b = p->kb_shape, nm = p->kb_norm;
    const double peak = kb_phi(0.0, h, b, nm);
    double worst = 0.0;
    std::fill(p->kbp, p->kbp + kPolyW * kPolyStride, 0.0f);
    for (int q = 0; q < (W + 1) / 2; ++q) {
        double V[K][K + 1];
        for (int j = 0; j < K; ++j) {
            const double u = 0.5 * std::cos((2 * j + 1) * M_PI / (2.0 * K));
            double pw = 1.0;
            for (int k = 0; k < K; ++k) {
                V[j][k] = pw;
                pw *= u;
            }
            V[j][K] = kb_phi(h - 1.0 - q + 0.5 + u, h, b, nm);
        }
        for (int c = 0; c < K; ++c) {
            int piv = c;
            for (int r = c + 1; r < K; ++r)
                if (std::fabs(V[r][c]) > std::fabs(V[piv][c])) piv = r;
            for (int k = 0; k <= K; ++k) std::swap(V[c][k], V[piv][k]);
            for (int r = c + 1; r < K; ++r) {
                const double f = V[r][c] / V[c][c];
                for (int k = c; k <= K; ++k) V[r][k] -= f * V[c][k];
            }
        }
        double coef[K];
        for (int c = K - 1; c >= 0; --c) {
            double v = V[c][K];
            for (int k = c + 1; k < K; ++k) v -= V[c][k] * coef[k];
            coef[c] = v / V[c][c];
        }
        const bool middle = 2 * q + 1 == W;
        float *row = p->kbp + q * kPolyStride;
        for (int j = 0; j < K / 2; ++j) {
            row[j] = (float)coef[2 * j];
            row[K / 2 + j] = middle ? 0.0f : (float)coef[2 * j + 1];
        }
        for (int e = 0; e <= 2000; ++e) {
            const double u = -0.5 + e / 2000.0, u2 = u * u;
            double ev = 0.0, od = 0.0;
            for (int j = K / 2 - 1; j >= 0; --j) {
                ev = ev * u2 + row[j];
                od = od * u2 + row[K / 2 + j];
            }
            worst = std::max(worst, std::fabs(ev + u * od - kb_phi(h - 1.0 - q + 0.5 + u, h, b, nm)));
            const int qm = W - 1 - q;   // the mirrored tap
            worst = std::max(worst, std::fabs(ev - u * od - kb_phi(h - 1.0 - qm + 0.5 + u, h, b, nm)));
        }
    }
    if (!(worst <= 1e-7 * peak))
        return fail(ML_ERR_DOMAIN, "window polynomial fit error " + std::to_string(worst / peak) + " of the peak");
    return ML_OK;
}

// ---------------------------------------------------------- parameters
// Window width W and oversampling sigma_os for a target error.  The
// Kaiser-Bessel window's error falls like exp(-pi W sqrt(1 - 1/sigma_os));
// measured worst cases (coincident or tightly clustered points, where the
// window errors add up coherently; sigma_os = 2: W = 5 -> 1.4e-4, W = 7 ->
// 1.2e-6) fit 9 exp(-pi W sqrt(1 - 1/sigma_os)).  Take the narrowest
// available width that reaches target/2 at sigma_os <= 3, then the smallest
// oversampling in {2, 2.5, 3} that reaches it with that width: the taps (W^d
// per point) dominate the cost, the grid grows only with sigma_os^d.
static double window_error(int W, double sig_os) { return 9.0 * std::exp(-M_PI * W * std::sqrt(1.0 - 1.0 / sig_os)); }

static void auto_window(double target, int *W_out, double *sig_out)
{
    static const int widths[] = {4, 5, 6, 7, 8, 10, 12, 14, 16};
    int W = 16;
    for (int w : widths)
        if (window_error(w, 3.0) <= 0.5 * target) {
            W = w;
            break;
        }
    double sig = 3.0;
    for (double s : {2.0, 2.5, 3.0})
        if (window_error(W, s) <= 0.5 * target) {
            sig = s;
            break;
        }
    *W_out = W;
    *sig_out = sig;
}

// automatic bandwidth for a box-domain layer from its largest bounding-box
// extent (the scaling of the box reading, then auto_N)
int auto_bandwidth_box(double sigma, double box, int d, double target);

static int auto_N(double sigma_s, double target)
{
    const double half = std::sqrt(std::log(10.0 / target)) / (M_PI * sigma_s);
    int N = 2 * (int)std::ceil(half);
    return std::max(N, 8);
}

int auto_bandwidth_box(double sigma, double box, int d, double target)
{
    double h = 0.5 * box;
    if (!(h > 0)) h = sigma;
    const double aa = std::min(0.25, 1.0 / (2.0 + (sigma / h) * std::sqrt(std::log(2.0 * d / (0.1 * target)))));
    return auto_N(aa / h * sigma, target);
}

// FP64 form: the largest B whose padded tile (B + W)^d of 8-byte cells stays
// within 23.5 KB per vector (with the staged inputs, several CTAs per SM),
// doubling the budget (up to 188 KB) while that leaves B < 4
static int choose_bin_f64(int d, int W)
{
    int b = 1;
    for (double kb = 23.5; kb <= 188.0; kb *= 2.0) {
        const int Pt = (int)std::floor(std::pow(kb * 1024.0 / 8.0, 1.0 / d) + 1e-9);
        b = Pt - W;
        if (d == 1) b = std::min(b, 512);
        if (b >= 4) break;
    }
    return std::max(b, 1);
}

// FP32 form: the largest B whose padded tile (B + W)^d of 8-byte cells stays
// within 48 KB per vector
static int choose_bin(int d, int W)
{
    const int budget = 48 * 1024 / 8;
    int Pt = 1;
    while (true) {
        int64_t v = 1;
        for (int a = 0; a < d; ++a) v *= (Pt + 1);
        if (v > budget) break;
        ++Pt;
        if (Pt >= 1024) break;
    }
    int B = Pt - W;
    if (d == 1) B = std::min(B, 512);
    return std::max(B, 1);
}

template <typename T>
static ml_status upload(DevBuf &buf, const std::vector<double> &src)
{
    std::vector<T> tmp(src.begin(), src.end());
    ML_TRY(buf.ensure(tmp.size() * sizeof(T)));
    ML_CUDA(cudaMemcpy(buf.p, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
    return ML_OK;
}

// FP64 form: tables as double-word pairs (hi = x rounded to float, lo = the
// remainder rounded to float)
static ml_status upload_dw(DevBuf &buf, const std::vector<double> &src)
{
    std::vector<float> tmp(2 * src.size());
    for (size_t i = 0; i < src.size(); ++i) {
        const float hi = (float)src[i];
        tmp[2 * i] = hi;
        tmp[2 * i + 1] = (float)(src[i] - (double)hi);
    }
    ML_TRY(buf.ensure(tmp.size() * sizeof(float)));
    ML_CUDA(cudaMemcpy(buf.p, tmp.data(), tmp.size() * sizeof(float), cudaMemcpyHostToDevice));
    return ML_OK;
}

void workspace_bytes(const ml_plan_s *p, int nv, size_t *scratch, size_t *work)
{
    if (p->dense) {   // a dense product needs no scratch
        *scratch = 0;
        *work = 0;
        return;
    }
    const size_t ts = p->prec == ML_F32 ? 4 : 8;
    const GridGeom &g = p->g;
    // subproblem tiles, then one tile per group of subproblems, then (FP32)
    // the box of cells each subproblem tile was written in (tile_boxes)
    *scratch = (size_t)(p->nsub + p->ngroups) * g.tile_cells() * nv * ts;
    if (p->prec == ML_F32) *scratch = ((*scratch + 15) & ~(size_t)15) + (size_t)p->nsub * 16;
    // transform stages: extents go from L to K one dim at a time and back
    int64_t mx = 1;
    for (int stage = 0; stage <= p->d; ++stage) {
        int64_t v = 1;
        for (int a = 0; a < p->d; ++a) v *= (a < stage ? g.K : g.L[a]);
        mx = std::max(mx, v);
    }
    *work = (size_t)mx * nv * ts;
}

ml_status ensure_workspace(ml_plan_s *p, int nv)
{
    size_t sb = 0, wb = 0;
    workspace_bytes(p, nv, &sb, &wb);
    ML_TRY(p->scratch.ensure(sb));
    ML_TRY(p->work[0].ensure(wb));
    ML_TRY(p->work[1].ensure(wb));
    ML_TRY(p->status.ensure(64));
    return ML_OK;
}

// Laplacian (ball domain always): window, cells across the inner region c,
// bandwidth N, eps_I = c/N and eps_B = max(1/16, eps_I) unless given; the
// scaling; b_l of K_R; and the measured max |K_RF - K_R| on probe distances.
// Above target/2 the automatic choices widen the inner region (c += 2, or a
// larger N when eps_I is fixed) and try again.
static ml_status laplace_setup(ml_plan_s *p, const double *points, int nblk, StreamBuf &part, cudaStream_t st)
{
    const int64_t n = p->n;
    const int d = p->d;
    {
        ProfScope pr_("plan", st);
        k_maxrad<<<nblk, 256, 0, st>>>(points, n, d, p->center[0], p->center[1], p->center[2], part.as<double>());
    }
    ML_CUDA(cudaGetLastError());
    std::vector<double> hp(nblk);
    ML_CUDA(cudaMemcpyAsync(hp.data(), part.p, nblk * sizeof(double), cudaMemcpyDeviceToHost, st));
    ML_CUDA(cudaStreamSynchronize(st));
    double r2 = 0.0;
    for (int b = 0; b < nblk; ++b) r2 = std::max(r2, hp[b]);
    double rmax = std::sqrt(r2);
    if (!(rmax > 0)) rmax = p->sigma;
    if (p->p_reg == 0) p->p_reg = 8;
    if (p->W == 0) {
        double sig_os = 2.0;
        auto_window(p->target, &p->W, &sig_os);
        if (p->sig_os_req == 0) p->sig_os_req = sig_os;
    }
    const bool fixN = p->N > 0, fixI = p->eps_I_req > 0;
    int c = laplace_cells(p->target);
    int N = p->N;
    for (int attempt = 0; attempt < 12; ++attempt) {
        double eI;
        if (fixI) {
            eI = p->eps_I_req;
            if (!fixN) N = std::max(16, 2 * (int)std::ceil(0.5 * c / eI));
        } else {
            if (!fixN) N = laplace_bandwidth(n, d, c, p->W, p->prec);
            eI = (double)c / N;
        }
        if (N > kMaxN)
            return fail(ML_ERR_DOMAIN, "Laplacian: bandwidth N=" + std::to_string(N) + " needed for eps_I beyond the limit");
        const double eB = p->eps_B_req > 0 ? p->eps_B_req : std::max(1.0 / 16, eI);
        if (!(eI < 0.5 - eB)) return fail(ML_ERR_ARG, "Laplacian: eps_I must stay below 1/2 - eps_B");
        p->N = N;
        p->eps_I = eI;
        p->eps_B = eB;
        p->scale = (0.25 - 0.5 * eB) / rmax;
        p->domain = 1;
        p->sigma_s = p->scale * p->sigma;
        LaplaceReg g;
        if (!laplace_reg_init(p->sigma_s, eB, eI, p->p_reg, g))
            return fail(ML_ERR_DOMAIN, "Laplacian: regulariser system is singular");
        ML_TRY(laplace_fourier(p, g, st));
        p->kernel_err = kernel_probe_error(p->bhat, N, d, g, d == 3 ? 48 : 96);
        p->nf_poly = g.c;
        if (p->kernel_err <= 0.5 * p->target) return ML_OK;
        if ((fixN && fixI) || c >= 24) break;
        c += 2;
    }
    char buf[160];
    snprintf(buf, sizeof buf, "Laplacian: kernel approximation error %.3g above target/2 (N=%d, eps_I=%.4g)",
             p->kernel_err, p->N, p->eps_I);
    return fail(ML_ERR_DOMAIN, buf);
}

static ml_status plan_impl(ml_plan_s *p, const double *points, cudaStream_t st)
{
    const int64_t n = p->n;
    const int d = p->d;
    // ---- bounding box
    const int nblk = grid_for(n);
    StreamBuf part(st);
    ML_TRY(part.ensure((size_t)nblk * 6 * sizeof(double)));
    { ProfScope pr_("plan", st);
    k_bbox<<<nblk, 256, 0, st>>>(points, n, d, part.as<double>());
    }
    ML_CUDA(cudaGetLastError());
    std::vector<double> hp((size_t)nblk * 6);
    ML_CUDA(cudaMemcpyAsync(hp.data(), part.p, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    ML_CUDA(cudaStreamSynchronize(st));
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
        lo[a] = INFINITY;
        hi[a] = -INFINITY;
        for (int b = 0; b < nblk; ++b) {
            lo[a] = std::min(lo[a], hp[b * 6 + 2 * a]);
            hi[a] = std::max(hi[a], hp[b * 6 + 2 * a + 1]);
        }
        if (!std::isfinite(lo[a]) || !std::isfinite(hi[a])) return fail(ML_ERR_ARG, "points contain non-finite values");
        p->center[a] = 0.5 * (lo[a] + hi[a]);
    }
    // ---- domain scaling (isotropic, exact for W)
    if (p->kernel == ML_KERNEL_LAPLACE) {
        ML_TRY(laplace_setup(p, points, nblk, part, st));
    } else if (p->eps_B > 0) {
        { ProfScope pr_("plan", st);
        k_maxrad<<<nblk, 256, 0, st>>>(points, n, d, p->center[0], p->center[1], p->center[2], part.as<double>());
        }
        ML_CUDA(cudaGetLastError());
        ML_CUDA(cudaMemcpyAsync(hp.data(), part.p, nblk * sizeof(double), cudaMemcpyDeviceToHost, st));
        ML_CUDA(cudaStreamSynchronize(st));
        double r2 = 0.0;
        for (int b = 0; b < nblk; ++b) r2 = std::max(r2, hp[b]);
        double rmax = std::sqrt(r2);
        if (!(rmax > 0)) rmax = p->sigma;
        p->scale = (0.25 - 0.5 * p->eps_B) / rmax;
        p->domain = 1;
    } else {
        double h = 0.0;
        for (int a = 0; a < d; ++a) h = std::max(h, 0.5 * (hi[a] - lo[a]));
        if (!(h > 0)) h = p->sigma;
        const double eps_wrap = 0.1 * p->target;
        const double aa = std::min(0.25, 1.0 / (2.0 + (p->sigma / h) * std::sqrt(std::log(2.0 * d / eps_wrap))));
        p->scale = aa / h;
        p->domain = 0;
    }
    p->sigma_s = p->scale * p->sigma;
    // ---- parameters
    if (p->N == 0) p->N = auto_N(p->sigma_s, p->target);
    double sig_os = p->sig_os_req > 0 ? p->sig_os_req : 2.0;
    if (p->W == 0) auto_window(p->target, &p->W, &sig_os);
    p->m = p->W / 2;
    if (p->N > kMaxN)
        return fail(ML_ERR_DOMAIN, "bandwidth N=" + std::to_string(p->N) + " needed for the target exceeds the limit");
    p->n_os = 2 * (int)std::ceil(0.5 * sig_os * p->N);   // even torus size
    p->kb_shape = M_PI * (2.0 - (double)p->N / p->n_os);  // b = pi (2 - 1/sigma_os)
    {
        const double b = p->kb_shape, h = 0.5 * p->W;
        p->kb_norm = h * std::exp(-b * h) / (1.0 - std::exp(-2.0 * b * h));
    }
    if (p->prec == ML_F32) ML_TRY(fit_window_poly(p));
    // ---- active grid
    TorusMap tm;
    for (int a = 0; a < 3; ++a) tm.c[a] = p->center[a];
    tm.s = p->scale;
    tm.n_os = p->n_os;
    tm.W = p->W;
    tm.d = d;
    StreamBuf lpart(st);
    ML_TRY(lpart.ensure((size_t)nblk * 6 * sizeof(long long)));
    { ProfScope pr_("plan", st);
    k_first_tap_range<<<nblk, 256, 0, st>>>(points, n, tm, lpart.as<long long>());
    }
    ML_CUDA(cudaGetLastError());
    std::vector<long long> lp((size_t)nblk * 6);
    ML_CUDA(cudaMemcpyAsync(lp.data(), lpart.p, lp.size() * sizeof(long long), cudaMemcpyDeviceToHost, st));
    ML_CUDA(cudaStreamSynchronize(st));
    GridGeom &g = p->g;
    g.d = d;
    g.W = p->W;
    g.K = p->N + 1;
    for (int a = 0; a < 3; ++a) {
        g.L[a] = 1;
        g.nb[a] = 1;
    }
    for (int a = 0; a < d; ++a) {
        long long fmin = LLONG_MAX, fmax = LLONG_MIN;
        for (int b = 0; b < nblk; ++b) {
            fmin = std::min(fmin, lp[b * 6 + 2 * a]);
            fmax = std::max(fmax, lp[b * 6 + 2 * a + 1]);
        }
        p->s0[a] = (int)fmin;
        // +1: an FP32 coordinate just below an integer may round up, moving
        // its first tap one cell to the right
        g.L[a] = (int)(fmax - fmin) + p->W + 1;
    }
    if (p->bin_req > 0) {
        g.B = p->bin_req;
    } else if (p->prec == ML_F32) {
        g.B = choose_bin(d, p->W);
    } else {
        g.B = choose_bin_f64(d, p->W);
    }
    {
        // a grid that fits in one bin: one bin, and a tile the size of the grid
        int Lmax = 1;
        for (int a = 0; a < d; ++a) Lmax = std::max(Lmax, g.L[a]);
        if (g.B + p->W > Lmax) {
            g.B = Lmax;
            g.Pt = Lmax;                // every tap index is < L <= Pt
        } else {
            g.Pt = g.B + p->W;          // first tap offset in [0, B], W taps
        }
    }
    g.R = 1 + (p->W - 1) / g.B;         // bins below that reach into a bin
    for (int a = 0; a < d; ++a) g.nb[a] = (g.L[a] + g.B - 1) / g.B;
    {
        // one shared tile per CTA (FP32: 4-byte cells; FP64: two 4-byte
        // fixed-point planes) plus, in FP64, the staged inputs of a subproblem
        const int64_t tc = g.tile_cells();
        const int64_t need1 = p->prec == ML_F32 ? tc * 4 : tc * 8 + (int64_t)kSubPoints * 8;
        if (need1 > 200 * 1024)
            return fail(ML_ERR_ARG, "bin edge " + std::to_string(g.B) + " gives a tile beyond the shared-memory budget");
        if (p->prec == ML_F32) {
            p->vp = (int)std::min<int64_t>(kMaxVec, std::max<int64_t>(1, (200 * 1024) / (tc * 4)));
            // when the spreading's warp slots (d = 3 row products, d = 2 one tap
            // per lane) fit next to the tile for one vector, keep every pass
            // width within that budget, so that all passes take the same
            // arithmetic
            auto fits = [&](int v) {
                return (((size_t)tc * 4 * v + 15) & ~(size_t)15) + warp_slot_bytes(d, p->W, v) <= kRowSpreadBudget;
            };
            if (warp_slots_on(d, p->W) && fits(1))
                while (p->vp > 1 && !fits(p->vp)) --p->vp;
        } else {
            int vp = 1;
            for (int v = kMaxVec; v >= 1; --v)
                if ((int64_t)tc * 8 * v + (int64_t)kSubPoints * 8 * v <= 200 * 1024) {
                    vp = v;
                    break;
                }
            p->vp = vp;
        }
    }
    // ---- keys, sort
    StreamBuf urel(st), keys(st), keys2(st), idx(st), idx2(st);
    ML_TRY(urel.ensure((size_t)n * d * sizeof(double)));
    ML_TRY(keys.ensure((size_t)n * 4));
    ML_TRY(keys2.ensure((size_t)n * 4));
    ML_TRY(idx.ensure((size_t)n * 4));
    ML_TRY(idx2.ensure((size_t)n * 4));
    KeyArgs ka;
    ka.tm = tm;
    for (int a = 0; a < 3; ++a) ka.s0[a] = p->s0[a];
    ka.B = g.B;
    ka.nb0 = g.nb[0];
    ka.nb1 = g.nb[1];
    const int64_t nbins = g.nbins();
    {
        // FP32 layers of several bins are ordered by cell within each bin (the
        // warp-summed spreading of points that share their taps).  A layer whose
        // grid is one tile keeps its points in input order (the batched
        // interpolation sums all such layers point by point in that order); the
        // FP64 form keeps the input order within a bin (its (point, slab) items
        // would meet the same cells in neighbouring lanes)
        int64_t cells = 1;
        for (int a = 0; a < d; ++a) cells *= g.B;
        ka.cells = (p->prec == ML_F32 && nbins > 1 && nbins * cells < ((int64_t)1 << 32)) ? (uint32_t)cells : 1u;
    }
    { ProfScope pr_("plan", st);
    k_keys<<<grid_for(n), 256, 0, st>>>(points, n, ka, urel.as<double>(), keys.as<uint32_t>(), idx.as<int>());
    }
    ML_CUDA(cudaGetLastError());
    int bits = 0;
    while ((1LL << bits) < nbins * (int64_t)ka.cells) ++bits;
    int *sorted_idx = nullptr;
    ML_TRY(radix_sort(keys.as<uint32_t>(), idx.as<int>(), keys2.as<uint32_t>(), idx2.as<int>(), n, bits, st,
                      &sorted_idx));
    // the sorted keys sit in the buffer paired with sorted_idx
    const uint32_t *sorted_keys = (sorted_idx == idx.as<int>()) ? keys.as<uint32_t>() : keys2.as<uint32_t>();
    ML_TRY(p->perm.ensure((size_t)n * 4));
    { ProfScope pr_("plan", st);
    k_copy_int<<<grid_for(n), 256, 0, st>>>(sorted_idx, p->perm.as<int>(), n);
    }
    ML_TRY(p->iperm.ensure((size_t)n * 4));
    { ProfScope pr_("plan", st);
    k_invert_perm<<<grid_for(n), 256, 0, st>>>(p->perm.as<int>(), n, p->iperm.as<int>());
    }
    const size_t ts = p->prec == ML_F32 ? 4 : 8;
    ML_TRY(p->coords.ensure((size_t)n * d * ts));
    if (p->prec == ML_F32)
        { ProfScope pr_("plan", st);
        k_gather_coords<float><<<grid_for(n), 256, 0, st>>>(urel.as<double>(), p->perm.as<int>(), n, d, p->coords.as<float>());
        }
    else
        { ProfScope pr_("plan", st);
        k_gather_coords<double><<<grid_for(n), 256, 0, st>>>(urel.as<double>(), p->perm.as<int>(), n, d, p->coords.as<double>());
        }
    ML_CUDA(cudaGetLastError());
    if (p->prec == ML_F64) {
        // FP64 window weights, once per plan
        ML_TRY(p->wts.ensure((size_t)n * d * p->W * sizeof(float2)));
        ProfScope pr_("plan", st);
        k_window_table_f64<<<grid_for(n * d * p->W), 256, 0, st>>>(
            p->coords.as<double>(), n, d, p->W, 0.25 * p->W * p->W, p->kb_shape, p->kb_norm, p->wts.as<float2>());
        ML_TRY(p->offs.ensure((size_t)n * sizeof(int)));
        k_first_taps<<<grid_for(n), 256, 0, st>>>(p->coords.as<double>(), n, d, p->W, p->offs.as<int>());
        ML_CUDA(cudaGetLastError());
    }
    // ---- bins -> subproblems
    StreamBuf counts(st);
    ML_TRY(counts.ensure((size_t)(nbins + 1) * 4));
    { ProfScope pr_("plan", st);
    k_bin_starts<<<grid_for(n + 1), 256, 0, st>>>(sorted_keys, n, ka.cells, (int)nbins, counts.as<int>());
    }
    ML_CUDA(cudaGetLastError());
    std::vector<int> hc(nbins), hstart(nbins + 1);
    ML_CUDA(cudaMemcpyAsync(hstart.data(), counts.p, (size_t)(nbins + 1) * 4, cudaMemcpyDeviceToHost, st));
    ML_CUDA(cudaStreamSynchronize(st));
    for (int64_t b = 0; b < nbins; ++b) hc[b] = hstart[b + 1] - hstart[b];
    if (p->prec == ML_F32 && nbins == 1 && ka.cells == 1) {
        // one tile: the points stay in input order (perm is the identity) and the
        // spreading visits them in the order of their first-tap cells
        int64_t cells = 1;
        for (int a = 0; a < d; ++a) cells *= g.B;
        if (cells < ((int64_t)1 << 32)) {
            KeyArgs kc = ka;
            kc.cells = (uint32_t)cells;
            { ProfScope pr_("plan", st);
            k_keys<<<grid_for(n), 256, 0, st>>>(points, n, kc, urel.as<double>(), keys.as<uint32_t>(), idx.as<int>());
            }
            ML_CUDA(cudaGetLastError());
            int cbits = 0;
            while ((1LL << cbits) < cells) ++cbits;
            int *cell_idx = nullptr;
            ML_TRY(radix_sort(keys.as<uint32_t>(), idx.as<int>(), keys2.as<uint32_t>(), idx2.as<int>(), n, cbits, st,
                              &cell_idx));
            ML_TRY(p->sidx.ensure((size_t)n * 4));
            { ProfScope pr_("plan", st);
            k_copy_int<<<grid_for(n), 256, 0, st>>>(cell_idx, p->sidx.as<int>(), n);
            }
            ML_CUDA(cudaGetLastError());
        }
    }
    std::vector<int> sb, ss, sc, bs(nbins + 1);
    int64_t pos = 0;
    for (int64_t b = 0; b < nbins; ++b) {
        bs[b] = (int)sb.size();
        const int c = hc[b];
        if (c > 0) {
            const int parts = (c + kSubPoints - 1) / kSubPoints;
            for (int q = 0; q < parts; ++q) {
                const int lo_i = (int)((int64_t)c * q / parts), hi_i = (int)((int64_t)c * (q + 1) / parts);
                sb.push_back((int)b);
                ss.push_back((int)(pos + lo_i));
                sc.push_back(hi_i - lo_i);
            }
        }
        pos += c;
    }
    bs[nbins] = (int)sb.size();
    p->nsub = (int)sb.size();
    p->sub_max = 0;
    for (int c : sc) p->sub_max = std::max(p->sub_max, c);
    ML_TRY(p->sub_bin.ensure(sb.size() * 4));
    ML_TRY(p->sub_start.ensure(sb.size() * 4));
    ML_TRY(p->sub_count.ensure(sb.size() * 4));
    ML_TRY(p->bin_sub.ensure(bs.size() * 4));
    ML_CUDA(cudaMemcpy(p->sub_bin.p, sb.data(), sb.size() * 4, cudaMemcpyHostToDevice));
    ML_CUDA(cudaMemcpy(p->sub_start.p, ss.data(), ss.size() * 4, cudaMemcpyHostToDevice));
    ML_CUDA(cudaMemcpy(p->sub_count.p, sc.data(), sc.size() * 4, cudaMemcpyHostToDevice));
    ML_CUDA(cudaMemcpy(p->bin_sub.p, bs.data(), bs.size() * 4, cudaMemcpyHostToDevice));
    // groups of consecutive subproblems of one bin: a bin with S subproblems
    // gets groups of ceil(sqrt(S)) (at most kGroupSubs), so that the group sums
    // and the fold that follows both read about sqrt(S) tiles per cell
    std::vector<int> gs, bg(nbins + 1);
    for (int64_t b = 0; b < nbins; ++b) {
        bg[b] = (int)gs.size();
        const int S = bs[b + 1] - bs[b];
        const int G = std::max(1, std::min(kGroupSubs, (int)std::ceil(std::sqrt((double)S))));
        for (int s = bs[b]; s < bs[b + 1]; s += G) gs.push_back(s);
    }
    bg[nbins] = (int)gs.size();
    p->ngroups = (int)gs.size();
    gs.push_back(p->nsub);
    ML_TRY(p->grp_sub.ensure(gs.size() * 4));
    ML_TRY(p->bin_grp.ensure(bg.size() * 4));
    ML_CUDA(cudaMemcpy(p->grp_sub.p, gs.data(), gs.size() * 4, cudaMemcpyHostToDevice));
    ML_CUDA(cudaMemcpy(p->bin_grp.p, bg.data(), bg.size() * 4, cudaMemcpyHostToDevice));
    urel.release();
    keys.release();
    keys2.release();
    idx.release();
    idx2.release();
    // ---- Fourier tables (host FP64) -> device
    window_fourier(p->n_os, 0.5 * p->W, p->kb_shape, p->N / 2, p->phihat);
    if (p->kernel != ML_KERNEL_LAPLACE)   // the Laplacian's b_l were formed with its scaling
        kernel_fourier(p->sigma_s, p->N, d, p->eps_B, p->p_reg, p->bhat);
    slot_multiplier(p->N, d, p->n_os, p->bhat, p->phihat, p->mult);
    for (int a = 0; a < d; ++a) {
        std::vector<double> M, Mt;
        trig_matrix(p->N, p->n_os, p->s0[a], g.L[a], M);
        Mt.assign(M.size(), 0.0);
        for (int s = 0; s < g.K; ++s)
            for (int j = 0; j < g.L[a]; ++j) Mt[(size_t)j * g.K + s] = M[(size_t)s * g.L[a] + j];
        if (p->prec == ML_F32) {
            ML_TRY(upload<float>(p->trig_f[a], M));
            ML_TRY(upload<float>(p->trig_b[a], Mt));
        } else {
            ML_TRY(upload_dw(p->trig_f[a], M));
            ML_TRY(upload_dw(p->trig_b[a], Mt));
        }
    }
    if (p->prec == ML_F32) ML_TRY(upload<float>(p->mult_d, p->mult));
    else ML_TRY(upload_dw(p->mult_d, p->mult));
    // ---- near-field cell list (Laplacian)
    if (p->kernel == ML_KERNEL_LAPLACE) ML_TRY(near_plan(p, points, st));
    // ---- degrees D = W~ 1 - K(0) (sorted order), D^{-1/2}
    ML_TRY(ensure_workspace(p, 1));
    ML_TRY(p->deg.ensure((size_t)n * 8));
    ML_TRY(p->dinv.ensure((size_t)n * 8));
    ApplyVec v{nullptr, 1, p->deg.as<double>(), 1, 1};
    ApplyOpts o;
    o.sorted_out = true;
    ML_TRY(apply_layer(p, v, o, st));
    ML_CUDA(cudaMemsetAsync(p->status.p, 0, 4, st));
    const int dblk = grid_for(n);
    StreamBuf range(st);
    ML_TRY(range.ensure((size_t)dblk * 2 * sizeof(double)));
    { ProfScope pr_("plan", st);
    k_dinv<<<dblk, 256, 0, st>>>(p->deg.as<double>(), n, p->dinv.as<double>(), p->status.as<int>(),
                                 range.as<double>());
    }
    ML_CUDA(cudaGetLastError());
    int bad = 0;
    std::vector<double> hr((size_t)dblk * 2);
    ML_CUDA(cudaMemcpyAsync(&bad, p->status.p, 4, cudaMemcpyDeviceToHost, st));
    ML_CUDA(cudaMemcpyAsync(hr.data(), range.p, hr.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    ML_CUDA(cudaStreamSynchronize(st));
    p->deg_min = INFINITY;
    p->deg_max = -INFINITY;
    for (int b = 0; b < dblk; ++b) {
        p->deg_min = std::min(p->deg_min, hr[2 * b]);
        p->deg_max = std::max(p->deg_max, hr[2 * b + 1]);
    }
    // raw products stay available; normalised ones report ML_ERR_DEGREE
    p->deg_ok = !bad;
    return ML_OK;
}

}  // namespace ml

int64_t ml_plan_s::device_bytes() const
{
    int64_t t = 0;
    const ml::DevBuf *bufs[] = {&perm, &iperm, &coords, &sidx, &wts, &offs, &deg, &dinv, &sub_bin, &sub_start, &sub_count, &bin_sub, &grp_sub, &bin_grp,
                                &trig_f[0], &trig_f[1], &trig_f[2], &trig_b[0], &trig_b[1], &trig_b[2],
                                &mult_d, &scratch, &work[0], &work[1], &stage_x, &stage_y, &status, &Wd,
                                &nf_loc, &nf_orig, &nf_sidx, &nf_start, &nf_task};
    for (auto *b : bufs) t += (int64_t)b->bytes;
    return t;
}

static void release_all(ml_plan_s *p)
{
    ml::DevBuf *bufs[] = {&p->perm, &p->iperm, &p->coords, &p->sidx, &p->wts, &p->offs, &p->deg, &p->dinv, &p->sub_bin, &p->sub_start, &p->sub_count,
                          &p->bin_sub, &p->grp_sub, &p->bin_grp, &p->trig_f[0], &p->trig_f[1], &p->trig_f[2], &p->trig_b[0], &p->trig_b[1],
                          &p->trig_b[2], &p->mult_d, &p->scratch, &p->work[0], &p->work[1], &p->stage_x,
                          &p->stage_y, &p->status, &p->batch_desc, &p->batch_part, &p->Wd, &p->sum_parts};
    for (auto *b : bufs) b->release();
}

extern "C" {

const char *ml_last_error(void) { return ml::g_err.c_str(); }

const char *ml_version(void) { return "ml_fastsum 0.1 (sm_103a)"; }

static ml_status plan_common(ml_plan_t *out, const double *points, int64_t n, int d, double sigma, int N, int W,
                             double sig_os, double eps_B, int p_reg, ml_prec prec, double target_rel_err,
                             int bin, int kernel, double eps_I, void *stream)
{
    using namespace ml;
    if (!out) return fail(ML_ERR_ARG, "out is null");
    *out = nullptr;
    if (!points) return fail(ML_ERR_ARG, "points is null");
    if (n < 2 || n > (int64_t)INT32_MAX - 1) return fail(ML_ERR_ARG, "n must be in [2, 2^31-2]");
    if (d < 1 || d > 3) return fail(ML_ERR_ARG, "d must be 1, 2 or 3");
    if (!(sigma > 0) || !std::isfinite(sigma)) return fail(ML_ERR_ARG, "sigma must be positive and finite");
    if (N != 0 && (N < 4 || N > kMaxN || (N & 1))) return fail(ML_ERR_ARG, "N must be 0 or even in [4, 512]");
    if (W != 0 && !((W >= 4 && W <= 8) || W == 10 || W == 12 || W == 14 || W == 16))
        return fail(ML_ERR_ARG, "window width must be 0, 4..8, 10, 12, 14 or 16 taps");
    if (sig_os != 0 && !(sig_os >= 1.5 && sig_os <= 4.0)) return fail(ML_ERR_ARG, "oversampling must be in [1.5, 4]");
    if (!(eps_B >= 0 && eps_B < 0.5)) return fail(ML_ERR_ARG, "eps_B must be in [0, 1/2)");
    if (kernel != ML_KERNEL_GAUSS && kernel != ML_KERNEL_LAPLACE)
        return fail(ML_ERR_ARG, "kernel must be ML_KERNEL_GAUSS or ML_KERNEL_LAPLACE");
    if (kernel == ML_KERNEL_GAUSS) {
        if (eps_B > 0 && (p_reg < 1 || p_reg > 8)) return fail(ML_ERR_ARG, "p_reg must be in [1, 8] when eps_B > 0");
        if (eps_I != 0) return fail(ML_ERR_ARG, "eps_I applies to the Laplacian kernel only");
    } else {
        if (p_reg < 0 || p_reg > 8) return fail(ML_ERR_ARG, "p_reg must be 0 (automatic) or in [1, 8]");
        if (!(eps_I == 0 || (eps_I >= 1.0 / 1024 && eps_I <= 0.25)))
            return fail(ML_ERR_ARG, "eps_I must be 0 (automatic) or in [1/1024, 1/4]");
        if (target_rel_err > 0 && target_rel_err < 1e-10)
            return fail(ML_ERR_DOMAIN, "Laplacian: the inner polynomial's conditioning bounds the accuracy near 1e-10");
    }
    if (prec != ML_F32 && prec != ML_F64) return fail(ML_ERR_ARG, "prec must be ML_F32 or ML_F64");
    if (bin < 0 || bin > 512) return fail(ML_ERR_ARG, "bin must be 0 (automatic) or in [1, 512]");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice", __FILE__, __LINE__);
    ml_plan_s *p = new (std::nothrow) ml_plan_s;
    if (!p) return fail(ML_ERR_OOM, "host allocation failed");
    p->n = n;
    p->d = d;
    p->sigma = sigma;
    p->N = N;
    p->W = W;   // 0 = automatic
    p->sig_os_req = sig_os;
    p->bin_req = bin;
    p->eps_B = eps_B;
    p->p_reg = eps_B > 0 ? p_reg : 0;
    p->kernel = kernel;
    if (kernel == ML_KERNEL_LAPLACE) {
        p->eps_B_req = eps_B;
        p->eps_I_req = eps_I;
        p->p_reg = p_reg;
    }
    p->prec = prec;
    p->target = target_rel_err > 0 ? target_rel_err : (prec == ML_F32 ? 1e-4 : 1e-6);
    // host points: copied to a device buffer on the call's stream, freed on
    // return (the set-up reads the points only before its last synchronisation)
    DevBuf staged;
    const double *dpts = points;
    {
        cudaPointerAttributes at;
        bool on_device = false;
        if (cudaPointerGetAttributes(&at, points) == cudaSuccess)
            on_device = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
        else
            cudaGetLastError();   // an unregistered host pointer
        if (!on_device) {
            const size_t bytes = (size_t)n * d * sizeof(double);
            ml_status sst = staged.ensure(bytes);
            cudaError_t ce = cudaSuccess;
            if (sst == ML_OK) {
                ce = cudaMemcpyAsync(staged.p, points, bytes, cudaMemcpyHostToDevice, (cudaStream_t)stream);
                if (ce != cudaSuccess) sst = cuda_fail(ce, "cudaMemcpyAsync (points)", __FILE__, __LINE__);
            }
            if (sst != ML_OK) {
                delete p;
                return sst;
            }
            dpts = staged.as<double>();
        }
    }
    ml_status st = plan_impl(p, dpts, (cudaStream_t)stream);
    if (st != ML_OK) {
        release_all(p);
        delete p;
        return st;
    }
    *out = p;
    return ML_OK;
}

ml_status ml_fastsum_plan(ml_plan_t *out, const double *points, int64_t n, int d, double sigma, int N, int m,
                          double eps_B, int p_reg, ml_prec prec, double target_rel_err, void *stream)
{
    if (m != 0 && (m < 2 || m > ml::kMaxM)) return ml::fail(ML_ERR_ARG, "m must be 0 or in [2, 8]");
    return plan_common(out, points, n, d, sigma, N, 2 * m, 0.0, eps_B, p_reg, prec, target_rel_err, 0,
                       ML_KERNEL_GAUSS, 0.0, stream);
}

ml_status ml_fastsum_plan_ex(ml_plan_t *out, const double *points, int64_t n, int d, double sigma,
                             const ml_plan_params *prm, void *stream)
{
    if (!prm) return ml::fail(ML_ERR_ARG, "params is null");
    return plan_common(out, points, n, d, sigma, prm->N, prm->taps, prm->oversampling, prm->eps_B, prm->p_reg,
                       prm->prec, prm->target_rel_err, prm->bin, prm->kernel, prm->eps_I, stream);
}

ml_status ml_plan_destroy(ml_plan_t plan)
{
    if (!plan) return ML_OK;
    release_all(plan);
    delete plan;
    return ML_OK;
}

ml_status ml_plan_get_info(ml_plan_t p, ml_plan_info *info)
{
    if (!p || !info) return ml::fail(ML_ERR_ARG, "null plan or info");
    std::memset(info, 0, sizeof(*info));
    info->n = p->n;
    info->d = p->d;
    info->N = p->N;
    info->m = p->m;
    info->taps = p->W;
    info->n_os = p->n_os;
    for (int a = 0; a < 3; ++a) {
        info->L[a] = p->g.L[a];
        info->center[a] = p->center[a];
    }
    info->bin = p->g.B;
    info->nbins = (int)p->g.nbins();
    info->nsub = p->nsub;
    info->prec = p->prec;
    info->domain = p->domain;
    info->p_reg = p->p_reg;
    info->eps_B = p->eps_B;
    info->sigma = p->sigma;
    info->sigma_s = p->sigma_s;
    info->scale = p->scale;
    info->target_rel_err = p->target;
    info->deg_min = p->deg_min;
    info->deg_max = p->deg_max;
    info->device_bytes = p->device_bytes();
    info->applied_vectors = p->applied;
    info->dense = p->dense ? 1 : 0;
    info->kernel = p->kernel;
    info->eps_I = p->eps_I;
    info->kernel_err = p->kernel_err;
    info->near_pairs = p->near_pairs;
    return ML_OK;
}

ml_status ml_plan_copy_table(ml_plan_t p, int which, double *out, int64_t count)
{
    if (!p || !out) return ml::fail(ML_ERR_ARG, "null plan or output");
    if (which == 0 || which == 1) {
        const std::vector<double> &t = which == 0 ? p->bhat : p->phihat;
        if (count < (int64_t)t.size()) return ml::fail(ML_ERR_ARG, "count too small");
        std::memcpy(out, t.data(), t.size() * sizeof(double));
        return ML_OK;
    }
    if (which == 2) {
        if (count < p->n) return ml::fail(ML_ERR_ARG, "count too small");
        std::vector<double> deg(p->n);
        std::vector<int> perm(p->n);
        ML_CUDA(cudaDeviceSynchronize());
        ML_CUDA(cudaMemcpy(deg.data(), p->deg.p, p->n * 8, cudaMemcpyDeviceToHost));
        ML_CUDA(cudaMemcpy(perm.data(), p->perm.p, p->n * 4, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < p->n; ++i) out[perm[i]] = deg[i];
        return ML_OK;
    }
    return ml::fail(ML_ERR_ARG, "unknown table");
}

}  // extern "C"

extern "C" ml_status ml_release_cached_memory(void) { return ml::release_cached(); }
