// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/ml_fastsum.h"

namespace ml {

// ------------------------------------------------------------------ errors
void set_error(const std::string &msg);
ml_status fail(ml_status st, const std::string &msg);
ml_status cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define ML_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) return ::ml::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define ML_TRY(expr)                             \
    do {                                         \
        ml_status s_ = (expr);                   \
        if (s_ != ML_OK) return s_;              \
    } while (0)

// --------------------------------------------------------- limits / sizes
constexpr int kMaxVec = 8;       // vectors per spreading/interpolation pass
constexpr int kMaxM = 8;         // window half-width limit
constexpr int kMaxN = 512;       // bandwidth limit
constexpr int kSubPoints = 1024; // points per subproblem (bounds per-cell counts)
constexpr int kBatchPtsTotal = 1024; // points per CTA of the batched interpolation (4 per thread)
constexpr int kGroupSubs = 64;   // most subproblem tiles summed per group before the fold

// Streaming multiprocessors of the current device (queried once per device and
// cached): grid-stride launches size their grids as a multiple of it.
int sm_count();

// ------------------------------------------------- tensor-core FP64 products
// Tall FP64 operands of the Lanczos products: element (i, c) of layer t at
// base + t * lstride + i * rs + c * cs (point-major: rs = ld, cs = 1;
// column-major: rs = 1, cs = ld).  ozaki.cu: the Gram A^T B and the update
// Y (-)= A M on the fp16 tensor cores through 8-bit slices of the FP64
// values, exact up to FP64 rounding; the tall operands must satisfy |v| < 2.
struct OzMat {
    const double *base;
    int64_t lstride, rs, cs;
};
struct OzOut {
    double *base;
    int64_t lstride, rs, cs;
};
bool oz_gram_ok(int rc, int cb);
bool oz_gemm_ok(int rc);
int oz_gram_blocks(int nslots, int64_t n);
// part[(y * nbx + x) * rc * cb + c * cb + j]: per-block partial Grams (y = slot)
ml_status oz_gram(OzMat A, int rc, OzMat B, int cb, const int *lay, int nslots, int64_t n, int nbx, double *part,
                  cudaStream_t st);
// Y_t[:, j] (-)= sum_r A_t[:, r] M_y[r, j], M_y[r, j] = M[y * mslot + r * mrs + j * mcs]
ml_status oz_gemm(OzMat A, int rc, const double *M, int64_t mrs, int64_t mcs, int64_t mslot, int cb, OzOut Y,
                  const int *lay, int nslots, int64_t n, bool sub, cudaStream_t st);
// the solvers' products of the basis: 0 FP64 pipe, 1 double-word FP32 (default), 2 tensor cores
int dense_products_kind();
bool oz_enabled();
ml_status oz_reset_error(cudaStream_t st);
ml_status oz_read_error(int *flags, cudaStream_t st);

// ------------------------------------------------------------ device buffer
// Owns one device allocation (freed on destruction; movable, not copyable).
// Blocks of 1 MiB and more go back to a per-device cache on release (after a
// device synchronisation, as cudaFree would imply) and are handed out again
// by ensure, so that plans made and destroyed step after step do not pay for
// the driver's allocation and mapping of hundreds of megabytes each time
// (ml_release_cached_memory returns the cache to the driver).
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    int dev = -1;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes), dev(o.dev)
    {
        o.p = nullptr;
        o.bytes = 0;
    }
    DevBuf &operator=(DevBuf &&o) noexcept
    {
        if (this != &o) {
            release();
            p = o.p;
            bytes = o.bytes;
            dev = o.dev;
            o.p = nullptr;
            o.bytes = 0;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    ml_status ensure(size_t nbytes);   // grow (contents not kept)
    void release();
    template <typename T> T *as() const { return static_cast<T *>(p); }
};

// Temporaries of one call on one stream, from a per-device stream-ordered
// pool (cudaMallocFromPoolAsync / cudaFreeAsync) that keeps its memory
// between calls: allocation and release are ordered with the stream's own
// work and never wait for the device, so calls on other streams (the layers'
// plans built concurrently) do not serialise on each other's frees.  Falls
// back to cudaMalloc / cudaFree where the device has no memory pools.
struct StreamBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;
    bool pooled = false;
    explicit StreamBuf(cudaStream_t s) : st(s) {}
    StreamBuf(const StreamBuf &) = delete;
    StreamBuf &operator=(const StreamBuf &) = delete;
    ~StreamBuf() { release(); }
    ml_status ensure(size_t nbytes);   // grow (contents not kept)
    void release();
    template <typename T> T *as() const { return static_cast<T *>(p); }
};

// ------------------------------------------------------------------ plan
struct GridGeom {
    int d = 1;
    int W = 4;          // window width: taps f0 .. f0+W-1 per dim
    int B = 8;          // bin edge (cells)
    int Pt = 0;         // padded tile edge = B + W (first tap offset in [0, B])
    int L[3] = {1, 1, 1};
    int nb[3] = {1, 1, 1};
    int R = 1;          // neighbour bins reaching into a bin per dim = 1 + (W-1)/B
    int K = 0;          // coefficient slots per dim = N + 1
    int64_t cells() const { return (int64_t)L[0] * L[1] * L[2]; }
    int64_t nbins() const { return (int64_t)nb[0] * nb[1] * nb[2]; }
    int64_t tile_cells() const {
        int64_t t = 1;
        for (int a = 0; a < d; ++a) t *= Pt;
        return t;
    }
};

struct ml_plan_impl;

}  // namespace ml

struct ml_plan_s {
    // parameters
    int64_t n = 0;
    int d = 0;
    int N = 0;
    int m = 0;             // window half-width, W/2 rounded down (paper's m_NFFT)
    int W = 0;             // window width in taps per dimension (half-width W/2)
    double sig_os_req = 0; // requested oversampling (0: automatic / 2)
    int bin_req = 0;       // requested bin edge (0: automatic rule)
    int n_os = 0;
    ml_prec prec = ML_F64;
    int domain = 0;
    int p_reg = 0;
    double eps_B = 0;
    double sigma = 0, sigma_s = 0, scale = 0;
    double center[3] = {0, 0, 0};
    double target = 0;
    double kb_shape = 0;   // b = pi (2 - 1/sigma_os)
    double kb_norm = 0;    // h e^{-b h} / (1 - e^{-2 b h}), h = W/2: phi_n(t) = norm (e^{bs} - e^{-bs})/s
    float kbp[192] = {};   // FP32 form: window polynomials, rows of 12 floats for the first ceil(W/2) taps (window_row_poly)
    int s0[3] = {0, 0, 0}; // torus index of active-grid cell 0 per dim
    ml::GridGeom g;
    int vp = 1;            // vectors per pass
    int sub_max = 0;       // largest subproblem (points)
    int ngroups = 0;       // groups of <= kGroupSubs consecutive subproblems of one bin
    int nsub = 0;
    double deg_min = 0, deg_max = 0;
    bool deg_ok = true;    // every degree positive and finite: D^{-1/2} defined
    int64_t applied = 0;   // vectors pushed through apply_layer
    bool dense = false;    // dense layer: W stored explicitly (Wd), no fast summation
    int kernel = 0;        // ml_kernel
    double eps_I_req = 0;  // Laplacian: requested near-field radius (0: automatic)
    double eps_B_req = 0;  // requested eps_B (the Laplacian picks one when 0)
    double eps_I = 0;      // Laplacian: near-field radius (scaled domain)
    double kernel_err = 0; // Laplacian: measured max |K_RF - K_R| on the probes
    int64_t near_pairs = 0;   // Laplacian: pairs the near-field pass examines per vector
    int nf_nc[3] = {1, 1, 1}; // near-field cells per dim
    double nf_h = 0;          // near-field cell edge (scaled domain)
    int nf_ntask = 0;         // near-field tasks (<= kNearThreads targets of one cell)
    std::vector<double> nf_poly;  // inner polynomial c_j of r^{2j}

    // host tables (FP64)
    std::vector<double> bhat;    // (N/2+1)^d
    std::vector<double> phihat;  // N/2+1
    std::vector<double> mult;    // K^d over coefficient slots

    // device data (sorted order unless noted)
    ml::DevBuf perm;      // int32 n: sorted position -> input index
    ml::DevBuf iperm;     // int32 n: input index -> sorted position
    ml::DevBuf coords;    // T n*d local grid coordinates
    ml::DevBuf sidx;      // int32 n (FP32 layers of one tile): the spreading order of the
                          // sorted positions, by first-tap cell (the others keep input order)
    ml::DevBuf wts;       // FP64 form: float2 [n][d][W] window weights (double-word pairs)
    ml::DevBuf offs;      // FP64 form: int n packed first taps o0 | o1 << 10 | o2 << 20
    ml::DevBuf deg;       // double n: degrees
    ml::DevBuf dinv;      // double n: D^{-1/2}
    ml::DevBuf sub_bin, sub_start, sub_count;  // int32 nsub
    ml::DevBuf bin_sub;   // int32 nbins+1: first subproblem of each bin
    ml::DevBuf grp_sub;   // int32 ngroups+1: first subproblem of each tile group
    ml::DevBuf bin_grp;   // int32 nbins+1: first tile group of each bin
    ml::DevBuf trig_f[3]; // K x L_a (forward, cos rows then sin rows): float, or float2 pairs (FP64 form)
    ml::DevBuf trig_b[3]; // L_a x K (backward = transpose), same element type
    ml::DevBuf mult_d;    // K^d slot multipliers, same element type
    ml::DevBuf Wd;        // dense layers: W, n x n row-major (FP32 or FP64), zero diagonal
    // Laplacian near field (cell order)
    ml::DevBuf nf_loc;    // float4 n: coordinates relative to the point's cell corner
    ml::DevBuf nf_orig;   // int32 n: input index
    ml::DevBuf nf_sidx;   // int32 n: position in the sorted (spreading) order
    ml::DevBuf nf_start;  // int32 cells+1: first point of each cell
    ml::DevBuf nf_task;   // int4 nf_ntask: cell, first point, count

    // workspace
    ml::DevBuf scratch;   // spreading tiles: nsub * Pt^d * vp (T)
    ml::DevBuf work[2];   // transform ping-pong buffers
    ml::DevBuf stage_x, stage_y;  // staging for host X / Y
    ml::DevBuf status;    // int flags written by device code
    ml::DevBuf batch_desc;               // per-layer descriptors of a batched apply led by this plan
    ml::DevBuf batch_part;               // per-group partial sums of a batched multilayer apply
    ml::DevBuf sum_parts;                // per-layer terms of a concurrent multilayer apply led by this plan
    std::vector<unsigned char> batch_host;  // host copy of the uploaded descriptors
    int64_t device_bytes() const;
};

namespace ml {

// --------------------------------------------------------- host math (FP64)
double bessel_i0(double x);
// Fourier coefficients phi_hat_n(k), k = 0..kmax, of the normalised window
// phi_n(t) = sinh(b sqrt(m^2 - t^2)) / sqrt(m^2 - t^2) / (sinh(b m)/m).
void window_fourier(int n_os, double h, double b, int kmax, std::vector<double> &out);
// b_l, l = 0..N/2 per dim, for the box domain (separable) or the ball domain.
void kernel_fourier(double sigma_s, int N, int d, double eps_B, int p_reg, std::vector<double> &bhat);
// the two-point Taylor regulariser's monomial coefficients in t = (r - r_I)/eps_B
bool regulariser_coeffs(double sigma_s, double eps_B, int p, std::vector<double> &q, int kernel);
// the Laplacian's regularised kernel K_R (inner polynomial c in r^2 on r < eps_I,
// outer two-point Taylor polynomial q on (1/2 - eps_B, 1/2])
struct LaplaceReg {
    double s = 0, eps_B = 0, eps_I = 0;
    std::vector<double> q, c;
};
bool inner_coeffs(double sigma_s, double eps_I, int p, std::vector<double> &c);
bool laplace_reg_init(double sigma_s, double eps_B, double eps_I, int p, LaplaceReg &g);
double laplace_regularised(double r, const LaplaceReg &g);
// largest |K_RF - K_R| on probe distances, b_l given on l_a = 0..N/2
double kernel_probe_error(const std::vector<double> &bhat, int N, int d, const LaplaceReg &g, int probes);

// ---------------------------------------------------- Laplacian kernel
constexpr int kNearThreads = 128;  // targets per near-field task
// grid cells across the inner region (c = N eps_I) for a target accuracy
int laplace_cells(double target);
// bandwidth N minimising the transform + near-field cost model
int laplace_bandwidth(int64_t n, int d, int c, int W, ml_prec prec);
// b_l of the Laplacian's K_R (FP64, on the device), copied to p->bhat
ml_status laplace_fourier(ml_plan_s *p, const LaplaceReg &g, cudaStream_t st);
// cell list of the near field (after the spreading order is fixed)
ml_status near_plan(ml_plan_s *p, const double *points, cudaStream_t st);
// LSD radix sort of (key, value) pairs over the low `bits` key bits
ml_status radix_sort(uint32_t *keys, int *vals, uint32_t *keys2, int *vals2, int64_t n, int bits,
                     cudaStream_t st, int **result_vals);
// multiplier over coefficient slots
void slot_multiplier(int N, int d, int n_os, const std::vector<double> &bhat,
                     const std::vector<double> &phihat, std::vector<double> &mult);
// forward trig matrix K x L for one dim (cos rows 0..N/2, sin rows 1..N/2)
void trig_matrix(int N, int n_os, int s0, int L, std::vector<double> &M);
// symmetric eigen-decomposition of a small dense matrix (cyclic Jacobi);
// a is n x n row-major (destroyed), evals ascending, evecs column j = vector j
void sym_eig(int n, std::vector<double> &a, std::vector<double> &evals, std::vector<double> &evecs);

// ------------------------------------------------------------- launchers
struct ApplyVec {      // one pass over up to kMaxVec vectors
    const double *X;   // input block base (point-major, row stride ldx), or null (ones)
    int ldx;
    double *Y;         // output base (row stride ldy)
    int ldy;
    int nv;            // vectors in this pass
};

// Device copy of the per-layer argument records of a batched pass, with the
// host image last uploaded (re-uploaded only when it changes).
struct DescSlot {
    DevBuf dev;
    std::vector<unsigned char> host;
};

// layer apply: y (+)= alpha * post(D^{-1/2}) * (W~ u - u),  u = pre(D^{-1/2}) * x
struct ApplyOpts {
    bool normalized = false;   // pre- and post-scale by D^{-1/2}
    bool accumulate = false;   // Y += instead of Y =
    bool sorted_out = false;   // write Y in sorted order, no post-scale (degree set-up)
    bool sorted_final = false; // write the finished value (post-scaled, no accumulation) at the sorted
                               // position: the layer terms gathered back to input order later
    double alpha = 1.0;
    double shift = 0.0;        // adds shift * x (input order) to the output: used for L_sym + delta I
    double self = 1.0;         // K(0): subtracted self term coefficient
    // batched passes only: per-layer input/output blocks (layer t applies its
    // own operator to layer_vecs[t], no sum over layers), and where the
    // argument records live (null: the first plan's slot)
    const ApplyVec *layer_vecs = nullptr;
    DescSlot *desc = nullptr;
};

ml_status apply_layer(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, cudaStream_t st);
// adds the Laplacian's near-field term of one layer pass to its output
ml_status run_near(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, cudaStream_t st);

// ---------------------------------------------------------------- tracing
bool profiling();
// counts one CUDA-graph replay of a captured solver iteration (diagnostics)
void count_graph_replay();
// Switches kernel timing off on this thread for its lifetime (timing creates
// CUDA events, which callers that must not allocate cannot accept).
class NoProfileScope {
public:
    NoProfileScope();
    ~NoProfileScope();

private:
    bool prev_;
};
// Records a CUDA event on `st` now and another when it goes out of scope,
// filed under `name`, while profiling is enabled; otherwise does nothing.
class ProfScope {
public:
    ProfScope(const char *name, cudaStream_t st);
    ~ProfScope();
    ProfScope(const ProfScope &) = delete;
    ProfScope &operator=(const ProfScope &) = delete;

private:
    const char *name_;
    cudaStream_t st_;
    void *a_ = nullptr;
    bool active_ = false;
};
ml_status ensure_workspace(ml_plan_s *p, int nv);
// product of a dense layer (W stored in the plan), same options as apply_layer
ml_status run_dense(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, cudaStream_t st);
// sign of each column of V (n x k, column-major): largest-magnitude entry positive
ml_status sign_fix_cols(double *V, int64_t n, int k, cudaStream_t st);

// Device workspace of one layer pass: the spreading tiles and the two
// transform buffers.
struct LayerWork {
    void *scratch;
    void *work0;
    void *work1;
};
// bytes of the tile scratch and of each transform buffer for nv vectors
void workspace_bytes(const ml_plan_s *p, int nv, size_t *scratch, size_t *work);
// run one layer pass on the given workspace (no allocation)
ml_status run_layer_ws(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, const LayerWork &w, cudaStream_t st);
// vectors in the next pass for `remaining` vectors
int pass_width(const ml_plan_s *p, int remaining);
// whether the layers can run as one batch (FP32, equal d and W, every grid a
// single tile, identical subproblem split) and the batched pass itself
bool batchable(ml_plan_s *const *layers, int T);
bool batchable_layers(ml_plan_s *const *layers, int T);
ml_status run_batch(ml_plan_s *const *layers, int T, const ApplyVec &v, const ApplyOpts &o, cudaStream_t st);

}  // namespace ml
