/*
 * ml_fastsum.h - C ABI of the GB300 multilayer Gaussian-graph fast summation
 * and Lanczos eigensolver.
 *
 * What is computed (Bergermann, Stoll, Volkmer, "Semi-supervised learning for
 * aggregated multilayer graphs using diffuse interface methods and fast
 * matrix vector products"):
 *   - per layer t, the fully connected graph on n points x_i in R^{d_t},
 *     d_t in {1,2,3}, with weights W_ij = exp(-||x_i - x_j||^2 / sigma_t^2),
 *     i != j, and zero diagonal (Sec. 2, Sec. 4);
 *   - the product W_t v by NFFT-based fast summation (Alg. 1), using
 *     W = W~ - K(0) I with K(0) = 1 (Sec. 4);
 *   - degrees D_t = diag(W_t 1) and the normalised operator
 *     D_t^{-1/2} W_t D_t^{-1/2} = I - L_sym^(t) (Sec. 2);
 *   - the multilayer operator I - L_1 = (1/T) sum_t D_t^{-1/2} W_t D_t^{-1/2}
 *     (Eq. I-L_1) and the shifted power mean L_{p,delta}^p (Eq.
 *     L_p_delta_power_p, delta = log(1+|p|) for p < 0);
 *   - the k smallest eigenpairs of L_1 or L_{p,delta} by the Lanczos method
 *     (Sec. 3).
 *
 * Conventions for every entry point:
 *   - Pointers are plain addresses; the caller owns every buffer it passes.
 *     "device" means memory of the current CUDA device; "host or device"
 *     arguments are detected with cudaPointerGetAttributes and staged
 *     through plan-owned device buffers when they live on the host.
 *   - Matrices of n points / n-vectors are row-major and point-major:
 *     element (i, c) of an n x b block is at [i*b + c].
 *   - All layers passed together must share n and the node order.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous on it unless stated otherwise.
 *   - No exception crosses the ABI.  On failure the call returns a non-zero
 *     ml_status and ml_last_error() describes the cause (thread-local).
 *   - The library never falls back to the CPU: without a usable GPU every
 *     call returns ML_ERR_CUDA.
 */
#ifndef ML_FASTSUM_H
#define ML_FASTSUM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ml_plan_s *ml_plan_t; /* opaque, library-owned */

typedef enum {
    ML_OK = 0,
    ML_ERR_ARG = 1,        /* invalid argument (null pointer, size, mode...) */
    ML_ERR_CUDA = 2,       /* a CUDA call failed, or no usable GPU */
    ML_ERR_OOM = 3,        /* device allocation failed */
    ML_ERR_DOMAIN = 4,     /* the requested accuracy needs a grid beyond the limits */
    ML_ERR_DEGREE = 5,     /* a degree D_i is not positive/finite: D^{-1/2} undefined */
    ML_ERR_BREAKDOWN = 6,  /* Lanczos could not extend the Krylov basis */
    ML_ERR_TIMEOUT = 7,    /* a bounded device-side wait gave up */
    ML_WARN_NOT_CONVERGED = 8 /* Lanczos stopped at maxit with nconv < k */
} ml_status;

typedef enum {
    ML_F32 = 0, /* window weights, spreading, grid transforms, interpolation in FP32
                   (spreading sums exact fixed-point integers)                       */
    ML_F64 = 1  /* the same steps FP64-class: values as unevaluated float pairs (about
                   48 significant bits) with exact FMA-based products on the FP32 pipes,
                   spreading into exact fixed-point integers; window weights from an
                   FP64 table                                                          */
} ml_prec;
/* In both precisions the degree normalisation, the multilayer accumulation,
 * the output vectors and every Lanczos quantity are FP64. */

/* apply modes */
#define ML_RAW_W 0        /* Y = (1/T) sum_t W_t X                          */
#define ML_NORMALIZED_A 1 /* Y = (1/T) sum_t D_t^{-1/2} W_t D_t^{-1/2} X    */
#define ML_DEGREE 2       /* Y = (1/T) sum_t D_t  (X unused, b must be 1)   */
#define ML_PER_LAYER 16   /* flag: X, Y hold T blocks of n x b; block t of Y
                             gets layer t's operator applied to block t of X
                             (no 1/T, no sum) */

/* Plan parameters chosen (or accepted) for one layer; see ml_plan_get_info. */
typedef struct {
    int64_t n;
    int d;
    int N;              /* bandwidth of K_RF, I_N = {-N/2..N/2-1}^d (Eq. K_RF)  */
    int m;              /* window half-width in grid cells, rounded down        */
    int n_os;           /* oversampled grid size per dim (torus of n_os cells)  */
    int L[3];           /* active grid extent per dim (cells that can be nonzero) */
    int bin;            /* spreading tile (bin) edge in cells                   */
    int nbins;          /* bins over the active grid                            */
    int nsub;           /* subproblems (point chunks of one bin)                */
    int prec;           /* ml_prec                                              */
    int domain;         /* 0 = box (periodised Gaussian), 1 = ball (eps_B > 0)  */
    int p_reg;          /* regularisation degree (ball domain)                  */
    double eps_B;       /* regularisation length (ball domain)                  */
    double sigma;       /* kernel width in input units                          */
    double sigma_s;     /* kernel width after scaling into the Alg. 1 domain    */
    double scale;       /* x' = scale * (x - center)                            */
    double center[3];
    double target_rel_err;
    double deg_min, deg_max; /* range of the computed degrees                    */
    int64_t device_bytes;    /* device memory owned by the plan                  */
    int64_t applied_vectors; /* vectors pushed through this layer's fast summation
                                since the plan was made (work counter)          */
    int taps;                /* window width: taps per dimension (half-width taps/2;
                                automatic choices may be odd)                    */
    int dense;               /* 1: dense layer (ml_dense_plan*), W stored; the
                                NFFT fields above are 0                          */
    int kernel;              /* ml_kernel of the layer                           */
    double eps_I;            /* Laplacian: near-field radius in the scaled domain
                                (0 for the Gaussian)                             */
    double kernel_err;       /* Laplacian: largest |K_RF - K_R| the plan measured
                                on its probe distances (0 for the Gaussian)      */
    int64_t near_pairs;      /* Laplacian: point pairs the near-field pass
                                examines per vector (cell-list neighbours)       */
} ml_plan_info;

/*
 * ml_fastsum_plan - set up one layer's fast summation (Alg. 1 input, Sec. 4)
 * and compute its degrees (Sec. 2).
 *
 *   out            receives the plan handle (caller destroys it).
 *   points         n x d row-major FP64, read during the call only: device
 *                  memory, or host memory, which the call copies to a device
 *                  buffer of its own on `stream` (freed on return).
 *   n, d           n >= 2, d in {1,2,3}.
 *   sigma          Gaussian width > 0 in the units of `points`.
 *   N              bandwidth (even, 4..512), or 0 to choose from target_rel_err.
 *   m              window half-width (2..8, i.e. 2m taps per dimension), or 0 to
 *                  choose the width (4..8, 10, ..., 16 taps, odd widths allowed)
 *                  from target_rel_err.
 *   eps_B, p_reg   eps_B = 0: box domain (periodised Gaussian, no regulariser);
 *                  0 < eps_B < 1/2: ball domain with the regularised kernel
 *                  K_R of degree 2*p_reg-1 on (1/2-eps_B, 1/2], p_reg in 1..8.
 *   prec           ML_F32 or ML_F64.
 *   target_rel_err accuracy the automatic choices aim at (<= 0: 1e-4 for
 *                  ML_F32, 1e-6 for ML_F64).
 *   stream         cudaStream_t used for the set-up kernels.
 * The call synchronises `stream` (it reads bounding boxes and bin counts back
 * to the host).  Errors: ML_ERR_ARG, ML_ERR_DOMAIN (grid beyond limits),
 * ML_ERR_OOM, ML_ERR_CUDA.  A degree <= 0 or non-finite (an isolated point
 * whose exact degree is below the approximation error) does not fail the
 * plan: raw products stay available, while normalised products and
 * ml_lanczos_eigs on that layer return ML_ERR_DEGREE (deg_min in
 * ml_plan_info shows it).
 */
ml_status ml_fastsum_plan(ml_plan_t *out, const double *points, int64_t n, int d, double sigma,
                          int N, int m, double eps_B, int p_reg, ml_prec prec,
                          double target_rel_err, void *stream);

/* Radial kernels of Sec. 4: the Gaussian exp(-||y||^2/sigma^2) and the
 * Laplacian exp(-||y||/sigma). */
typedef enum { ML_KERNEL_GAUSS = 0, ML_KERNEL_LAPLACE = 1 } ml_kernel;

/* Explicit parameters for ml_fastsum_plan_ex (0 = automatic choice). */
typedef struct {
    int N;               /* bandwidth of K_RF (even, 4..512)                                 */
    int taps;            /* window width W per dim: 4..8, 10, 12, 14 or 16                   */
    double oversampling; /* n_os / N in [1.5, 4]; automatic with taps = 0, else 2 when 0    */
    double eps_B;        /* as ml_fastsum_plan                                               */
    int p_reg;
    ml_prec prec;
    double target_rel_err;
    int bin;             /* spreading tile (bin) edge in grid cells, 0 = automatic rule;
                            larger tiles must fit the shared-memory budget (ML_ERR_ARG) */
    int kernel;          /* ml_kernel; 0 = the Gaussian                                      */
    double eps_I;        /* Laplacian: near-field radius in the scaled domain, 0 = automatic */
} ml_plan_params;

/*
 * ml_fastsum_plan_ex - ml_fastsum_plan with the window width and the
 * oversampling of the NFFT (Alg. 1 steps 1 and 3) chosen by the caller
 * (e.g. the learned parameter model below, ml_fastsum_plan_learned).
 * Same errors as ml_fastsum_plan, plus ML_ERR_ARG for out-of-range entries.
 *
 * kernel = ML_KERNEL_LAPLACE selects K(y) = exp(-||y||/sigma) (Sec. 4).  Its
 * cusp at y = 0 is handled by the near-field scheme of the fast summation of
 * non-smooth radial kernels that Sec. 4 cites: the ball domain is always used
 * (eps_B = 0 picks eps_B = max(1/16, eps_I)); K_R is in addition replaced on
 * ||y|| < eps_I by the even polynomial sum_{j<p_reg} c_j ||y||^{2j} matching
 * K's derivatives 0..p_reg-1 at eps_I (p_reg = 0: 8); Alg. 1 sums K_R and a
 * direct pass over a cell list of edge eps_I adds
 *     sum_{j: ||x_i - x_j|| < eps_I} (K - K_R)(x_i - x_j) u_j
 * (the pair j = i included).  Automatic choices: eps_I = c/N with c from
 * target_rel_err (c = 4..16 grid cells), and N by a cost model that balances
 * the grid transforms against the near-field pairs of a uniform cloud.  After
 * the Fourier coefficients are formed the plan measures max |K_RF - K_R| on
 * probe distances; above target_rel_err/2 it returns ML_ERR_DOMAIN.  The
 * near-field pass evaluates K - K_R in FP32 (ML_F32, FP64 accumulation) or
 * entirely in FP64 (ML_F64).  The inner polynomial's system (powers of eps_I
 * up to 2 p_reg - 2) limits the attainable error near 1e-10: target_rel_err
 * below 1e-10 returns ML_ERR_DOMAIN.  Dense clusters make the near field
 * quadratic: more than 2^40 examined pairs return ML_ERR_DOMAIN.
 */
ml_status ml_fastsum_plan_ex(ml_plan_t *out, const double *points, int64_t n, int d, double sigma,
                             const ml_plan_params *params, void *stream);

/*
 * ml_dense_plan - a dense layer for small graphs (the explicit regime, any
 * feature dimension): W_ij = exp(-||x_i - x_j||^2 / sigma^2), i != j (Sec. 2),
 * formed once on the GPU (squared distances summed from coordinate
 * differences in FP64) and stored n x n in FP64 (ML_F64) or FP32 (ML_F32);
 * the degrees are its row sums.  Products stream W once per pass of up to
 * 8 vectors with FP64 accumulation.  The plan is accepted everywhere a
 * fast-summation plan is (ml_fastsum_apply, the eigensolvers, layers mixed
 * with fast-summation layers).
 *   points  device, n x d row-major FP64, read during the call;  d >= 1.
 *   n       2..131072 (W takes n^2 x 8 or 4 bytes of device memory).
 * Synchronises `stream`.  Errors: ML_ERR_ARG, ML_ERR_OOM, ML_ERR_CUDA.
 *
 * ml_dense_plan_matrix - the same from a given symmetric weight matrix W
 * (device, n x n row-major FP64, e.g. the adjacency matrix of a stochastic
 * block model layer); its diagonal is taken as zero (no self-edges, Sec. 2).
 */
ml_status ml_dense_plan(ml_plan_t *out, const double *points, int64_t n, int d, double sigma, ml_prec prec,
                        void *stream);
ml_status ml_dense_plan_matrix(ml_plan_t *out, const double *W, int64_t n, ml_prec prec, void *stream);

/*
 * ml_fastsum_plan_autotune - ml_fastsum_plan_ex with the spreading tile (bin)
 * edge chosen by measurement (not from the paper: a GPU tuning step).  Plans
 * are built for the automatic rule's edge and a few edges around it, one
 * nv-vector product W X (ML_RAW_W) is timed on `stream` with CUDA events for
 * each (after one untimed product), and the fastest plan is returned; the
 * others are destroyed.  The winner is cached per layer shape (d, precision,
 * window width, grid size, active grid extents, nv, log2 n), so a later call
 * for a layer of the same shape builds one plan only.  Layers whose active
 * grid is a single tile have nothing to tune.
 *   params     as ml_fastsum_plan_ex (its bin field is ignored).
 *   nv         vectors per product the caller will apply (1..8).
 *   bin_chosen host, may be NULL: the chosen edge.
 * Synchronises `stream`.  Errors as ml_fastsum_plan_ex.
 */
ml_status ml_fastsum_plan_autotune(ml_plan_t *out, const double *points, int64_t n, int d, double sigma,
                                   const ml_plan_params *params, int nv, int *bin_chosen, void *stream);

/*
 * ml_fastsum_plan_many - the plans of T layers sharing n (ml_fastsum_plan_ex
 * with the same params for every layer), built concurrently by host threads,
 * each on its own non-blocking stream (not from the paper: plan set-up is
 * latency-bound, the layers are independent).
 *   out     host array of T handles (all NULL on failure).
 *   points  host array of T pointers (layer t: n x d[t] FP64), device memory
 *           ready in stream order on `stream`, or host memory (copied to the
 *           device by the layer's plan, as in ml_fastsum_plan).
 *   d, sigma host arrays of T.
 * Returns when every plan is complete.  Errors as ml_fastsum_plan_ex, with
 * the failing layer named in ml_last_error().
 */
ml_status ml_fastsum_plan_many(ml_plan_t *out, const double *const *points, int64_t n, const int *d,
                               const double *sigma, const ml_plan_params *params, int T, void *stream);

/*
 * ml_direct_sum_rows - the exact definition of the product on selected rows:
 * out[r] = sum_{j != rows[r]} exp(-||x_{rows[r]} - x_j||^2 / sigma^2) v_j
 * (W v of Sec. 2 / Sec. 4, direct O(nrows n) summation in FP64 on the GPU).
 * It is the reference for the fast summation's error and the product of the dense
 * regime for small graphs.
 *   points  device, n x d FP64;  v device, n FP64;  rows device, nrows int64
 *   (each in [0, n));  out device, nrows FP64.  Asynchronous on `stream`.
 */
ml_status ml_direct_sum_rows(const double *points, int64_t n, int d, double sigma, const double *v,
                             const int64_t *rows, int64_t nrows, double *out, void *stream);

/*
 * Point-cloud statistics used by the parameter model (not from the paper):
 *   [0] log10 n, [1] d, [2] log10(sigma / box) with box the largest bounding-box
 *   extent, [3..5] the bounding-box extents / box in decreasing order (0 past d),
 *   [6..8] log10 of the 5 %, 50 %, 95 % quantiles of the nearest-neighbour
 *   distance / sigma within an evenly strided sample of min(n, 2048) points.
 * points device n x d FP64; feat host, ML_FEATURES floats.  Synchronises `stream`.
 */
#define ML_FEATURES 9
ml_status ml_cloud_features(const double *points, int64_t n, int d, double sigma, float *feat, void *stream);

/*
 * Learned parameter model (not from the paper): a small FP32 MLP,
 * n_in -> hidden (tanh) -> hidden (tanh) -> n_out, with input and output
 * standardisation, trained and evaluated on the GPU by the library's own
 * kernels.  Parameters are packed [W1 (h x n_in), b1, W2 (h x h), b2,
 * W3 (n_out x h), b3], row-major.
 *   ml_mlp_create        random initialisation (SplitMix64 seed)
 *   ml_mlp_set_norm      x -> (x - in_mean)/in_std, y = out_mean + out_std * net
 *   ml_mlp_forward       X host or device (batch x n_in), Y same kind (batch x n_out)
 *   ml_mlp_loss_grad     mean squared error on standardised targets and its
 *                        gradient w.r.t. the packed parameters (host outputs)
 *   ml_mlp_train         `epochs` full-batch Adam steps (lr, beta 0.9/0.999);
 *                        loss per epoch to `losses` (host, may be NULL)
 *   ml_mlp_set_margins   3 safety factors on the error target, one per
 *                        bandwidth factor {0.7, 0.85, 1} of the planner below
 *                        (0 = use the planner's `margin` argument)
 * All return ML_ERR_ARG on size mismatches.
 */
typedef struct ml_mlp_s *ml_mlp_t;
ml_status ml_mlp_create(ml_mlp_t *out, int n_in, int hidden, int n_out, uint64_t seed);
int64_t ml_mlp_param_count(ml_mlp_t mlp);
ml_status ml_mlp_get_params(ml_mlp_t mlp, float *params, int64_t count);
ml_status ml_mlp_set_params(ml_mlp_t mlp, const float *params, int64_t count);
ml_status ml_mlp_set_norm(ml_mlp_t mlp, const float *in_mean, const float *in_std, const float *out_mean,
                          const float *out_std);
ml_status ml_mlp_forward(ml_mlp_t mlp, const float *X, int batch, float *Y);
ml_status ml_mlp_loss_grad(ml_mlp_t mlp, const float *X, const float *Yt, int batch, float *loss, float *grad);
ml_status ml_mlp_train(ml_mlp_t mlp, const float *X, const float *Yt, int batch, int epochs, float lr,
                       float *losses);
ml_status ml_mlp_set_margins(ml_mlp_t mlp, const double *margins, int count);
ml_status ml_mlp_destroy(ml_mlp_t mlp);

/*
 * ml_fastsum_plan_learned - plan with parameters chosen by a trained model
 * (n_in = ML_FEATURES + 3, n_out = 2: predicted log10 relative error and
 * log10 product time of a candidate).  Candidates: N = f * N0 for
 * f in {0.7, 0.85, 1} (N0 the automatic bandwidth for the target),
 * taps in {4..8}, oversampling in {2, 2.5, 3}; the model input is the cloud's
 * features followed by (f, taps, oversampling).  The cheapest candidate whose
 * predicted error is at most target / margin is used (margin: the model's
 * per-factor margin when set, else the argument); if none qualifies, or
 * mlp is NULL, the automatic choice of ml_fastsum_plan is used.
 * `chosen` (host, may be NULL) receives {f, taps, oversampling}.
 */
ml_status ml_fastsum_plan_learned(ml_plan_t *out, const double *points, int64_t n, int d, double sigma,
                                  ml_prec prec, double target_rel_err, ml_mlp_t mlp, double margin,
                                  double *chosen, void *stream);

/*
 * ml_fastsum_apply - Y = multilayer operator applied to X (Alg. 1 per layer,
 * then the D^{-1/2} scaling and the 1/T sum of Eq. I-L_1).
 *
 *   layers, T   T >= 1 plans sharing n.
 *   X           host or device, n x b FP64 (T blocks with ML_PER_LAYER);
 *               ignored for ML_DEGREE.
 *   b           vectors per block, 1..64.
 *   Y           host or device, n x b FP64 (T blocks with ML_PER_LAYER),
 *               overwritten.  Must not overlap X.
 *   mode        ML_RAW_W, ML_NORMALIZED_A or ML_DEGREE, optionally | ML_PER_LAYER.
 * Asynchronous on `stream` for device X and Y; with host X or Y the call
 * copies through plan-owned buffers and synchronises `stream`.  Two calls
 * that use the same plan must not run concurrently (they share its
 * workspace).  Errors: ML_ERR_ARG, ML_ERR_OOM, ML_ERR_CUDA, ML_ERR_DEGREE
 * (ML_NORMALIZED_A on a layer with a degree <= 0).
 */
ml_status ml_fastsum_apply(const ml_plan_t *layers, int T, const double *X, int b, double *Y,
                           int mode, void *stream);

/*
 * ml_fastsum_apply_noalloc - ml_fastsum_apply without any device allocation.
 * (Not from the paper: the paper has no counterpart; it is a deployment aid.)
 *
 * Who needs it: callers that must not call cudaMalloc/cudaFree during the
 * matrix-vector product, e.g. code that runs under a memory allocator which
 * owns the whole device (a framework's caching allocator), real-time or
 * latency-bound loops where an allocation stalls or synchronises the device,
 * and embedded/safety builds where allocation after start-up is forbidden.
 * ml_fastsum_apply may grow the plan's workspace (and, for host X/Y, its
 * staging buffers) with cudaMalloc; this entry point never does.
 *
 * How: all scratch of the call - the spreading tiles of every subproblem and
 * the two grid-transform buffers - is taken from one file-scope device array
 * of 32 MiB (every GPU that loads the library holds it until the process
 * exits).  The plans' own data were allocated by ml_fastsum_plan.
 *
 * Arguments and results are those of ml_fastsum_apply, except:
 *   - X and Y must be device memory (host buffers would need staging copies);
 *     ML_ERR_ARG otherwise.
 *   - ML_ERR_ARG, with the required size in ml_last_error(), when the layers'
 *     scratch (tiles and their boxes + two transform buffers at the widest
 *     vector pass)
 *     exceeds 32 MiB.
 *   - kernel timing (ml_profile_enable) is not recorded for these calls.
 * Set-up: the first call on each device looks the array's device address up
 * with cudaGetSymbolAddress (with that device current); make that first call
 * before any stream capture.  The address is kept for the life of the
 * process: after cudaDeviceReset (or anything else that destroys the
 * device's primary context) do not call this entry point again in that
 * process.
 * Sharing: every call uses the same array and leaves its contents behind; the
 * kernels read only scratch values that the same call wrote (FP32 tiles are
 * written and read within the box of cells their points reach), so nothing
 * needs clearing, but calls whose executions overlap on the GPU (other streams,
 * other threads) race on the array and must be serialised by the caller.
 * ML_DEGREE reads stored degrees and uses no scratch.
 */
ml_status ml_fastsum_apply_noalloc(const ml_plan_t *layers, int T, const double *X, int b, double *Y,
                                   int mode, void *stream);

/*
 * ml_lanczos_eigs - the k smallest eigenpairs of the power mean Laplacian of
 * the T layers by thick-restart Lanczos with full reorthogonalisation (Sec. 3).
 *
 *   p == 1   eigenpairs of L_1: the k largest theta of I - L_1 (Eq. I-L_1),
 *            lambda = 1 - theta.
 *   p < 0    eigenpairs of L_{p,delta}, delta = log(1+|p|): the k largest mu
 *            of L_{p,delta}^p = (1/T) sum_t (L_sym^(t) + delta I)^p
 *            (Eq. L_p_delta_power_p), lambda = mu^(1/p).  For p = -1 each
 *            term is an inner conjugate gradient solve driven by the fast
 *            summation; for other p in [-64, 0) it is the Lanczos
 *            approximation of the matrix power (tridiagonal solves for
 *            integer p, the tridiagonal eigendecomposition otherwise),
 *            stopped at relative change max(1e-12, 1e-2 tol).
 *   tol      relative residual ||A phi - theta phi|| <= tol * |theta_max|
 *            (<= 0: 1e-10).
 *   maxit    limit on outer operator applications (<= 0: 2000).
 *   block    1 (single-vector Lanczos); reserved for block variants.
 *   seed     seed of the start vector (SplitMix64 counter stream).
 *   evals    host, k FP64: ascending eigenvalues lambda of L_1 / L_{p,delta}.
 *   evecs    host or device, n x k FP64, column-major (column j contiguous),
 *            unit 2-norm, sign fixed so the largest-magnitude entry is
 *            positive; may be NULL.
 *   nconv    host, number of converged pairs (may be NULL).
 * Synchronises `stream`.  Returns ML_WARN_NOT_CONVERGED when maxit is reached
 * with fewer than k converged pairs (evals/evecs then hold the best Ritz
 * pairs); ML_ERR_ARG for k < 1, k > n/2, p not 1 and not in [-64, 0).
 */
ml_status ml_lanczos_eigs(const ml_plan_t *layers, int T, int k, double p, double tol, int maxit,
                          int block, uint64_t seed, double *evals, double *evecs, int *nconv,
                          void *stream);

/*
 * ml_lanczos_eigs_layers - for every layer t separately, the k smallest
 * eigenpairs of L_sym^(t) = I - D_t^{-1/2} W_t D_t^{-1/2} (Sec. 2), by block
 * thick-restart Lanczos with full reorthogonalisation (the Lanczos method of
 * Sec. 3 with `block` vectors per step).  All T eigenproblems advance
 * together: each step applies every unfinished layer's operator to its own
 * block in one batched fast summation (one launch per stage when the layers
 * are FP32 plans of one d and window width) and orthogonalises all blocks
 * with kernels batched over the layers.  A layer leaves the batch when its
 * k pairs have converged.
 *
 *   layers, T  T >= 1 plans sharing n.
 *   k          1 <= k <= n/2; the basis (ncv plus one block) must stay within
 *              96 columns (k <= ~30 at block = 8 with the automatic ncv).
 *   tol        relative residual ||A phi - theta phi|| <= tol * |theta_max|
 *              per layer (<= 0: 1e-10).
 *   maxit      limit on operator applications per layer (<= 0: 2000).
 *   block      vectors per step, 1..8.
 *   ncv        basis columns per restart cycle (rounded up to a multiple of
 *              block), or 0 for max(2k+1, 20) + block rounded up; at most
 *              96 - block.  After a cycle the largest Ritz vectors (about
 *              (ncv+k)/2 of them) are kept.
 *   seed       seed of the start blocks (SplitMix64 counter streams, one per layer).
 *   evals      host, T x k FP64 (row t: ascending eigenvalues of L_sym^(t)).
 *   evecs      host or device, T blocks of n x k FP64 column-major (block t =
 *              layer t), unit 2-norm, largest-magnitude entry positive; may be NULL.
 *   nconv      host, T ints: converged pairs per layer (may be NULL).
 * Synchronises `stream`.  Returns ML_WARN_NOT_CONVERGED when some layer
 * reached maxit with fewer than k converged pairs; ML_ERR_ARG for k or block
 * out of range; ML_ERR_DEGREE for a layer with a degree <= 0.  When a block
 * becomes numerically rank-deficient its dependent directions are dropped
 * (the block deflates) instead of failing; dropped directions take no part
 * in the Rayleigh-Ritz step, so a layer whose basis holds fewer than k
 * directions reports ML_WARN_NOT_CONVERGED with NaN in the evals entries
 * that have no Ritz pair.  Each block step removes the three-term terms
 * first and runs its second Gram-Schmidt pass only where the first removed
 * more than half of some column's norm squared.
 */
ml_status ml_lanczos_eigs_layers(const ml_plan_t *layers, int T, int k, double tol, int maxit, int block,
                                 int ncv, uint64_t seed, double *evals, double *evecs, int *nconv, void *stream);

/* Parameters of the Allen-Cahn scheme (Sec. 6; the image experiments of Sec. 8
 * use eps = 0.005, omega0 = 1000, c = omega0 + 3/eps, dt = 0.01, tol = 1e-6,
 * max_iter = 500). */
typedef struct {
    double eps;     /* interface parameter epsilon > 0                        */
    double omega0;  /* fidelity weight of the labelled nodes                  */
    double c;       /* convexity-splitting constant; <= 0: omega0 + 3/eps      */
    double dt;      /* time step                                              */
    double tol;     /* stop when relative_change <= tol                        */
    int max_iter;   /* iteration limit, >= 1                                   */
} ml_ac_params;

/*
 * ml_allen_cahn - class scores of every node by the multiclass multilayer
 * graph Allen-Cahn scheme (Alg. 2, steps 2-4) from k eigenpairs of L_1 or
 * L_{p,delta} (e.g. ml_lanczos_eigs):
 *   Z = [(1 + c dt) I + eps dt Lambda_k]^{-1} Phi_k^T;
 *   U^0: e_j on labelled nodes of class j, (1/m) 1 elsewhere;
 *   repeat: T^l = T(U^l) (Eq. def:T_ij),
 *           V^{l+1} = Z((1 + c dt) U^l - dt/(2 eps) T^l - dt omega (U^l - F)),
 *           U^{l+1} = rows of Phi_k V^{l+1} projected onto the Gibbs simplex
 *                     (sort-and-threshold projection of Chen & Ye 2011),
 *   until max_i ||u_i^{l+1} - u_i^l||^2 / max_i ||u_i^{l+1}||^2 <= tol or
 *   max_iter iterations.
 *   Phi        device, n x k FP64 column-major (the eigenvectors).
 *   lambda     host, k FP64 (the eigenvalues of the Laplacian).
 *   labels     device, n int32: class id in [0, m) of labelled nodes, -1 else.
 *   m          classes, 2..16;  k in 1..64.
 *   U          device, n x m FP64 point-major: the scores of the last iterate.
 *   pred       device, n int32 (may be NULL): row-wise argmax of U, ties to
 *              the lowest class id.
 *   iters, last_change  host (may be NULL): iterations done and their last
 *              relative change.
 * All arithmetic FP64.  Synchronises `stream`.  ML_ERR_ARG for sizes or
 * labels out of range.
 */
ml_status ml_allen_cahn(const double *Phi, const double *lambda, int64_t n, int k, const int *labels, int m,
                        const ml_ac_params *params, double *U, int *pred, int *iters, double *last_change,
                        void *stream);

/* Copy the plan's parameters into *info (host).  Never fails on a valid plan. */
ml_status ml_plan_get_info(ml_plan_t plan, ml_plan_info *info);

/*
 * ml_plan_copy_table - copy one of the plan's host-side FP64 tables (for
 * tests and inspection):
 *   which = 0: b_l for l = 0..N/2 in every dim, (N/2+1)^d values, dim 0 fastest
 *              (the Fourier coefficients of K_RF, Eq. K_RF; b_l is even in each l_a)
 *   which = 1: the window's Fourier coefficients phi_hat(k), k = 0..N/2
 *   which = 2: the degrees D_i in input order (n values)
 * `out` is host memory of `count` doubles; count must be at least the size.
 */
ml_status ml_plan_copy_table(ml_plan_t plan, int which, double *out, int64_t count);

/*
 * Kernel timing (tracing; the paper has no counterpart).  While enabled, every
 * library kernel launch is bracketed by two CUDA events recorded on the
 * stream it is launched on; ml_profile_read synchronises those events and
 * returns, per kernel family ("spread", "fold", "axis", "mult", "interp",
 * "dots", "update", ...), the number of launches and the summed device time.
 *   ml_profile_enable(1/0)   switch recording on/off (off by default)
 *   ml_profile_reset()       drop all records
 *   ml_profile_read(i, name, launches, ms): entry i (0-based) of the table;
 *            returns ML_ERR_ARG when i is past the end.  `name` receives a
 *            pointer to a static string owned by the library.
 * Recording costs two event records per launch; it is meant for measurement
 * runs, not for production.
 */
ml_status ml_profile_enable(int on);
ml_status ml_profile_reset(void);
ml_status ml_profile_read(int i, const char **name, int64_t *launches, double *ms);
/*
 * Dense products of the Lanczos solvers on the fp16 tensor cores (Sec. 3:
 * the block Gram-Schmidt reorthogonalisation, the three-term update and the
 * Ritz vectors are products of the Krylov basis with small matrices).  FP64
 * operands are split into eight 8-bit slices (64-bit fixed point), every
 * slice product is summed exactly in FP32 on the tensor cores (tcgen05.mma,
 * at most 256 rows between integer drains), the pairs of slices whose weight
 * is above 2^-70 are combined in 64-bit integers and converted to FP64 once
 * (the error-free splitting of Ozaki, Ogita, Oishi and Rump, Numer.
 * Algorithms 59 (2012)).  The result is as accurate as an FP64 product
 * where it matters for an orthonormal basis: each entry's error is at most a
 * few units of 2^-53 times sum_i |a_i||b_i|, plus the resolution of A's fixed
 * scale, 2^-62 times the sum of the other factor's magnitudes.
 *
 * ml_block_gram - G = A^T B.
 *   A   device, n x rc, row i at A + i * lda (point-major), |A_ij| < 2
 *       (e.g. orthonormal basis columns); rc in 1..48.
 *   B   device, n x cb, row i at B + i * ldb, any magnitude (each column is
 *       scaled by a power of two over the rows one thread block handles);
 *       cb in 1..8.
 *   G   device, rc x cb row-major FP64, overwritten.
 * ml_block_update - Y[:, 0:cb] = A M, or Y[:, 0:cb] -= A M with sub != 0.
 *   A   device, n x rc as above (|A_ij| < 2, rc in 1..48).
 *   M   device, rc x cb row-major FP64, any magnitude (scaled per column).
 *   Y   device, n x cb, row i at Y + i * ldy; may be A itself only when the
 *       columns written are not columns read.
 * Both synchronise `stream` (they read the device's status flag).  Errors:
 * ML_ERR_ARG (sizes), ML_ERR_DOMAIN (an entry of A with |v| >= 2),
 * ML_ERR_TIMEOUT (a bounded wait of the kernel gave up), ML_ERR_OOM,
 * ML_ERR_CUDA.
 *
 * ml_set_dense_products - how the eigensolvers form their products of the
 * Krylov basis (Q^T x, x - Q h, the Ritz vectors Q S; in the per-layer
 * solver the block Gram and update products on the tensor cores only):
 *   kind = 0  on the FP64 pipe;
 *   kind = 1  (default) in double-word arithmetic on the FP32 pipes (each
 *             value an unevaluated pair of floats, about 47 significant
 *             bits; exact products by FMA, compensated sums): GB300 runs
 *             FP64 at 1/64 of the FP32 rate, and these products are bound by
 *             it on the FP64 pipe;
 *   kind = 2  on the tensor cores as above (FP64-accurate, but not faster
 *             for these shapes: the slicing of every FP64 element costs more
 *             issue slots than the multiply-adds it replaces).
 * Process-wide.  A tensor-core solve that meets an operand beyond |v| < 2
 * repeats itself on the FP64 pipe.  ML_ERR_ARG for other kinds.
 */
ml_status ml_block_gram(const double *A, int64_t n, int rc, int64_t lda, const double *B, int cb, int64_t ldb,
                        double *G, void *stream);
ml_status ml_block_update(const double *A, int64_t n, int rc, int64_t lda, const double *M, int cb, double *Y,
                          int64_t ldy, int sub, void *stream);
ml_status ml_set_dense_products(int kind);

/*
 * ml_measure_peak - measured throughput of one GPU resource, the denominator
 * of a roofline fraction (measurement aid; the paper has no counterpart).
 * Runs a micro-kernel on the current device, 8 CTAs of 256 threads per SM,
 * one untimed and three timed launches on `stream` (CUDA events), and
 * returns the best of the three:
 *   what = 0   FP32 FMA pipe: 8 independent fmaf chains per thread, in
 *              TFLOP/s (2 flop per FMA);
 *   what = 1   FP64 FMA pipe, the same with doubles, in TFLOP/s;
 *   what = 2   32-bit integer shared-memory atomic adds on conflict-free
 *              addresses (one wavefront per warp instruction), in 1e12
 *              atomics per second.
 *   rate       host, receives the figure.
 * Synchronises `stream`.  Errors: ML_ERR_ARG (what out of range, rate
 * NULL), ML_ERR_OOM, ML_ERR_CUDA.
 */
ml_status ml_measure_peak(int what, double *rate, void *stream);

/* CUDA-graph replays of captured inner solver iterations since the library
 * was loaded (diagnostics: 0 means every iteration launched eagerly). */
int64_t ml_graph_replays(void);

/* Release the plan and all device memory it owns.  NULL is accepted.  Blocks
 * of 1 MiB and more are kept by the library for later plans and workspaces of
 * the same device (a per-device cache of at most 64 GiB, filled after a device
 * synchronisation), so that plans made step after step do not pay for the
 * driver's allocations; ml_release_cached_memory returns them to the driver. */
ml_status ml_plan_destroy(ml_plan_t plan);

/* Free the library's cached device blocks of the current device (after a
 * device synchronisation), and return the memory its stream-ordered pool for
 * plan-time temporaries keeps.  Errors: ML_ERR_CUDA. */
ml_status ml_release_cached_memory(void);

/* Thread-local description of the last failure on this thread ("" if none). */
const char *ml_last_error(void);

/* Library version string. */
const char *ml_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ML_FASTSUM_H */
