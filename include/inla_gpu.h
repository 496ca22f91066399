/*
 * inla_gpu.h -- C ABI of the GB300 library for INLA's hyperparameter phase.
 *
 * What it computes (Gaedke-Merzhaeuser et al., "Parallelized integrated
 * nested Laplace approximations for fast Bayesian inference"):
 *
 *   For each hyperparameter point theta of a batch, the objective
 *     f(theta) = -log pi~(theta | y)                          (Sec. 3.1)
 *   where pi~ is the Laplace approximation of Eq. post_theta_approx,
 *     pi~(theta|y) = pi(theta) pi(x|theta) pi(y|x,theta) / pi_G(x|theta,y) at x = x*(theta),
 *   together with its gradient (central differences, Eq. central_diff, or
 *   an adjoint of the same formula), the latent mode x*(theta) (Sec. 2.2;
 *   Newton iteration for Poisson and binomial data), and the marginal variances
 *   diag(Q_c(theta)^-1) by selected inversion (Sec. 2.3, Sec. 2.4.2,
 *   Eq. sel_inv_cov / Eq. takahashi_recursion).
 *
 * The model is the spatio-temporal latent Gaussian model of Sec. 2.1 with
 *   Q(theta)   = Q_t(rho) (x) Q_s(kappa, tau) (+) tau_b I_{n_b},
 *   Q_s        = tau^2 (kappa^4 C + 2 kappa^2 G + G C^-1 G)   (SPDE, alpha = 2),
 *   Q_t        = stationary AR(1) precision, unit marginal variance,
 *   Q_c(theta) = Q(theta) + A^T D A,  D = tau_y I (Gaussian) or diag(b''(eta)) at the
 *   current latent field (Poisson: E e^eta; binomial: N p (1 - p)),
 * latent vector ordered time-major with the n_b fixed effects last, so
 * Q and Q_c are block tridiagonal with an arrowhead (Fig. arrowhead_matrices).
 * theta = (theta_1..theta_4): Gaussian: (log tau_y, log range, log sigma,
 * logit rho) with kappa = sqrt(8)/range, tau^2 = 1/(4 pi kappa^2 sigma^2) and
 * tau_b fixed by the model; Poisson and binomial data: theta_1 = log tau_b instead of log tau_y.
 * The prior pi(theta) is a product of independent normals.
 *
 * Conventions
 *   - Every function returns an inla_status; 0 = INLA_OK.  On a non-OK
 *     return, inla_last_error() gives a message (thread-local).
 *   - Argument, size and allocation errors are reported synchronously.
 *     Numerical failures are reported per point in out->status[b]:
 *     INLA_ERR_NOT_SPD (a pivot block lost positive definiteness),
 *     INLA_ERR_NO_CONVERGENCE (Newton did not reach the tolerance); such a
 *     point gets f = +inf and NaN in its other outputs.  Kernels never trap
 *     and contain no unbounded waits.
 *   - Pointers named *_dev are device pointers, all others host pointers.
 *     All floating point is IEEE binary64 ("double"), arrays are dense and
 *     contiguous (row-major where two-dimensional).
 *   - Calls on one model share its device workspace.  The library orders
 *     each evaluation after the previous one on the same model, whatever
 *     the streams, so results are never mixed; a model must still not be
 *     used from two host threads at once.  Distinct models are independent.
 */
#ifndef INLA_GPU_H
#define INLA_GPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  INLA_OK = 0,
  INLA_ERR_ARG = 1,             /* invalid argument or inconsistent sizes      */
  INLA_ERR_CUDA = 2,            /* a CUDA runtime call failed                  */
  INLA_ERR_OOM = 3,             /* device allocation failed                    */
  INLA_ERR_NOT_SPD = 4,         /* per point: Q or Q_c not positive definite   */
  INLA_ERR_NO_CONVERGENCE = 5,  /* per point: Newton iteration did not converge */
  INLA_ERR_TIMEOUT = 6,         /* per point: a bounded device-side wait ran out */
  INLA_ERR_UNSUPPORTED = 7      /* option not available in this build          */
} inla_status;

/* Likelihoods: Gaussian y ~ N(eta, 1/tau_y); Poisson y ~ Pois(E exp(eta));
 * binomial y ~ Bin(N, 1 / (1 + exp(-eta))) with the number of trials N in the
 * E array; negative binomial y ~ NB(mean E exp(eta), size r) with the size r
 * (overdispersion, var = mean + mean^2 / r) a fixed model constant (nb_size).
 * The non-Gaussian ones are handled by the Laplace approximation with a Newton
 * inner loop (Sec. 2.2); for the negative binomial's log link, which is not
 * canonical, the Newton weight is the observed information. */
enum { INLA_LIK_GAUSSIAN = 0, INLA_LIK_POISSON = 1, INLA_LIK_BINOMIAL = 2, INLA_LIK_NEGBINOMIAL = 3 };
/* Gradient of f: none; central differences (Eq. central_diff: 2d + 1 = 9
 * evaluations per centre); the adjoint (selected-inverse traces, one extra
 * solve for non-Gaussian data); forward differences (d + 1 = 5 evaluations
 * per centre, (f(theta + eps e_j) - f(theta)) / eps, first-order accurate: the
 * cheaper scheme the paper mixes in for later iterations). */
enum { INLA_GRAD_NONE = 0, INLA_GRAD_FD_CENTRAL = 1, INLA_GRAD_ADJOINT = 2, INLA_GRAD_FD_FORWARD = 3 };
/* How log|Q| and tr(Q^-1 dQ) of the prior are obtained.  KRONECKER uses
 * log|Q_t (x) Q_s| = n_s log|Q_t| + n_t log|Q_s| with one dense n_s x n_s
 * inversion of Q_s; BTA runs the same block factorisation (and selected
 * inversion, for the gradient) on Q as on Q_c.  Both are exact. */
enum { INLA_PRIOR_KRONECKER = 0, INLA_PRIOR_BTA = 1 };
/* Arithmetic of the dense n_s x n_s blocks (the Schur-complement inverses,
 * their sweep updates and the selected-inversion products).  INLA_FP64: all
 * FP64.  INLA_MIXED: those blocks are stored and multiplied in FP32, while
 * the pivot-block inversions, every log-determinant, the sparse assembly
 * inputs, all vectors, reductions and traces stay FP64, and the mode is
 * refined with FP64 residuals r = b - Q_c x (three refinement steps). */
enum { INLA_FP64 = 0, INLA_MIXED = 1 };
/* FP32 GEMM of the mixed selected inversion (inla_set_tiles): 64 or 128 =
 * FP32 FMA on the CUDA cores with 64 x 64 or 128 x 128 output tiles;
 * INLA_GEMM_TF32X3 = 128 x 128 tiles on the tensor cores (tcgen05, kind::tf32)
 * with the 3xTF32 split product, used where n_s rounded up to 64 is a
 * multiple of 128 (elsewhere the 128 x 128 CUDA-core GEMM runs). */
#define INLA_GEMM_TF32X3 3
/* FP32 block sweep (inla_set_tiles): 32 or 64 = pivot width with the rank-G
 * tile updates on the CUDA cores; INLA_SWEEP_TF32X3 = 64-wide pivots with the
 * rank-64 updates of the lower tiles on the tensor cores (tcgen05, kind::tf32,
 * 3xTF32 split product; the pivot row and column and the next pivot block stay
 * on the CUDA cores), used where n_s rounded up to 64 is a multiple of 128
 * (elsewhere the 64-wide CUDA-core sweep runs).  Not the default: with K = 64
 * per launch it measured slower than the CUDA-core update on GB300. */
#define INLA_SWEEP_TF32X3 3
/* FP32 blocks (inla_set_tiles): D_t^-1 by the 2 x 2 block recursion whose
 * products run on the tensor cores in 3xTF32 (TMA-fed, as the selected
 * inversion's), with 64-wide sweeps only on base blocks of at most 256 rows; used where
 * n_s rounded up to 64 is a multiple of 128 (elsewhere the 64-wide CUDA-core
 * sweep runs).  The default for FP32 blocks of 2048 rows or more. */
#define INLA_INV_BLOCKED 4

/* Model description.  Every pointer is a HOST pointer; the arrays are read
 * (and copied to the device) by inla_model_create and may be freed after it
 * returns. */
typedef struct {
  int32_t n_t;            /* number of time steps (>= 1)                          */
  int32_t n_s;            /* number of mesh vertices (>= 1)                       */
  int32_t n_b;            /* number of fixed effects (>= 0)                       */
  int32_t lik;            /* INLA_LIK_GAUSSIAN, _POISSON, _BINOMIAL, _NEGBINOMIAL  */
  int64_t m;              /* number of observations (>= 1)                        */
  const double *C_diag;   /* [n_s] lumped mass matrix C (all > 0)                 */
  const int32_t *G_rowptr;/* [n_s+1] CSR row pointers of the stiffness matrix G   */
  const int32_t *G_col;   /* [nnz(G)] column indices (symmetric pattern)          */
  const double *G_val;    /* [nnz(G)] values                                       */
  const int64_t *A_rowptr;/* [m+1] CSR row pointers of A (m x n, n = n_t n_s + n_b)*/
  const int32_t *A_col;   /* column indices: each row has 1..3 spatial entries in  */
                          /* one time block [t n_s, (t+1) n_s) and any number of   */
                          /* fixed-effect entries in [n_t n_s, n)                   */
  const double *A_val;    /* values                                                */
  const double *y;        /* [m] observations (Poisson, negative binomial:         */
                          /* non-negative integers; binomial: integers 0..N)       */
  const double *E;        /* [m] Poisson, negative binomial: exposures (> 0);      */
                          /* binomial: numbers of trials N (positive integers);    */
                          /* NULL for Gaussian                                      */
  double tau_b;           /* fixed-effect prior precision (Gaussian; > 0; the      */
                          /* other likelihoods take tau_b = exp(theta_1))          */
  double prior_mean[4];   /* hyperprior: theta_j ~ N(prior_mean[j], prior_sd[j]^2) */
  double prior_sd[4];
  double nb_size;         /* negative binomial: size r > 0 (ignored otherwise)     */
} inla_model_desc;

typedef struct {
  int32_t grad;           /* INLA_GRAD_NONE / _FD_CENTRAL / _ADJOINT               */
  int32_t prior_mode;     /* INLA_PRIOR_KRONECKER or INLA_PRIOR_BTA                */
  int32_t precision;      /* INLA_FP64 or INLA_MIXED                               */
  int32_t want_mode;      /* nonzero: write x*(theta) to out->x_mode               */
  int32_t want_marg_var;  /* nonzero: write diag(Q_c^-1) to out->marg_var          */
  int32_t max_newton;     /* Poisson/binomial: iteration limit (<= 0: 50)          */
  double newton_tol;      /* Poisson/binomial: stop when ||x^{k+1} - x^k||_2 < tol (<= 0: 1e-8) */
  double fd_eps;          /* central-difference step (<= 0: 1e-3)                  */
  int32_t use_graph;      /* nonzero (batch in one wave): the whole evaluation is   */
                          /* captured once per batch size and options as a CUDA    */
                          /* graph and replayed on later calls; for Poisson and     */
                          /* binomial data the Newton loop is a conditional while   */
                          /* node that repeats on the device until every point has  */
                          /* converged or hit max_newton (no host synchronisation)  */
} inla_eval_opts;

/* Outputs of inla_eval_batch: DEVICE pointers owned by the caller.  Layout
 * is [B] or [B][n] / [B][4] row-major.  x_mode, marg_var, grad and
 * newton_iters may be NULL when not wanted. */
typedef struct {
  double *f_dev;          /* [B]    f(theta_b)                                     */
  double *grad_dev;       /* [B][4] gradient (needs opts.grad != NONE)             */
  double *x_mode_dev;     /* [B][n] latent mode x*(theta_b)                        */
  double *marg_var_dev;   /* [B][n] diag(Q_c(theta_b)^-1), latent order            */
  int32_t *status_dev;    /* [B]    per-point inla_status (required)               */
  int32_t *newton_iters_dev; /* [B] Newton iterations (Poisson/binomial), 0 for Gaussian */
} inla_eval_out;

/* Host-buffer twin of inla_eval_out (all HOST pointers, same layout). */
typedef struct {
  double *f;
  double *grad;
  double *x_mode;
  double *marg_var;
  int32_t *status;
  int32_t *newton_iters;
} inla_eval_out_host;

typedef struct inla_model inla_model;

/* Build a model on CUDA device `device` (the latent Gaussian model of Sec. 2.1:
 * the spatial SPDE and temporal AR(1) precisions, the fixed effects and the
 * observation matrix A of the linear predictor): validates the description, sorts
 * the observations by time, builds the index structures on the host and
 * computes every theta-free value (G C^-1 G, A^T A, A^T y, ...) with device
 * kernels.  On success *out owns all device memory of the model.
 * Errors: INLA_ERR_ARG (bad sizes / indices / values), INLA_ERR_OOM,
 * INLA_ERR_CUDA.  Synchronous. */
int inla_model_create(const inla_model_desc *desc, int device, inla_model **out);

/* Bytes of device workspace that inla_eval_batch allocates (and keeps in
 * the model for reuse) for a batch of B points with these options: per point
 * the block factorisation of Sec. 2.4 (n_t inverted n_s x n_s Schur blocks)
 * and two live blocks of the selected inversion (Sec. 2.4.2).  Central
 * differences (Eq. central_diff) evaluate B * 9 points.  model and opts are
 * HOST pointers, *bytes is written on success.  Errors: INLA_ERR_ARG. */
int inla_workspace_bytes(const inla_model *model, int B, const inla_eval_opts *opts, size_t *bytes);

/* Evaluate B >= 1 points (B = 0 is an argument error).  theta_dev: DEVICE [B][4].  out: DEVICE buffers as
 * above.  stream: a cudaStream_t (NULL = legacy default stream).  Work is
 * enqueued on `stream`; the call returns after enqueueing, except for
 * Poisson and binomial data without use_graph, whose Newton loop reads a
 * convergence flag back to the host once per iteration (with use_graph the
 * loop runs on the device).  The workspace grows on first use (device
 * allocation), so the first call with a larger B may allocate.
 * With opts->grad == INLA_GRAD_FD_CENTRAL each point is the centre of a
 * 2d+1 = 9 point stencil (Eq. central_diff); f, x_mode and marg_var are
 * those of the centre.  Errors: INLA_ERR_ARG, INLA_ERR_OOM, INLA_ERR_CUDA,
 * INLA_ERR_UNSUPPORTED; numerical failures go to out->status_dev. */
int inla_eval_batch(inla_model *model, int B, const double *theta_dev, const inla_eval_opts *opts,
                    const inla_eval_out *out, void *stream);

/* No counterpart in the paper: a variant of inla_eval_batch that allocates no
 * device memory, for callers that cannot call cudaMalloc once they are
 * running -- a serving loop that must keep a fixed device-memory footprint
 * after start-up, or a plugin inside a host framework whose own caching
 * allocator owns the device memory, so that a raw cudaMalloc could fail or
 * fragment that pool.  Its workspace is one array of INLA_STATIC_SCRATCH_BYTES
 * (64 MiB), a file-scope __device__ array of the library.  The array is
 * committed on a device, and its device address looked up with that device
 * current, by the first inla_model_create on that device; from then on every
 * GPU that has a model holds it until the process exits.  The model itself
 * (inla_model_create) allocates, so create models at start-up.  Kernel code
 * is loaded on first use under the CUDA runtime's default lazy module
 * loading, which the driver backs with a little device memory; callers that
 * need the very first call to touch no new device memory either set
 * CUDA_MODULE_LOADING=EAGER or make one warm-up call at start-up.
 * Arguments, outputs and results are those of inla_eval_batch, with two
 * differences: opts->use_graph is ignored (the call always launches its
 * kernels directly), and for Poisson and binomial data the call reads a
 * convergence flag back to the host once per Newton iteration, as
 * inla_eval_batch does without use_graph.  The whole batch must fit in the
 * array in one pass: inla_workspace_bytes() plus about 96 bytes per point
 * (B points, or 9 B with central differences) up to 64 MiB; a larger batch
 * returns INLA_ERR_ARG and does nothing.  All calls on a device share the
 * array, which keeps the last call's contents (every call clears what it
 * needs); calls on one model are ordered like inla_eval_batch, but calls from
 * two models that overlap on the GPU race on the array.  Errors as for
 * inla_eval_batch. */
#define INLA_STATIC_SCRATCH_BYTES ((size_t)64 << 20)
int inla_eval_batch_static(inla_model *model, int B, const double *theta_dev, const inla_eval_opts *opts,
                           const inla_eval_out *out, void *stream);

/* Same as inla_eval_batch with HOST buffers: copies theta to the device,
 * evaluates on the model's internal stream, copies the results back and
 * synchronises.  theta: HOST [B][4]. */
int inla_eval_batch_host(inla_model *model, int B, const double *theta, const inla_eval_opts *opts,
                         const inla_eval_out_host *out);

/* Tile autotuner (the project's own; no counterpart in the paper).  Times
 * full evaluations of this batch (theta_dev: DEVICE [B][4], opts as for
 * inla_eval_batch) for each candidate block-tile shape of the precision in
 * opts -- the sweep's pivot/tile width (32 or 64; in INLA_MIXED also
 * INLA_SWEEP_TF32X3) and, in INLA_MIXED, the FP32 GEMM (64, 128 or
 * INLA_GEMM_TF32X3) -- keeps the fastest in the model for later
 * calls, and writes {FP64 sweep width, FP32 sweep width, FP32 GEMM tile} to
 * choice[3] (may be NULL).  Synchronous; allocates and frees its own trial
 * output buffers; drops captured graphs of the model.  Results of every
 * candidate agree to rounding (all are the same algorithm). */
int inla_autotune(inla_model *model, int B, const double *theta_dev, const inla_eval_opts *opts, int32_t *choice);

/* Set the tile shapes explicitly (e.g. a choice saved from inla_autotune):
 * sweep width 32 or 64 for FP64 blocks; 32, 64, INLA_SWEEP_TF32X3 or
 * INLA_INV_BLOCKED for FP32 blocks; FP32 GEMM 64, 128 or INLA_GEMM_TF32X3.  A
 * new model starts at (32, 64 or INLA_INV_BLOCKED by size, INLA_GEMM_TF32X3).
 * Errors: INLA_ERR_ARG for other values. */
int inla_set_tiles(inla_model *model, int sweep_fp64, int sweep_fp32, int gemm_fp32);

/* Bound on each wait of the tensor-core kernels for their own asynchronous
 * copies and matrix products (no counterpart in the paper; the library's
 * failure detection).  Process-wide; seconds in (0, 2], default 2; below
 * 1e-6 every wait is a single non-blocking test of completion.  A wait
 * that runs out marks its evaluation point INLA_ERR_TIMEOUT (f = +inf, NaN in
 * the point's other outputs) -- or, in inla_gemm_tf32x3, its batch entry --
 * and the kernel then waits, with the full 2 s bound, for the work it has in
 * flight before it releases its shared and tensor memory and returns.  Takes
 * effect for kernels launched after the call; a CUDA graph keeps the limit it
 * was captured with.  Errors: INLA_ERR_ARG. */
int inla_set_wait_limit(double seconds);

/* Where the FP64 path's selected-inversion products run (Eq. sel_inv_cov on
 * the n_s x n_s blocks, 3 n_s^3 flops per time step): tensor = 1 (the default)
 * on the BF16 tensor cores through error-free digit splitting (as
 * inla_gemm_f64), used where n_s rounded up to 64 is a multiple of 128;
 * tensor = 0 with FP64 FMA on the CUDA cores.  Both meet the FP64 tolerances;
 * results differ in rounding.  Drops captured graphs.  Errors: INLA_ERR_ARG. */
int inla_set_fp64_products(inla_model *model, int tensor);

/* Nested dissection of the time chain (Sec. 3.3: the independent blocks Q_A and
 * Q_B are factorised in parallel before their separator Q_S, and the partial
 * inverse is computed the other way round, the separator's entries first).
 * parts = 2 (the default, for n_t >= 3): every factorisation splits the chain
 * at its middle block k = n_t / 2 -- blocks 0..k-1 and n_t-1..k+1 are eliminated
 * as two independent chains on two streams, then block k with the Schur
 * complements of both neighbours, then the fixed effects; the block substitution
 * for the mode and the selected inversion (block k first, then both chains
 * outwards) run in the matching order.  No fill and no extra flops: the same
 * log-determinants, mode, marginal variances and gradients up to rounding, in
 * half the sequential steps, with a second set of per-point scratch blocks in
 * the workspace (inla_workspace_bytes).  parts = 1: one chain, from t = 0 up.
 * Takes effect at the next call.  Errors: INLA_ERR_ARG. */
int inla_set_time_partition(inla_model *model, int parts);

/* Point groups (the paper's "level 1" parallelism over independent evaluation
 * points, Sec. 3.1, applied inside one call).  groups = 2: for Gaussian data in
 * calls with use_graph the factorisation of Q_c and the solve for the mode run
 * as two groups of points (the first and second half of each wave), each on its
 * own pair of streams, concurrently; the dense kernels of a wave are
 * latency-bound, so two groups of half the points overlap (groups = 2 is the
 * default; eager calls keep one group, whose launches cost half the host
 * time).  Results are
 * bit-identical to groups = 1: every point's arithmetic is unchanged.  Takes
 * effect at the next call.  Errors: INLA_ERR_ARG. */
int inla_set_point_groups(inla_model *model, int groups);

/* Latent dimension n = n_t n_s + n_b of a model. */
int64_t inla_model_latent_dim(const inla_model *model);

/* Number of kernel launches the last inla_eval_batch issued (diagnostics). */
int64_t inla_last_launch_count(const inla_model *model);

/* Live kernel timing (diagnostics, off by default).  While enabled
 * (enable = k >= 1), every k-th launch of each kernel below is bracketed by
 * CUDA events on the launch stream; inla_profile_read synchronises those events and returns, for one
 * kernel, the summed event time in ms, the number of launches and the
 * number of algorithmic units processed (a unit is one 64 x 64 x 64 tile
 * product, 2 * 64^3 flops).  Enabling resets the records.
 *   kernel 0: tile update of the block sweep inversion, FP64 blocks
 *   kernel 1: tile GEMM of the selected inversion (FP64, FP32, or 3xTF32
 *             on the tensor cores)
 *   kernel 2: pivot-block inversion        kernel 3: pivot-panel product
 *   kernel 4: tile update of the block sweep inversion, FP32 blocks */
int inla_profile_enable(inla_model *model, int enable);
int inla_profile_read(inla_model *model, int kernel, double *total_ms, int64_t *launches, double *units);

/* C[b] = X[b] Y[b]^T for b < batch: n x n row-major FP32 matrices (DEVICE,
 * contiguous one after another, 16-byte aligned; n a positive multiple of
 * 128), on the tensor cores with the 3xTF32 split product: each FP32 value
 * x = x_hi + x_lo with x_hi = tf32(x), x_lo = tf32(x - x_hi) (round to
 * nearest, ties away), and X Y^T ~ X_lo Y_hi^T + X_hi Y_lo^T + X_hi Y_hi^T
 * accumulated in FP32 -- the product the mixed selected inversion uses
 * (Eq. sel_inv_cov on n_s x n_s blocks).  status (DEVICE [batch], may be
 * NULL) receives INLA_OK, or INLA_ERR_TIMEOUT where a bounded wait of the
 * kernel ran out (C is then not written).  Asynchronous on `stream` (a
 * cudaStream_t; NULL = legacy default stream).  Errors: INLA_ERR_ARG
 * (sizes, NULL or unaligned pointers), INLA_ERR_CUDA. */
int inla_gemm_tf32x3(int n, int batch, const float *X, const float *Y, float *C, int32_t *status, void *stream);

/* C[b] = X[b] Y[b]^T for b < batch: n x n row-major FP64 matrices (DEVICE,
 * contiguous one after another; n a positive multiple of 128) -- the product
 * the FP64 selected inversion uses (Eq. sel_inv_cov on n_s x n_s blocks),
 * computed on the BF16 tensor cores by error-free splitting (the Ozaki scheme):
 * each row of X and of Y is scaled by the power of two 2^e above its largest
 * magnitude and written as 8 integer digits of 7 bits (|digit| <= 64, exact in
 * BF16) plus a rounding error below 2^(e-56); the 36 digit products of
 * combined weight >= 2^-49 run on the tensor cores (tcgen05, kind::f16,
 * FP32 accumulation that is exact for the leading four weights), and their
 * sum is formed in 64-bit integer and FP64 arithmetic.  Error per entry
 * within K 2^(e_r + e_c - 50) + 2^-52 |C_rc| (e_r, e_c the row and column
 * exponents); integer matrices whose products fit 53 bits are multiplied
 * exactly.  work: DEVICE scratch of inla_gemm_f64_workspace_bytes(n, batch)
 * bytes, 256-byte aligned, owned by the caller.  status (DEVICE [batch], may
 * be NULL) receives INLA_OK, or INLA_ERR_TIMEOUT where a bounded wait ran out
 * (C is then incomplete).  Asynchronous on `stream` (a cudaStream_t; NULL =
 * legacy default stream).  Errors: INLA_ERR_ARG, INLA_ERR_CUDA. */
int inla_gemm_f64(int n, int batch, const double *X, const double *Y, double *C, void *work, size_t work_bytes,
                  int32_t *status, void *stream);
/* Scratch bytes inla_gemm_f64 needs (0 for invalid sizes). */
size_t inla_gemm_f64_workspace_bytes(int n, int batch);

/* Synthetic workload (host helper, not on the hot path; no counterpart in the
 * paper): fills *desc with a spatio-temporal SPDE x AR(1) model on an nx x nx
 * vertex grid of [0,1]^2 (n_s = nx^2; P1 lumped mass C and stiffness G), n_t
 * time steps, n_b covariates and m observations at uniform random times and
 * locations (A rows: the 3 barycentric weights of the containing triangle,
 * then the covariates), simulated at theta_true (HOST [4]; NULL: (1, -1, 0,
 * 1.5), Poisson (log 1e-3, -1, 0, 1.5)) from a Matern(nu = 1) field with an
 * AR(1) recursion; lik INLA_LIK_GAUSSIAN (y = A x + noise) or
 * INLA_LIK_POISSON (y ~ Pois(E exp(A x)), E ~ U(0.5, 2)).  Random numbers are
 * counter-based SplitMix64 streams keyed by seed, the same as the project's
 * Python generator.  Every pointer in *desc is a HOST pointer into *owner,
 * which the caller releases with inla_synth_free (after inla_model_create,
 * which copies the arrays).  Errors: INLA_ERR_ARG (sizes: n_t >= 1, nx >= 2,
 * 0 <= n_b <= 16, m >= 1; or a Poisson mean above 700), INLA_ERR_OOM. */
int inla_synth_build(int32_t n_t, int32_t nx, int32_t n_b, int64_t m, int32_t lik, uint64_t seed,
                     const double *theta_true, inla_model_desc *desc, void **owner);

/* The five benchmark workloads (cfg_id 1..5): n_t / grid / n_b / m / likelihood =
 * 8 / 8x8 / 2 / 2000 / Gaussian, 50 / 32x32 / 4 / 100 000 / Gaussian,
 * 100 / 45x45 / 6 / 400 000 / Gaussian, 200 / 50x50 / 6 / 1 000 000 / Gaussian,
 * 100 / 64x64 / 8 / 500 000 / Poisson, built by inla_synth_build at the default
 * theta_true.  Same ownership and errors as inla_synth_build. */
int inla_synth_grid_model(int32_t cfg_id, uint64_t seed, inla_model_desc *desc, void **owner);

/* Release the arrays of a synthetic workload.  NULL is allowed. */
void inla_synth_free(void *owner);

/* Free every device resource of the model built by inla_model_create (the
 * device copy of the Sec. 2.1 model, the workspace, captured graphs).
 * Synchronises the model's work first.  NULL is allowed. */
void inla_model_destroy(inla_model *model);

/* Message of the last non-OK return on this thread ("" if none); the string
 * is owned by the library and valid until the thread's next call.  No
 * counterpart in the paper (error reporting of the C ABI). */
const char *inla_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* INLA_GPU_H */
