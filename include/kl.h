/*
 * kl.h -- C ABI of the GB300 matrix-free isogeometric Karhunen-Loeve operator.
 *
 * The library computes the discrete Karhunen-Loeve eigenpairs of a covariance
 * kernel with the interpolation-based-quadrature (IBQ) Galerkin method of
 * Mika, Hughes, Schillinger, Wriggers, Hiemstra (arXiv 2011.13861):
 *
 *   standard-form operator (Sec. 4.4.1):
 *     A~' = L^{-1} M^T B~^{-1} J Gamma J B~^{-T} M L^{-T}
 *   with the univariate Kronecker factors Z_k = L_k L_k^T (Sec. 4.1, eq. cholesky),
 *   the Greville collocation matrices B~_k (Sec. 4.2, eq. interpolation_matrix),
 *   the mixed mass matrices M_k (Sec. 4.3, eq. univariate_mass_matrix2),
 *   J = diag(sqrt(det DF)) at the mapped Greville points and Gamma the kernel
 *   evaluated on the fly at every pair of mapped Greville points (Algorithm 1).
 *
 * Conventions shared by every entry point
 *   - Vectors are float64, column-major blocks of `nvec` columns with leading
 *     dimension `ld` (elements).  A trial-space vector has N = n_1 ... n_d entries,
 *     an interpolation-space vector Ntilde = n~_1 ... n~_d entries, both in the
 *     paper's vec ordering (Sec. 2.2): index i_1 + i_2 n_1 + i_3 n_1 n_2, i_1 fastest.
 *   - Pointers named *_dev are device pointers owned by the caller; the library
 *     never frees them.  *_host pointers are host memory owned by the caller.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls that take a stream are asynchronous on it unless stated otherwise.
 *   - Every call returns a kl_status.  On error nothing is aborted; a message is
 *     available from kl_last_error() (thread-local, valid until the next call
 *     on the same thread).  There is no CPU fallback: every compute step runs in
 *     the library's CUDA kernels.
 *   - A handle owns its device workspace (allocated in kl_create and grown on
 *     demand by kl_apply / kl_eigs, which then synchronise the stream once);
 *     kl_destroy frees it.  A handle may be used by one thread at a time.
 */
#ifndef KL_H_
#define KL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kl_handle_s* kl_handle;

typedef enum {
    KL_OK = 0,
    KL_ERR_INVALID_ARG = 1,   /* bad size, pointer, enum or unsupported combination */
    KL_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed */
    KL_ERR_OOM = 3,           /* device allocation failed */
    KL_ERR_NOT_CONVERGED = 4, /* kl_eigs reached maxiter before every residual met tol */
    KL_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
    KL_ERR_NUMERIC = 6        /* non-finite values or a failed factorisation */
} kl_status;

/* Geometry map F of the parametric cube [0,1]^d onto the physical domain (Sec. 2.4).
 * KL_GEOM_BOX is the affine map F(x^) = lo + (hi - lo) * x^ (det DF constant).
 * KL_GEOM_NURBS is a tensor-product NURBS map (Sec. 2.4): F = sum_I N_I w_I P_I / sum_I N_I w_I
 * over the control records P_I = (x, y, z), weight w_I; the knot vectors must be open on
 * [0, 1] (the parametric domain of the spline spaces), degree 1..15, weights positive, and
 * det DF > 0 at every Greville point (KL_ERR_INVALID_ARG otherwise).  The points and
 * J = sqrt(det DF) are evaluated once on the host in float64; knots and ctrl are host
 * pointers read during kl_create only. */
typedef enum { KL_GEOM_BOX = 0, KL_GEOM_NURBS = 1 } kl_geom_kind;

typedef struct {
    int dim;                /* d = 1, 2 or 3 */
    int kind;               /* kl_geom_kind */
    double lo[3];           /* BOX: corner, hi[k] > lo[k] */
    double hi[3];
    int deg[3];             /* NURBS: degree per parametric direction k < dim */
    int nctrl[3];           /* NURBS: control points per direction */
    const double* knots[3]; /* NURBS: nctrl[k] + deg[k] + 1 knots each */
    const double* ctrl;     /* NURBS: prod nctrl[k<dim] records (x, y, z, w), direction 1 fastest */
} kl_geometry;

/* Trial space B_h (degree deg[k], elems[k] uniform elements, C^{deg-1}, Sec. 2.3)
 * and interpolation space B~_h (interp_deg / interp_elems; 0 = same as trial;
 * Sec. 4.2).  Open uniform knot vectors on [0,1]: n_k = elems[k] + deg[k].
 *
 * Multipatch domains (Sec. 3.6): interfaces[k] lists n_interfaces[k] patch-interface
 * parameters in direction k (host array, read during kl_create; NULL / 0 = none).  Each must
 * be an interior breakpoint j/elems[k] of the trial mesh and of the interpolation mesh.  The
 * trial space is C^0 there (knot multiplicity deg[k]: n_k grows by deg[k] - 1 per interface)
 * and the interpolation space C^{-1} (multiplicity interp_deg[k] + 1: n~_k grows by
 * interp_deg[k]), as in the examples of Sec. 6.2 and 6.3; its two Greville abscissae at an
 * interface are evaluated from the left and from the right, and so is det DF of a NURBS map
 * with a C^0 knot there.  KL_ERR_INVALID_ARG for a value that is not such a breakpoint. */
typedef struct {
    int deg[3];
    int elems[3];
    int interp_deg[3];
    int interp_elems[3];
    int n_interfaces[3];
    const double* interfaces[3];
} kl_space;

/* Covariance kernels (Sec. 3.1 names the exponential and Gaussian kernels with
 * variance sigma^2 and a correlation length; formulas as read for this library):
 *   KL_K_EXP            sigma^2 exp(-|x - x'|_2 / L)
 *   KL_K_GAUSS          sigma^2 exp(-|x - x'|_2^2 / L^2)
 *   KL_K_EXP_SEPARABLE  sigma^2 exp(-sum_k |x_k - x'_k| / L)
 *   KL_K_POLY_TEST      sigma^2 prod_k (1 + x_k x'_k)^m, m = (int)L  (test kernel, 0 <= m <= 8) */
typedef enum { KL_K_EXP = 0, KL_K_GAUSS = 1, KL_K_EXP_SEPARABLE = 2, KL_K_POLY_TEST = 3 } kl_kernel_kind;

typedef struct {
    int kind;       /* kl_kernel_kind */
    double sigma;   /* > 0 */
    double L;       /* > 0 */
} kl_kernel;

/* Arithmetic of the on-the-fly kernel product (stage 5 of Algorithm 1).
 *   KL_P_FP64  kernel, distance and accumulation in float64 (matvec rel. error ~1e-14).
 *   KL_P_FP32  kernel and distance in float32 (MUFU ex2 / rsqrt), float32 partial sums
 *              over column chunks combined in float64; contractions in float32.
 *              Relative error ~1e-6.
 *   KL_P_DF64  kernel, distance and accumulation in double-float arithmetic (pairs of
 *              float32, ~48 significant bits) on the float32 pipe: float64-level results
 *              (matvec rel. error ~1e-14) at several times the float64 pipe's throughput on
 *              GB300; contractions in float64.
 *   KL_P_TC32  float32-accurate stage 5 on the tensor cores (tcgen05): float32 kernel values
 *              and u (scaled per vector by a power of two) cut into three exact 8-bit bfloat16
 *              slices each; the six slice products of the three leading levels are summed
 *              exactly in tensor memory and drained every 128 columns (relative error ~1e-6,
 *              like KL_P_FP32, at any size); contractions in float32.
 *              Calls that launch it synchronise the stream once to read a device status
 *              word (KL_ERR_TIMEOUT if a bounded wait inside the kernel gave up).
 *   KL_P_TC64  float64-class stage 5 on the tensor cores: double-float kernel values and the
 *              float64 u (scaled per vector by a power of two) cut into six exact 8-bit
 *              bfloat16 slices each; the 21 slice products of weight >= 2^-48 are summed in
 *              tensor memory, the four leading levels exactly (drained every 128 columns),
 *              so the product matches KL_P_DF64 (matvec rel. error ~1e-14); contractions in
 *              float64.  Same status-word synchronisation as KL_P_TC32.  No counterpart in
 *              the paper, which evaluates the kernel and sums in float64 (Sec. 4.4). */
typedef enum { KL_P_FP64 = 0, KL_P_FP32 = 1, KL_P_DF64 = 2, KL_P_TC32 = 3, KL_P_TC64 = 4 } kl_precision;

/* Build the univariate factors, the mapped Greville grid and J on the host in
 * float64 (Sec. 3.5, 4.1-4.3), upload them, and return a handle.
 * Fails with KL_ERR_INVALID_ARG for dim outside 1..3, deg < 1, elems < 1,
 * n~_k > 4096, Ntilde > 2^31-1, or a non-positive sigma / L / box extent.
 * Synchronous. */
kl_status kl_create(const kl_geometry* geom, const kl_space* space, const kl_kernel* kernel,
                    kl_handle* out);

/* N = trial-space dimension, Ntilde = number of interpolation (Greville) points. */
kl_status kl_size(kl_handle h, int64_t* N, int64_t* Ntilde);

/* Per-direction sizes: n[k] = trial functions, ntilde[k] = Greville points of direction k
 * (k = 0..2; directions beyond dim report 1).  Either pointer may be NULL. */
kl_status kl_dims(kl_handle h, int* n, int* ntilde);

/* y = A~' v for nvec columns (Algorithm 1, all nine stages), float64 arithmetic.
 * v_dev, y_dev: N x nvec, leading dimension ldv >= N; v and y must not overlap. */
kl_status kl_apply(kl_handle h, const double* v_dev, double* y_dev, int nvec, int64_t ldv,
                   void* stream);

/* Same as kl_apply with the stage-5 arithmetic chosen by `precision` (kl_precision). */
kl_status kl_apply_prec(kl_handle h, int precision, const double* v_dev, double* y_dev, int nvec,
                        int64_t ldv, void* stream);

/* Stages 1-4 of Algorithm 1: u = J . B~^{-T} M L^{-T} v   (N x nvec -> Ntilde x nvec). */
kl_status kl_forward(kl_handle h, const double* v_dev, int64_t ldv, double* u_dev, int64_t ldu,
                     int nvec, void* stream);

/* Stage 5 of Algorithm 1: z = Gamma u with Gamma(x_k, x_l) evaluated on the fly at the
 * mapped Greville points (never stored).  u, z: Ntilde x nvec. */
kl_status kl_covmv(kl_handle h, int precision, const double* u_dev, int64_t ldu, double* z_dev,
                   int64_t ldz, int nvec, void* stream);

/* kl_covmv without any device allocation (the paper has no counterpart: this is a deployment
 * convenience).  For callers that cannot call cudaMalloc when they apply the operator: programs
 * that take their whole device-memory budget at start-up and forbid allocation afterwards (for
 * example a component running inside a host application that owns the device memory), or
 * loops that cannot afford the implicit device synchronisation of cudaMalloc/cudaFree between
 * steps.  kl_covmv may grow the handle's workspace; this call instead keeps its split partial
 * sums in a fixed 32 MiB file-scope device array that every GPU loading the library holds until
 * exit.
 *   - precision must be KL_P_FP64; u, z as for kl_covmv; the handle itself comes from
 *     kl_create, which does allocate, so create it beforehand.
 *   - Ntilde x min(nvec, 16) must not exceed 4 Mi (4,194,304) doubles, else KL_ERR_INVALID_ARG
 *     with nothing launched.  Near that limit fewer column splits fit in the array (at 16
 *     vectors and 133k points only one), so the product runs on fewer CTAs and can be much
 *     slower than kl_covmv; the result is the same.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *     with that device current; make that first call before any stream capture.  The address
 *     is cached with the identity of its CUDA context and looked up again after the context
 *     was destroyed and recreated (cudaDeviceReset).
 *   - All calls share the array: launches that overlap on the GPU (other streams, other host
 *     threads) race on it, so order them.  No part of it needs clearing between calls.
 * Results agree with kl_covmv to rounding (the split count may differ). */
kl_status kl_covmv_noalloc(kl_handle h, int precision, const double* u_dev, int64_t ldu, double* z_dev,
                           int64_t ldz, int nvec, void* stream);

/* Stages 6-9 of Algorithm 1: y = L^{-1} M^T B~^{-1} (J . z)   (Ntilde x nvec -> N x nvec). */
kl_status kl_backward(kl_handle h, const double* z_dev, int64_t ldz, double* y_dev, int64_t ldy,
                      int nvec, void* stream);

/* Copy set-up data to host memory (synchronous), for inspection and checks:
 * C_host: n~_k x n_k row-major matrix C_k = B~_k^{-T} M_k L_k^{-T} of direction k (0-based);
 * X_host: Ntilde x 3 row-major mapped Greville points (unused coordinates 0);
 * J_host: Ntilde values sqrt(det DF).  Any pointer may be NULL. */
kl_status kl_get_factor(kl_handle h, int k, double* C_host);
kl_status kl_get_points(kl_handle h, double* X_host, double* J_host);

/* Eigensolver options for kl_eigs.
 *   method 0 (plain):  thick-restart block Lanczos, every operator application in
 *                      float64 (the paper's implicitly restarted Lanczos, Sec. 4.4.2).
 *   method 1 (mixed):  the same iteration with KL_P_FP32 operator applications until the
 *                      residual estimates reach `tol_low`, then block Lanczos from the
 *                      float32 Ritz vectors whose first block takes the float64 operator
 *                      (float64 polish; see polish_accurate).
 *   method 2 (LOBPCG): block LOBPCG (Knyazev's locally optimal block conjugate gradient,
 *                      no preconditioner) on a block of max(k, block) vectors (default
 *                      max(k, 32), at most 48): each step applies the operator to the residual
 *                      block only and runs Rayleigh-Ritz on span[X, P, R], kept orthonormal in
 *                      float64 with its products; every application in `precision`.
 *   method 3 (mixed LOBPCG): method 2 with `low_precision` applications until the residuals
 *                      reach `tol_low`, then `precision` from the float32 Ritz block.
 *           For methods 2 and 3, start_dev holds the whole block (N x max(k, block)), ncv,
 *           polish_block, polish_ncv and nstart are unused, and maxiter bounds the steps.
 *   block   b >= 1 (1 = classic single-vector Lanczos); ncv = basis size (0 = default
 *           max(2k+1, k + 3b) rounded up to a multiple of b; at most 160).
 *   start_dev: optional N x block start block (leading dimension N); NULL = seeded
 *           counter-based random block from `seed` (splitmix64, uniform(-1,1)). */
typedef struct {
    int method;
    int block;
    int ncv;
    int maxiter;            /* maximum restarts (0 = 1000) */
    uint64_t seed;
    const double* start_dev;
    double tol_low;         /* method 1: switch-over residual (0 = 1e-6 before a KL_P_TC64 polish, else 1e-5) */
    int verify;             /* final residuals ||A~'y - theta y|| / |theta|:
                             * 1 = from the operator products of the basis, carried through every
                             *     restart (A~'Y = (A~'V) S; no extra application);
                             * 2 = from a fresh application with the float64 kernel;
                             * 0 = the Lanczos estimates */
    int precision;          /* accurate-phase arithmetic: KL_P_FP64 (0, default), KL_P_DF64 or KL_P_TC64;
                             * method 0: every application, method 1: the polish.  Method 0 also
                             * takes KL_P_FP32 or KL_P_TC32 (float32-class results: tolerances of
                             * ~1e-5 and above, e.g. training data for the warm start) */
    int polish_block;       /* method 1: width of the polish block (k..48; 0 = k, or max(k, 32)
                             * for KL_P_TC64, whose launches cost the same up to 32 vectors) */
    int polish_ncv;         /* method 1: polish basis size (0 = 3 x polish_block, at most 160) */
    int low_precision;      /* method 1: first-phase arithmetic, KL_P_FP32 (0 = default) or KL_P_TC32 */
    int nstart;             /* columns of start_dev (0 = block; block..64, at most the basis size).
                             * With nstart > block the start columns are orthonormalised, the
                             * first-phase operator is applied to them once, and the iteration
                             * starts from their `block` leading Ritz vectors (Rayleigh-Ritz
                             * compression of a wider warm-start subspace). */
    int polish_accurate;    /* method 1: 0 (default) = only the polish's first application (on the
                             * float32 Ritz block) in `precision`, its correction blocks in
                             * `low_precision`: their coefficients in the refined Ritz vectors are
                             * of the size of the float32 residual, so the float32 operator's error
                             * reaches the residuals only as a product of the two (~1e-13 of
                             * ||A~'||); 1 = every polish application in `precision` */
} kl_eig_opts;

typedef struct {
    int applies;            /* operator applications counted per vector, all precisions */
    int applies_fp64;       /* of which float64 */
    int block_applies;      /* kl_apply launches (each on up to `block` or more vectors) */
    int restarts;
    int converged;          /* number of wanted pairs meeting tol */
    double resid[64];       /* ||A~'y_i - theta_i y_i||_2 / |theta_i|, float64 operator if verify */
    double ms_total;        /* wall time of the call */
    double ms_fp32_phase;   /* method 1: time spent before the float64 polish */
    /* stage-5 launches (kernel product + split combine) timed with CUDA events on `stream` */
    int stage5_calls_fp64, stage5_calls_fp32, stage5_calls_df64;
    double ms_stage5_fp64, ms_stage5_fp32, ms_stage5_df64;
    double pairs_fp64, pairs_fp32, pairs_df64;  /* kernel evaluations (Ntilde^2 per launch group) */
    int applies_df64;       /* operator applications counted per vector in KL_P_DF64 */
    int stage5_calls_tc64;  /* stage-5 launch groups, time and kernel evaluations in KL_P_TC64 */
    double ms_stage5_tc64, pairs_tc64;
    int applies_tc64;       /* operator applications counted per vector in KL_P_TC64 */
    int stage5_calls_tc32;  /* the same for KL_P_TC32 (the other float32-class counts above are KL_P_FP32's) */
    double ms_stage5_tc32, pairs_tc32;
    int applies_tc32;
} kl_eig_info;

/* ---- Many independent problems at once (no counterpart in the paper) ----------------
 * The instances (each its own kl_handle: size, degree, kernel, geometry may all differ) share
 * one persistent launch of stage 5 per step: items of 128 rows (256 in float32 up to 16
 * vectors: two rows a thread) x a column range of every instance are taken from a global
 * work counter, the kernel kind is read per item, and the
 * launch sequence is replayed from a captured CUDA graph; the column-range size is chosen by
 * timing candidates on the first batch.  Arithmetic as in KL_P_FP32 / KL_P_DF64. */

/* y_i = A~'_i v_i for i < count, on `stream`: stages 1-4 of every instance, one batched stage 5,
 * stages 6-9.  precision: KL_P_FP32 or KL_P_DF64.  v_dev, y_dev: count device pointers
 * (N_i x nvec[i], leading dimension ldv[i], or N_i when ldv is NULL), 0 <= nvec[i] <= 32.
 * A handle may appear once.  Asynchronous on `stream`. */
kl_status kl_apply_batched(kl_handle* handles, int count, int precision, const double* const* v_dev,
                           double* const* y_dev, const int* nvec, const int64_t* ldv, void* stream);

typedef struct {
    int rounds;             /* batched stage-5 launches */
    int cols_per_split;     /* column range chosen by the timing of the first representative batch */
    double ms_total;        /* wall time of the call */
    double ms_stage5;       /* batched stage-5 time on the GPU (CUDA events around every launch) */
    long long requests;     /* instance applications served by those launches */
} kl_batch_info;

/* kl_eigs for count instances with the same k, tol and options (opts may be NULL): one host
 * thread and one CUDA stream per instance run the solver of kl_eigs; every KL_P_FP32 and
 * KL_P_DF64 operator application of every instance joins a rendezvous, and the last instance
 * to arrive launches the batched stage 5 for all of them, or the first one whose batching
 * window has passed (200 microseconds; the environment variable KL_BATCH_WINDOW_US overrides
 * it, a negative value waits for every instance); instances that finish leave the
 * rendezvous.  Instance threads wait for the device asleep (blocking-sync events), not
 * spinning, so more instances than host cores is fine.
 * evals_host: count x k (row i = instance i); evecs_dev: NULL or count device
 * pointers (NULL entries allowed), leading dimensions ldv (NULL: N_i); infos, statuses,
 * binfo may be NULL.  Synchronous.  Returns the first non-KL_OK instance status (statuses[i]
 * holds every instance's), e.g. KL_ERR_NOT_CONVERGED. */
kl_status kl_eigs_batched(kl_handle* handles, int count, int k, double tol, const kl_eig_opts* opts,
                          double* evals_host, double* const* evecs_dev, const int64_t* ldv, kl_eig_info* infos,
                          kl_status* statuses, kl_batch_info* binfo);

/* ---- Learned warm start (no counterpart in the paper) ---------------------------------
 * A multilayer perceptron maps problem parameters to k standard-form vectors on a coarse
 * mesh; kl_prolong carries them exactly to a finer nested mesh, where they start kl_eigs
 * (opts.start_dev, block k).  Weights and layer inputs are bfloat16, sums float32, hidden
 * layers tanh, output linear; training minimises the mean of ||Y Y^T - V V^T||_F^2 / k over
 * samples (V: orthonormal target vectors, Y: predicted vectors; invariant under rotations and
 * sign flips of Y) with Adam (float32 master weights).  All device pointers are float32. */
typedef struct kl_mlp_s* kl_mlp;

/* n_in inputs, `depth` hidden layers of `width`, n_out outputs; weights uniform(+-sqrt(3/fan_in))
 * from a splitmix64 stream of `seed`, biases 0.  KL_ERR_INVALID_ARG for non-positive sizes. */
kl_status kl_mlp_create(int n_in, int width, int depth, int n_out, uint64_t seed, kl_mlp* out);
kl_status kl_mlp_num_params(kl_mlp m, int64_t* n);
/* Copy the float32 parameters (per layer: weights in x out row-major, then biases) to host
 * (direction 0) or from host (direction 1; the bfloat16 copy is refreshed).  Synchronous. */
kl_status kl_mlp_params(kl_mlp m, float* host, int direction);
/* out_dev (batch x n_out) = network(x_dev (batch x n_in)).  Asynchronous on `stream`. */
kl_status kl_mlp_forward(kl_mlp m, const float* x_dev, int batch, float* out_dev, void* stream);
/* One forward and backward pass (batch <= 65535, k <= 64): per-sample losses to loss_dev (batch floats) and, when
 * grad_host is not NULL, the gradient of the batch-mean loss (same layout as the parameters;
 * synchronous then).  tgt_dev: batch x (k n), vector j of sample s at s*k*n + j*n; k n = n_out. */
kl_status kl_mlp_loss_grad(kl_mlp m, const float* x_dev, const float* tgt_dev, int batch, int k, int n,
                           float* loss_dev, float* grad_host, void* stream);
/* `epochs` passes of Adam (learning rate lr) over `samples` rows in minibatches of `batch`
 * (seeded shuffle; an incomplete last batch is skipped); loss_host (epochs doubles, may be NULL)
 * receives each epoch's mean loss.  Synchronous on `stream`. */
kl_status kl_mlp_train(kl_mlp m, const float* x_dev, const float* tgt_dev, int samples, int k, int n, int epochs,
                       int batch, double lr, uint64_t seed, double* loss_host, void* stream);
void kl_mlp_destroy(kl_mlp m);

/* Exact prolongation of standard-form vectors (Sec. 4.1: v' = L^T v) from the trial space of
 * `coarse` to that of `fine`: every direction must have the same degree and a fine element
 * count that is a multiple of the coarse one (nested uniform knots), so each coarse spline is a
 * fine spline (knot insertion); per direction Q_k = L_f^T P_k L_c^{-T} with P_k from collocation
 * at the fine Greville points, applied as one contraction per direction.  v_dev: N_c x nvec,
 * y_dev: N_f x nvec, leading dimensions N_c and N_f; spaces with patch interfaces are rejected
 * (KL_ERR_INVALID_ARG).  Synchronous on `stream` (the factors
 * are uploaded per call and released once the contractions have run); it uses the apply
 * workspace of `fine`, so it must not overlap other calls on `fine`. */
kl_status kl_prolong(kl_handle coarse, kl_handle fine, const double* v_dev, double* y_dev, int nvec, void* stream);

/* The k (<= 64) largest eigenvalues of A~' (descending) to relative residual tol.
 * evals_host: k values (host).  evecs_dev: N x k orthonormal eigenvectors in standard
 * form (v'^T v' = I), leading dimension ldv (may be NULL).  info may be NULL.
 * Synchronous on `stream`.  Returns KL_ERR_NOT_CONVERGED (with the best pairs found
 * written out) when maxiter restarts did not converge every wanted pair. */
kl_status kl_eigs(kl_handle h, int k, double tol, const kl_eig_opts* opts, double* evals_host,
                  double* evecs_dev, int64_t ldv, kl_eig_info* info, void* stream);

/* v = L^{-T} v' : B-spline coefficients of the eigenfunctions, phi = sum v_i B_i / sqrt(det DF)
 * (Sec. 3.4, eq. basis; Sec. 4.1).  N x nvec blocks. */
kl_status kl_to_bspline(kl_handle h, const double* vprime_dev, double* v_dev, int nvec, int64_t ld,
                        void* stream);

/* Host only (no device use): the univariate set-up of one parametric direction exactly as
 * kl_create builds it, for inspection and for testing without a GPU.
 *   deg, elems               trial space (Sec. 2.3: open uniform knots, C^{deg-1})
 *   interp_deg, interp_elems interpolation space (Sec. 4.2); 0 = same as the trial space
 *   n_interfaces, interfaces patch interfaces in this direction, as in kl_space (Sec. 3.6)
 * On KL_OK, *n and *nt hold the numbers of trial and interpolation functions, and each
 * output that is not NULL is filled (caller-owned host arrays):
 *   greville  nt doubles: Greville abscissae of the interpolation space (Sec. 4.2)
 *   side      nt ints: -1 where the abscissa is evaluated as a left limit (C^{-1} knot), else 0
 *   L         n*n doubles, row-major: the lower Cholesky factor of Z_k = L_k L_k^T (Sec. 4.1)
 *   C         nt*n doubles, row-major: C_k = B~_k^{-T} M_k L_k^{-T} (Sec. 4.2-4.4), the folded
 *             factor the forward contraction applies
 * Call once with NULL outputs to learn n and nt.  Errors: KL_ERR_INVALID_ARG for the argument
 * rules of kl_create, a null n/nt, or a negative interface count (or a null array with a
 * positive one); KL_ERR_NUMERIC for an indefinite mass matrix or a singular collocation
 * matrix.  Outputs are not written on error. */
kl_status kl_direction_factors(int deg, int elems, int interp_deg, int interp_elems, int n_interfaces,
                               const double* interfaces, int* n, int* nt, double* greville, int* side,
                               double* L, double* C);

/* Host only (no device use): the mapped Greville grid and J exactly as kl_create builds them
 * (Sec. 2.4 map, Sec. 4.2 Greville abscissae, J = sqrt(det DF) as in Sec. 4.4.1; one-sided at
 * patch interfaces, Sec. 3.6), for inspection and for testing without a GPU.  geom and space
 * as for kl_create.  On KL_OK *Ntilde holds the number of points and each output that is not
 * NULL is filled (caller-owned host arrays): X Ntilde*3 doubles, point-major (x, y, z of point
 * i at 3i; unused coordinates 0), points in the paper's vec order (direction 1 fastest);
 * J Ntilde doubles.  Call once with NULL outputs to learn Ntilde.  Errors: those of kl_create
 * for the geometry and the space (KL_ERR_INVALID_ARG, KL_ERR_NUMERIC); outputs are not
 * written on error. */
kl_status kl_mapped_points(const kl_geometry* geom, const kl_space* space, int64_t* Ntilde, double* X, double* J);

/* Host only (no device use): the standard-form prolongation Q_k = L_f^T P_k L_c^{-T} of one
 * direction (the factor kl_prolong applies; P_k = B~_f^{-1} B_c(x_f) interpolates every coarse
 * B-spline at the fine Greville points, exact on nested spaces, Sec. 4.2 and 4.1), for
 * inspection and testing without a GPU.  deg: degree of both spaces; elems_coarse, elems_fine:
 * uniform element counts, elems_fine a multiple of elems_coarse.  On KL_OK *nc and *nf hold
 * the numbers of coarse and fine functions and, if Q is not NULL, Q (nf*nc doubles, row-major,
 * caller-owned) holds the factor.  Call once with Q = NULL to learn the sizes.  Errors:
 * KL_ERR_INVALID_ARG for the rules of kl_create, a null nc/nf, or meshes that are not nested. */
kl_status kl_prolongation_factor(int deg, int elems_coarse, int elems_fine, int* nc, int* nf, double* Q);

/* Workspace bound of the symmetric stage-5 kernels (float64, float32 and double-float blocks of
 * up to 8 vectors), which evaluate each kernel value once for the pairs (k, l) and (l, k)
 * (symmetry of Gamma, listed as future work in the paper's conclusions).  Their partial sums
 * take one slot of min(nvec, 8) x Ntilde doubles per 256-point tile (one launch, a slot count
 * growing with Ntilde) while that stays within `bytes` (default 512 MiB), and otherwise a
 * banded schedule of several launches with a fixed 20 slots, so that the workspace stays linear
 * in Ntilde (Sec. 5.4: matrix-free storage).  Both give the same sums up to rounding order.
 * Process-wide; affects workspaces sized after the call.  bytes < 0: KL_ERR_INVALID_ARG. */
kl_status kl_set_sym_slot_limit(int64_t bytes);

/* Schedule of the tensor-core float64-class stage 5 (KL_P_TC64), process-wide.  enable = 0
 * (default): all Ntilde^2 kernel values are evaluated, sums in a fixed order.  enable != 0: each
 * value once for both pairs (k, l) and (l, k) (symmetry of Gamma, future work in the paper's
 * conclusions): row blocks of 128 points meet only the column chunks of their own and later
 * column blocks, the same bfloat16 value slices feed the row-side product and, read
 * transposed, the column-side product, and the column sums are added with float64 atomics (their
 * order of addition, and the last bits of the result, may differ between runs).  It evaluates
 * half the values but measured slower on GB300 (the column side's drains and 168 extra MMAs per
 * chunk stall the pipeline), so it stays an option.  Problems with fewer than 256 points always
 * use the full evaluation.  Affects later calls. */
kl_status kl_set_tc_symmetric(int enable);

/* Measured throughput of the arithmetic pipes that bound the stage-5 kernels (no counterpart
 * in the paper: the denominators of the roofline fractions that the benchmark reports).
 * Runs four (five) short microbenchmarks on the current device (about 0.1 s in total, synchronous)
 * and writes, as operations per second for the whole GPU: rates_host[0] float64 FMA,
 * [1] float32 FMA, [2] MUFU ex2 (float32), [3] MUFU rsqrt (float32); with n >= 8 also the SM
 * clock in MHz that each of the four timed launches ran at ([4..7], from the SM cycle counter
 * and the global timer of one thread); with n >= 10 also the packed float32 pair FMA
 * (fma.rn.f32x2, counted as two FMAs) in [8] and its clock in [9].  n >= 4, else
 * KL_ERR_INVALID_ARG. */
kl_status kl_pipe_rates(double* rates_host, int n, void* stream);

/* Failure-detection self-test (no counterpart in the paper): one GPU thread waits on an
 * mbarrier that nothing completes, with the bounded-wait helper of the tensor-core kernels,
 * gives up after `seconds` (0 < seconds <= 2) and reports it.  Returns KL_ERR_TIMEOUT, the
 * status a stalled tensor-core pipeline returns; the context stays usable.  Synchronous. */
kl_status kl_wait_selftest(double seconds, void* stream);

/* Self-check of the packed-pair arithmetic of the tensor-core stage-5 producers (no counterpart
 * in the paper): n random pairs of column points (and a row point each) are evaluated through
 * the exponential, Gaussian and separable-exponential kernels in double-float (float64 class:
 * values, six slices, their sum) and in float32 (float32 class: values, three slices), once value
 * by value (the scalar code) and once two values per packed float32-pair instruction;
 * *mismatches receives the number of float words that differ (0: the two are bit-identical).  Synchronous on `stream`.  n >= 0, mismatches non-NULL, else
 * KL_ERR_INVALID_ARG. */
kl_status kl_df2_selftest(int64_t n, uint64_t seed, int64_t* mismatches, void* stream);

/* Number of CUDA kernels this library has launched since it was loaded (all handles, all
 * threads); for tracing and launch accounting. */
uint64_t kl_kernel_launches(void);

const char* kl_last_error(void);
void kl_destroy(kl_handle h);

#ifdef __cplusplus
}
#endif

#endif /* KL_H_ */
