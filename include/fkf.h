/*
 * fkf.h -- C-ABI of the GB300 fast random-walk Kalman filter.
 *
 * The method (Saibaba, Miller, Kitanidis, "Fast Kalman filter using
 * hierarchical matrices and a low-rank perturbative approach"):
 *   state model   s_k = s_{k-1} + w_k,  w_k ~ N(0, Gamma)       (Sec. 2.1, F_k = I)
 *   measurements  y_k = H_k s_k + v_k,  v_k ~ N(0, R_k)          (Sec. 2.1)
 *   posterior     Sigma_k|k = alpha_k Gamma - W_k D_k W_k^T,
 *                 W_k^T Gamma^-1 W_k = I, D_k diagonal           (Eq. sigmakk)
 * Gamma is a Matern covariance (Eq. maternfamily) held as a hierarchical
 * (H-) matrix (Sec. 2.2.1).  One filter step = predict (alpha += 1, Sec. 2.4)
 * + update with (y_k, H_k, R_k) through a data-space generalized
 * eigenproblem (Eqs. ghep, geneigendecomposition), a Gamma^-1-orthonormal
 * merge of the new directions (Alg. lowrankaddition) and the
 * Sherman-Morrison-Woodbury update of alpha_k, D_k, W_k (Sec. 2.4).
 *
 * Conventions (every entry point):
 *  - Every call returns fkf_status; FKF_OK = 0.  On error the objects are
 *    left as they were before the call (a filter step is transactional) and
 *    fkf_last_error(ctx) returns a one-line explanation.
 *  - Ownership: the library owns the opaque objects and all memory it
 *    allocates for them; the caller owns every pointer it passes and keeps it
 *    valid for the duration of the call.
 *  - Pointers named *_dev are device pointers on the context's device; all
 *    others are host pointers unless a flag says otherwise.  Device work is
 *    issued on the context's stream; host outputs are complete on return.
 *    Inside a call the library may also run work on two streams of its own
 *    (a high-priority one for the Cholesky's critical chain, a low-priority
 *    one for FP64 products that share the SMs with the tensor-core H-apply),
 *    ordered against the context's stream by events: seen from the context's
 *    stream, every call's work is complete where the call's own work is.
 *  - Point order: all N-indexed inputs/outputs use the caller's original
 *    point order (the library permutes internally to cluster order).
 *  - Dense N x n blocks of vectors are row-major: element (i, j) at
 *    ptr[i*ld + j], ld >= n.
 *  - Not thread-safe per object: calls on the same ctx must be serialised.
 */
#ifndef FKF_H
#define FKF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fkf_ctx fkf_ctx;
typedef struct fkf_hmat fkf_hmat;
typedef struct fkf_filter fkf_filter;

typedef enum {
  FKF_OK = 0,
  FKF_EINVAL = 1,   /* bad argument (size, pointer, parameter) */
  FKF_ENOMEM = 2,   /* device or host allocation failed */
  FKF_ENOTSPD = 3,  /* a matrix that must be SPD is not (innovation covariance, Gram) */
  FKF_ENOCONV = 4,  /* eigensolver did not converge */
  FKF_ETIMEOUT = 5, /* a bounded device wait gave up */
  FKF_ECUDA = 6,    /* CUDA runtime / library error */
  FKF_ESTATE = 7    /* object in a state that does not allow the call */
} fkf_status;

typedef enum {
  FKF_FP64 = 0, /* all N-scale storage and arithmetic in FP64 */
  FKF_FP32 = 1  /* N-scale storage/arithmetic in FP32; m x m and r x r work in FP64 */
} fkf_precision;

/* Matern kernel (Eq. maternfamily) with inverse scale 1/ell and variance
 * sigma2: C(r) = sigma2 * 2^(1-nu)/Gamma(nu) * (sqrt(2 nu) r/ell)^nu K_nu(...).
 * Supported: nu in {0.5, 1.5, 2.5} (exponential-times-polynomial closed forms). */
typedef struct {
  double nu;
  double ell;
  double sigma2;
} fkf_matern;

/* H-matrix construction (Sec. 2.2.1; the paper defers the construction to
 * the H-matrix literature).  leaf: maximum points per leaf cluster; eta:
 * admissibility min(diam t, diam s) <= eta * dist(t, s) on bounding boxes
 * (eta = 0 makes every block dense, i.e. Gamma exactly); aca_tol: relative
 * Frobenius tolerance of each low-rank block (Sec. 4.1.2); k_cap: maximum
 * block rank (a block that does not converge within k_cap is subdivided, or
 * stored dense when it cannot be). */
typedef struct {
  int32_t leaf;
  double eta;
  double aca_tol;
  int32_t k_cap;
} fkf_hparams;

/* Statistics of a built H-matrix (exact counts from the built trees). */
typedef struct {
  int64_t n;              /* points */
  int32_t dim;            /* 2 or 3 */
  int32_t precision;      /* fkf_precision */
  int64_t n_clusters;
  int64_t n_leaves;
  int64_t n_far;          /* admissible (low-rank) blocks, t <= s */
  int64_t n_near;         /* dense leaf blocks, t <= s */
  int64_t far_entries;    /* sum over far blocks of k_b (|t| + |s|) */
  int64_t near_entries;   /* sum over near blocks of |t||s| (stored once) */
  int64_t max_rank;
  double mean_rank;
  int64_t device_bytes;   /* device memory the operator holds now (values, schedules, streams, apply workspaces) */
  int64_t flops_per_col;  /* 2 * (entries of Gamma_H used per apply column) */
  int64_t bytes_per_col;  /* algorithmic bytes per apply column besides the operator (read X, write Y) */
  int64_t operator_bytes; /* algorithmic operator bytes read per apply panel */
  double build_seconds;
} fkf_hmat_info;

/* ---- context -------------------------------------------------------------
 * fkf_create: bind to CUDA device `device` and the CUDA stream `cuda_stream`
 * (a cudaStream_t, or NULL for a library-created stream).  The context
 * creates its internal streams on first use and destroys them in
 * fkf_destroy.  */
fkf_status fkf_create(fkf_ctx** out, int32_t device, void* cuda_stream);
void fkf_destroy(fkf_ctx* ctx);
const char* fkf_last_error(const fkf_ctx* ctx);
/* Kernels of this library launched by this context since creation. */
int64_t fkf_launch_count(const fkf_ctx* ctx);
/* cuSOLVER dense-routine calls (potrf, potrs) issued by this context. */
int64_t fkf_library_call_count(const fkf_ctx* ctx);

/* Symmetric eigendecomposition in FP64 on the device: the solver the filter
 * uses for the data-space generalized eigenproblem (Eq. ghep, solved as the
 * standard problem of R^-1/2 H Gamma H^T R^-1/2) and for the merge eigenproblem
 * of Alg. lowrankaddition (step 4).  Householder reduction to tridiagonal form,
 * divide and conquer on the tridiagonal, back-transformation of the wanted
 * eigenvectors.  A_dev: n x n symmetric (the mean of A and A^T is used),
 * row-major doubles, overwritten: rows 0..want-1 receive the eigenvectors of
 * the `want` largest eigenvalues, ascending (row q belongs to w[n - want + q]).
 * w_dev: all n eigenvalues, ascending.  Device workspace of about
 * 5 n^2 + n want doubles is allocated for the call.  Synchronises the
 * context's stream.  Errors: EINVAL, ENOMEM, ENOCONV (an iteration or a
 * bounded device wait did not finish), ECUDA. */
fkf_status fkf_eigh(fkf_ctx* ctx, int32_t n, double* A_dev, double* w_dev, int32_t want);

/* ---- H-matrix (Sec. 2.2.1) ----------------------------------------------
 * fkf_hmatrix_build: points (host, N x dim row-major, dim 2 or 3) -> Gamma_H.
 * Construction runs on the host CPU (cluster tree, block tree, ACA with
 * partial pivoting) and the result is laid out as flat arrays on the device.
 * Errors: EINVAL (N < 1, dim, nu unsupported, leaf < 1, aca_tol <= 0,
 * k_cap < 1), ENOMEM, ECUDA. */
fkf_status fkf_hmatrix_build(fkf_ctx* ctx, const double* points, int64_t n, int32_t dim, fkf_matern kernel,
                             fkf_hparams hp, fkf_precision prec, fkf_hmat** out);
fkf_status fkf_hmatrix_info(const fkf_hmat* h, fkf_hmat_info* info);
/* Y = Gamma_H X for an N x ncols block (row-major, original point order).
 * X_dev / Y_dev hold doubles for FKF_FP64 and floats for FKF_FP32; they
 * must not overlap.  ldx, ldy >= ncols.  Errors: EINVAL, ENOMEM, ECUDA. */
fkf_status fkf_hmatrix_apply(fkf_hmat* h, const void* X_dev, int64_t ldx, void* Y_dev, int64_t ldy, int64_t ncols);
/* Adjoint of Y = Gamma_H X for reverse-mode differentiation: gX = Gamma_H^T gY
 * = Gamma_H gY (every far block and near tile is stored once and serves both
 * (t, s) and (s, t), so the adjoint is the same sweep), and, with Y the forward
 * result, grad_sigma2 = <gY, Y> / sigma2, the derivative with respect to the
 * Matern variance (Gamma_H = sigma2 Gamma_1,H, so dY/dsigma2 = Y / sigma2).
 * gY_dev, Y_dev, gX_dev: device, N x ncols row-major, original point order,
 * the operator's element type; grad_sigma2 (host, nullable; Y_dev may be NULL
 * then).  Errors: as fkf_hmatrix_apply. */
fkf_status fkf_hmatrix_apply_adjoint(fkf_hmat* h, const void* gY_dev, int64_t ldg, const void* Y_dev, int64_t ldy,
                                     void* gX_dev, int64_t ldgx, int64_t ncols, double* grad_sigma2);
/* Same product with X and Y already in cluster order (no permutation). */
fkf_status fkf_hmatrix_apply_clustered(fkf_hmat* h, const void* X_dev, int64_t ldx, void* Y_dev, int64_t ldy,
                                       int64_t ncols);
/* Size of the fixed device scratch used by fkf_hmatrix_apply_clustered_noalloc:
 * one file-scope device array of this many bytes, which every GPU that loads
 * this library holds until the process exits. */
#define FKF_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* fkf_hmatrix_apply_clustered without any device memory allocation.  The
 * paper has no counterpart; this is a deployment variant of the same product.
 *
 * Who needs it: callers that must not call cudaMalloc/cudaFree while they
 * run -- for example a real-time assimilation loop whose latency budget
 * cannot absorb an allocator call (cudaMalloc can synchronise the device and
 * block), or a host process whose device memory is entirely owned by another
 * allocator (a framework's caching pool) so that extra driver allocations
 * would fail or fragment it.  The regular apply grows library-owned
 * workspaces with cudaMalloc on first use; this one never allocates.
 *
 * Same arguments and layout as fkf_hmatrix_apply_clustered (X, Y in cluster
 * order, row-major, precision's element type; the caller passes and owns
 * both), and the same product: an FP64 operator always runs the FP64 SIMT
 * tile engine here (the same result as engine 0 up to summation order; against
 * engine 3 about 1e-13 relative); an FP32 operator always runs the FP32 SIMT
 * tile engine here, whatever fkf_hmatrix_set_engine chose, so against the
 * default tensor-core apply it agrees to FP32 rounding (about 1e-5 relative).
 * The slot workspace and the split-reduction partials live in a
 * library-wide static device array of FKF_NOALLOC_SCRATCH_BYTES bytes; the
 * columns are processed in panels as wide as that array allows (at least one
 * column).  An operator that needs more than FKF_NOALLOC_SCRATCH_BYTES for a
 * single column is rejected with FKF_EINVAL and a message giving both sizes.
 * No cudaMalloc, cudaFree or allocating library routine is called.
 *
 * Set-up: the first call on each device looks up the device address of the
 * array (cudaGetSymbolAddress, with that device current) and caches it;
 * make that first call before any stream capture.
 * Sharing: all calls, from every context and stream of the process, share
 * the one array, which keeps the last call's contents; nothing in it has to
 * start at zero (each call writes every element it later reads).  Calls that
 * overlap on the GPU (different streams, or different host threads) race on
 * the array and give wrong results: serialise them.
 * The stream is synchronised before return, like fkf_hmatrix_apply_clustered.
 * Errors: EINVAL (arguments, operator too large for the scratch), ECUDA. */
fkf_status fkf_hmatrix_apply_clustered_noalloc(fkf_hmat* h, const void* X_dev, int64_t ldx, void* Y_dev,
                                               int64_t ldy, int64_t ncols);
/* Basis rotation product of the merge step (Alg. lowrankaddition, the
 * rotation W' = [W G] E of the new factor): C = A E[0:K, 0:ncols] for
 * row-major FP32 device arrays A (rows x K, leading dimension lda), E
 * (ke x ncols, lde; ke >= K) and C (rows x ncols, ldc), on the 5th-generation
 * tensor cores (tcgen05.mma kind::f16 with a two-term FP16 split of operands
 * scaled by powers of two per row of A and per column of E, FP32 accumulation
 * in TMEM) -- the kernel the FP32 filter step uses for W' and X'.  The
 * caller owns the three arrays; C must not overlap A or E.  The context keeps
 * a workspace (about 4 bytes per element of A and of E, grown on demand).  The context's stream is synchronised
 * before return.  Errors: EINVAL (negative sizes, K > ke, a leading
 * dimension below the row length, C overlapping A or E), ENOMEM, ECUDA,
 * ETIMEOUT (a tensor-core wait expired). */
fkf_status fkf_rotate_f32(fkf_ctx* ctx, const float* A_dev, int64_t lda, int64_t rows, int32_t K, const float* E_dev,
                          int64_t lde, int64_t ke, int32_t ncols, float* C_dev, int64_t ldc);
/* FP64 GEMM on the 5th-generation tensor cores: C = alpha op(A) op(B) +
 * beta C for row-major FP64 device matrices (op(A): M x K, op(B): K x N;
 * trans_a / trans_b nonzero: A is stored K x M, B is stored N x K; leading
 * dimensions in elements).  The FP64 products come from seven 7-bit integer
 * slices of every value (op(A) scaled per row, op(B) per column by powers of
 * two; Ozaki's error-free splitting) as FP16 MMAs whose FP32 sums stay exact
 * per block of 512 K, the engine-3 kernel of the H-apply; each element of C
 * carries an error below about 2^-48 of K max_k |op(A)_ik| max_k |op(B)_kj|
 * (49 bits of every value relative to its row or column scale).  This is
 * the product the library's eigensolver uses for its large GEMMs (the paper has
 * no counterpart: it serves the data-space GEP and merge eigensolves of
 * Eq. ghep and Alg. lowrankaddition).  The caller owns all three arrays; C
 * must not overlap A or B.  The context keeps a workspace of about 14 bytes
 * per element of A and of B (grown on demand).  Synchronises the context's
 * stream.  Errors: EINVAL (negative sizes, a leading dimension below its row
 * length, C overlapping A or B), ENOMEM, ECUDA, ETIMEOUT. */
fkf_status fkf_gemm_f64(fkf_ctx* ctx, int32_t trans_a, int32_t trans_b, int64_t M, int64_t N, int64_t K, double alpha,
                        const double* A_dev, int64_t lda, const double* B_dev, int64_t ldb, double beta, double* C_dev,
                        int64_t ldc);
/* Engine of the H-apply (the product with Gamma_H of Sec. 2.2.1).
 * FP32 operators: 2 (default) = 5th-generation tensor cores, tcgen05.mma
 * kind::f16 with a two-term FP16 split of power-of-two scaled operands
 * (hi*hi + hi*lo + lo*hi at twice the TF32 rate; scales per slot, point and X
 * column keep FP32-level accuracy); 1 = tensor cores, kind::tf32 with a
 * 3xTF32 split; both accumulate in FP32 in TMEM; 0 = the FP32 SIMT tile
 * engine.  FP64 operators: 0 (default) = the FP64 SIMT tile engine (exact
 * FP64 arithmetic); 3 = tensor cores with FP64 products assembled from seven
 * 7-bit integer slices of every value (Ozaki's error-free splitting; FP16
 * MMAs whose FP32 sums stay exact over blocks of 512 K, 64-bit integer
 * accumulation between blocks): every value keeps 49 bits relative to its row
 * or column scale and the slot products 49 bits relative to their L1 bound,
 * about 1e-13 of max |Y| on random vectors.  Selecting engine 1-3 rewrites
 * the operator's split (sliced) stream when it is not there yet (device
 * work, synchronous; engine 3 adds about 14 bytes per stored operator entry
 * and a sliced slot workspace of 14 bytes per slot and column).  Errors:
 * EINVAL (engine not 0-3, 1-2 for an FP64 operator, 3 for an FP32 one),
 * ENOMEM.  A tensor-core wait that expires makes the apply (or the filter
 * step) return FKF_ETIMEOUT. */
fkf_status fkf_hmatrix_set_engine(fkf_hmat* h, int32_t engine);
/* Poll limit of the tensor-core H-apply's pipeline waits (producer -> MMA ->
 * epilogue mbarrier hand-offs inside a CTA).  A wait that is not satisfied
 * within `polls` polls gives up: the CTA marks itself failed, every role
 * unwinds (the MMA thread waits for its issued MMAs, the producer for its
 * issued bulk copies, both with the full default limit, and TMEM is freed),
 * and the apply -- or the filter step that ran it -- returns FKF_ETIMEOUT with
 * the outputs undefined; the operator stays usable.  polls < 0 restores the
 * default 2^22; 0 makes every wait that is not already satisfied give up at
 * once (the way to exercise the time-out path).  Errors: EINVAL (polls >
 * 2^32 - 1). */
fkf_status fkf_hmatrix_set_wait_limit(fkf_hmat* h, int64_t polls);
/* Frees the device copy of an FP32 operator's factor and near-block values
 * (FP32, about 4 bytes per stored entry), keeping only the split stream that
 * the tensor-core engine in use (1 or 2) reads, for batches of filters that
 * must fit many operators in device memory.  Irreversible: afterwards the
 * SIMT engine, fkf_hmatrix_apply_clustered_noalloc and switching the engine
 * return FKF_ESTATE; applies, steps and densify on the current engine work
 * as before (the same results).  Errors: EINVAL (null), ESTATE (an FP64
 * operator, or engine 0). */
fkf_status fkf_hmatrix_release_values(fkf_hmat* h);
/* Current engine of the H-apply (see fkf_hmatrix_set_engine).  Errors: EINVAL (null). */
fkf_status fkf_hmatrix_get_engine(const fkf_hmat* h, int32_t* engine);
/* Autotuner of the tensor-core pipeline shape (engine 2): times the FP16
 * kernels with four K-chunks per stage and two stages (variant 0) and with two
 * chunks per stage and four stages (variant 1) on an apply of ncols columns
 * (deterministic test vectors, CUDA events on the context stream) and keeps
 * the faster for this operator; the results do not depend on the shape.
 * variant (nullable): the shape kept; ms (nullable): its time per apply (0
 * when the engine is not 2, where nothing is tuned).  Allocates two N x ncols
 * FP32 buffers for the duration of the call.  Errors: EINVAL, ENOMEM, ECUDA,
 * ETIMEOUT. */
fkf_status fkf_hmatrix_autotune(fkf_hmat* h, int64_t ncols, int32_t* variant, double* ms);
/* Permutation: perm[i] = original index of the i-th point in cluster order. */
fkf_status fkf_hmatrix_permutation(const fkf_hmat* h, int64_t* perm_host);
/* Dense copy of Gamma_H (host, N x N row-major, original order); N <= 8192. */
fkf_status fkf_hmatrix_densify(fkf_hmat* h, double* out_host);
void fkf_hmatrix_destroy(fkf_hmat* h);

/* ---- filter ---------------------------------------------------------------
 * fkf_filter_create: s_0 = s0 (host, N, original order; NULL = 0),
 * Sigma_0|0 = alpha0 * Gamma (Sec. 2.3 induction start; alpha0 >= 0),
 * trunc_tol: eigenvalues of the merged low-rank term below trunc_tol times the
 * largest are dropped (Alg. lowrankaddition step 4; relative reading);
 * m_max: largest measurement count per step; r_max: rank cap of W_k. */
fkf_status fkf_filter_create(fkf_hmat* h, const double* s0, double alpha0, double trunc_tol, int32_t m_max,
                             int32_t r_max, fkf_filter** out);
void fkf_filter_destroy(fkf_filter* f);

/* Flags for fkf_filter_step. */
#define FKF_STEP_INPUTS_ON_DEVICE 1 /* y, H_rowptr, H_col, H_val, R are device pointers */
#define FKF_STEP_SKIP_MEAN_SYNC 2   /* do not copy the NLL to the host (nll_out ignored) */
#define FKF_STEP_FULL_UPDATE 4      /* always take the merge path (GEP, orthonormalisation, merge,
                                       rotation), even when the step brings no information outside
                                       span(W) and the basis could be kept */
#define FKF_STEP_ALLOW_FIXED_H 8    /* fixed-H fast path (Alg. kalmanconstantH): if H_k and R_k are
                                       byte-identical to the previous step's and that step kept the
                                       basis, reuse its products G = Gamma_H H^T and H [W G] instead
                                       of recomputing them (no densify, no H-apply, no gathers) */
#define FKF_STEP_DENSE_HT 16        /* give the H-apply a dense H^T even where its FP16 split engine
                                       would take H^T straight from the sparse column index (same
                                       result, bit for bit; for checks and measurements) */

/* One predict + update (Sec. 2.4 / Alg. extkalman without linearisation):
 *   y (m), H_k as CSR m x N (rowptr int64 m+1, col int32 original point
 *   indices, val double), R_k = diag(R) (m doubles) or, if R == NULL,
 *   r_scalar * I (r_scalar > 0).  nll_out (host, nullable) receives the
 *   innovation negative log-likelihood 1/2 (nu^T S^-1 nu + log det S + m log 2 pi).
 * Errors: EINVAL (m < 1 or > m_max, bad CSR, nonpositive R), ENOTSPD (S not
 * SPD), ENOCONV, ECUDA; the filter state is unchanged on error. */
fkf_status fkf_filter_step(fkf_filter* f, const double* y, int32_t m, const int64_t* H_rowptr, const int32_t* H_col,
                           const double* H_val, const double* R, double r_scalar, int32_t flags, double* nll_out);

/* Extended Kalman filter step with the Box-Cox measurement map (Sec. 4.2,
 * Eq. nonlinear, Alg. extkalman).  The filtered field x is the Box-Cox
 * transform of the physical field s, x = a (s^(1/a) - 1), and the
 * measurements are y = H s(x) + v with s(x) = ((x + a)/a)^a.  The step
 * predicts (alpha += 1, mean unchanged), linearises at the predicted mean
 * x_pred: innovation nu = y - H s(x_pred), Jacobian
 * H_k = H diag(s'(x_pred)), s'(x) = ((x + a)/a)^(a - 1), and updates with H_k
 * through the general path (data-space GEP, Gamma^-1-orthonormal merge with
 * the filter's truncation, rotation) exactly as fkf_filter_step does for a
 * linear operator; the Jacobian changes every step, so the rank grows until
 * the truncation (trunc_tol, r_max) bounds it.  One linearisation per step.
 * Arguments as for fkf_filter_step (H is the linear operator H of h(x) =
 * H s(x), CSR over original point indices); boxcox_a > 0.  For a non-integer
 * a the map needs x > -a at every cell the rays cross (the power of a negative
 * base is undefined); a = 1 is the linear filter on y - H 1.  The fixed-H fast
 * path does not apply (FKF_STEP_ALLOW_FIXED_H is ignored).
 * Errors: as fkf_filter_step, and EINVAL for boxcox_a <= 0. */
fkf_status fkf_filter_step_ekf(fkf_filter* f, const double* y, int32_t m, const int64_t* H_rowptr,
                               const int32_t* H_col, const double* H_val, const double* R, double r_scalar,
                               double boxcox_a, int32_t flags, double* nll_out);

/* One filter's inputs and outputs for fkf_filter_step_batched. */
typedef struct {
  fkf_filter* filter;
  const double* y;
  int32_t m;
  const int64_t* H_rowptr;
  const int32_t* H_col;
  const double* H_val;
  const double* R;   /* m doubles or NULL (then r_scalar * I) */
  double r_scalar;
  double nll;        /* out: innovation NLL of this step */
  int32_t status;    /* out: fkf_status of this filter's step */
  int32_t merged;    /* out: 1 if this step's H-apply ran in the batch's merged launches */
} fkf_step_desc;

/* Step many independent filters at once (uneven N, m, kernels).  Every
 * filter must belong to a different context (each context owns one CUDA
 * stream); each step runs on its own host thread.  The steps' H-applies (S2)
 * of FP32 operators on the same tensor-core engine and device are merged:
 * one persistent launch per apply phase serves all of them (a step waits in
 * its H-apply until every step of the batch has reached its own or finished
 * without one); the rest of each step runs on its own context's stream, so
 * the GPU overlaps the filters' kernels.  Results are bitwise those of
 * stepping the filters one at a time.  Each filter's step is transactional
 * on its own; descs[i].status reports it.  Returns FKF_OK when every step
 * succeeded, else the status of the first failing entry.  flags as for
 * fkf_filter_step (applied to every entry).  Errors: EINVAL (nb < 1, a
 * context used twice), or the per-filter errors. */
fkf_status fkf_filter_step_batched(fkf_step_desc* descs, int32_t nb, int32_t flags);

/* Current state: s_hat (host, N, original order; nullable), alpha, rank r,
 * D (host, r doubles; nullable), W (device, N x r row-major in original
 * order, precision's element type; nullable, ldw >= r). */
fkf_status fkf_filter_get(fkf_filter* f, double* s_hat, double* alpha, int32_t* r, double* D, void* W_dev, int64_t ldw);
/* Bookkeeping of the filter (no device work). */
typedef struct {
  int64_t k;          /* steps taken */
  double alpha;       /* alpha_k */
  int32_t r;          /* rank of the low-rank term */
  int32_t last_path;  /* last step: 0 = new directions merged (GEP, orthonormalisation,
                         merge, rotation); 1 = no information outside span(W): basis kept,
                         weight updated in information form; 3 = as 1 with the previous
                         step's products reused (FKF_STEP_ALLOW_FIXED_H, unchanged H_k, R_k) */
  int32_t diagonal;   /* 1 if the weight is currently diagonal (the paper's D_k) */
  /* last merge step (last_path 0): */
  int32_t gep_rank;   /* data-space GEP eigenvalues kept (above gep_tol * max) */
  int32_t new_dirs;   /* new Gamma^-1-orthonormal directions merged (T eigenvalues above orth_tol) */
  int32_t t_eig;      /* 1 if T = I - P^T P was factored (pivoted Cholesky, pivots above
                         orth_tol); 0 if ||T||_F <= orth_tol showed nothing new */
  double t_lmax;      /* ||T||_F, a bound on every eigenvalue of T */
  int64_t chol_exact_retries; /* innovation factorisations redone with exact FP64 products after
                                 the tensor-core slice products left a non-positive pivot */
} fkf_filter_stats;
fkf_status fkf_filter_get_stats(const fkf_filter* f, fkf_filter_stats* out);

/* Posterior variance diag(Sigma_k|k) = alpha_k diag(Gamma) - diag(W D W^T)
 * (Sec. 3.1) into var_dev (device, N doubles, original order). */
fkf_status fkf_variance(fkf_filter* f, double* var_dev);
/* Conditional realizations (Sec. 3.3): out = s_hat + sqrt(alpha)(a - W Sig X^T a),
 * Sig = I - (I - D/alpha)^(1/2), for ns columns a = L_Gamma s_u supplied by the
 * caller (any L_Gamma with L_Gamma L_Gamma^T = Gamma).  a_dev, out_dev:
 * device, N x ns row-major doubles, original order. */
fkf_status fkf_conditional_realization(fkf_filter* f, const double* a_dev, int32_t ns, double* out_dev);
/* Relative entropy H[s_k|w_k] = 1/2 (N log alpha + sum_j log(1 - d_j/alpha)) and
 * A-optimality Trace(Sigma_k|k) = alpha Trace(Gamma) - sum_j d_j ||W_j||^2 (Sec. 3.1, 3.2). */
fkf_status fkf_uncertainty_scalars(fkf_filter* f, double* rel_entropy, double* trace_sigma);
/* Orthonormality drift max |X^T W - I| with X = Gamma^-1 W carried alongside W. */
fkf_status fkf_filter_orthonormality(fkf_filter* f, double* max_abs_err);
/* Re-establish W = Gamma_H X and W^T Gamma^-1 W = I (the invariant of
 * Eq. sigmakk, which FP32 storage of W and X lets drift): one H-apply of r
 * columns (the Gamma_sys W_k product), the Gram Q = X^T Gamma_H X,
 * W <- (Gamma_H X) Q^-1/2 and the weight re-diagonalised in that basis; the
 * covariance it represents is kept.  Works for any r <= r_max (a scratch of
 * N x r elements is allocated on first use when r exceeds m_max).
 * Errors: ENOTSPD (Q not positive definite), ENOMEM, ECUDA. */
fkf_status fkf_filter_refresh(fkf_filter* f);
/* Randomized generalized eigensolver for the merge steps (App. B, Alg.
 * randomizedghepuncert, with A = H_k^T R^-1 H_k and B = Gamma^-1): instead of
 * the exact data-space GEP (an m x m eigendecomposition), each merge step
 * keeps the k dominant modes of the sketch Ybar = A Omega of l = k + p
 * Gaussian columns: a Gamma-orthonormal basis of Ybar (rank-revealing), the
 * Rayleigh-Ritz matrix T = Q^T A Q (l x l) and its k largest eigenpairs.  All
 * of it runs in data space (O(m^2 l) instead of O(m^3)); the mean update and
 * the innovation covariance stay exact, the covariance update uses the k
 * modes (the approximation App. B bounds).  omega_dev: device, N x (k + p)
 * row-major FP64 in original point order, the caller's Gaussian draws (the
 * algorithm's input Omega), copied by the call (the caller may free it) and
 * used by every later merge step until changed.  k = 0 restores the exact
 * GEP (omega_dev ignored).  Errors: EINVAL (k < 0, p < 0, k + p > m_max,
 * omega_dev NULL with k > 0), ENOMEM, ECUDA. */
fkf_status fkf_filter_set_randomized_ghep(fkf_filter* f, int32_t k, int32_t p, const double* omega_dev);
/* Schedule fkf_filter_refresh after every `every`-th step (k % every == 0,
 * counted over the filter's lifetime) of fkf_filter_step / _ekf; 0 (the
 * default) never refreshes.  A scheduled refresh runs after the step has
 * committed; if it fails, the step's status is the refresh's error and the
 * state is the step's result.  Errors: EINVAL (every < 0). */
fkf_status fkf_filter_set_refresh(fkf_filter* f, int32_t every);
/* Checkpoint / restore of (k, alpha, r, s_hat, D, W, X) to a binary file. */
fkf_status fkf_filter_checkpoint(fkf_filter* f, const char* path);
fkf_status fkf_filter_restore(fkf_filter* f, const char* path);
/* Summed innovation NLL of K steps with a FIXED measurement operator H
 * (the setting of Alg. kalmanconstantH, Sec. 2.3) and its exact gradient by
 * reverse mode, with respect to the measurements y_k, the prior mean s_0, the
 * Matern variance sigma2 (Gamma = sigma2 * Gamma_1) and the noise variance rho
 * (R = rho I).  For a fixed H the NLL depends on the state only through
 * h_k = H s_k|k and T_k = H Sigma_k|k H^T, whose recursion closes in data
 * space (m x m) once A = H Gamma_H H^T is known (one H-apply); the adjoint
 * recursion runs backwards over k and recomputes the Cholesky factors of the
 * innovation covariances S_k from stored T_{k-1} instead of storing them.
 * The NLL equals the sum of fkf_filter_step's nll_out over the same steps
 * started from (s0, alpha0).
 *   y (host, K x m row-major), H as CSR (host; rowptr m+1, col original point
 *   indices), s0 (host, N original order, or NULL = 0), alpha0 >= 0, rho > 0.
 *   Outputs (host, each nullable): nll_out, grad_y (K x m), grad_s0 (N,
 *   original order), grad_sigma2, grad_rho.  Device memory: O(K m^2 + N m).
 * Errors: EINVAL (sizes, CSR, rho <= 0), ENOTSPD, ENOMEM, ECUDA. */
fkf_status fkf_nll_gradient(fkf_hmat* h, int32_t K, int32_t m, const double* y, const int64_t* H_rowptr,
                            const int32_t* H_col, const double* H_val, double rho, const double* s0, double alpha0,
                            double* nll_out, double* grad_y, double* grad_s0, double* grad_sigma2,
                            double* grad_rho);
/* Numerical thresholds of the step (all relative, in [0, 1)):
 *  gep_tol   -- data-space GEP modes with eigenvalue <= gep_tol * largest are
 *               dropped (they carry no information: null directions of H);
 *  orth_tol  -- candidate new directions whose Gamma^-1-norm squared outside
 *               span(W) is <= orth_tol are taken as already in span(W)
 *               (Alg. lowrankaddition step 2 made rank-revealing);
 *  trunc_tol -- merged low-rank eigenvalues <= trunc_tol * largest are
 *               truncated (Alg. lowrankaddition step 4).
 * Defaults: FP64 1e-13 / 1e-10 / (create's trunc_tol); FP32 1e-7 / 1e-3 / same. */
fkf_status fkf_filter_set_tolerances(fkf_filter* f, double gep_tol, double orth_tol, double trunc_tol);
/* Per-phase device time of the last step in milliseconds (CUDA events on the
 * context stream): [0] densify H^T, [1] H-apply, [2] gathers, innovation and
 * mean update, [3] data-space GEP, [4] orthonormalisation + merge, [5] rotation. */
fkf_status fkf_filter_phase_times(fkf_filter* f, double* ms6);

#ifdef __cplusplus
}
#endif
#endif /* FKF_H */
