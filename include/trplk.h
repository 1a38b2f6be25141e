/*
 * trplk.h -- C ABI of libtrplk, a GB300 (sm_103a) implementation of the hot
 * path of TRPL+K, the thick-restart preconditioned Lanczos method with +K
 * (locally optimal) restarting of Wu, Xue and Stathopoulos (arXiv 1711.10128).
 *
 * The library finds the p smallest eigenpairs of a sparse symmetric pencil
 * A v = lambda B v with B symmetric positive definite (Sec. 1, eq. (1)), with
 * B-orthonormal eigenvectors.  Everything runs on one GPU in hand-written CUDA
 * kernels; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Sparse matrices are CSR with int64 row pointers (n + 1 entries,
 *    rowptr[0] = 0), int32 column indices sorted within each row, and values
 *    of the dtype named by the matrix (TRPLK_F64 = double, TRPLK_F32 = float).
 *    A and B must be symmetric; the library does not check symmetry.
 *  - Dense blocks of n-vectors are column-major with a leading dimension
 *    `ld` >= n.  Inside the library ld is n rounded up to a multiple of 256 and
 *    rows n..ld-1 are kept at zero; the step-level entry points below take the
 *    caller's ld and require ld % 256 == 0 and the padding rows to be zero.
 *  - Ownership: the caller owns every buffer it passes and every output
 *    buffer; the library never frees caller memory.  Device pointers are used
 *    in place and must stay valid for the duration of the call.  The library
 *    owns its workspace until trplk_destroy.
 *  - Every call is synchronous with respect to the host: it returns after its
 *    GPU work on the handle's stream has finished (or failed).  One handle
 *    must not be used by two threads at once.
 *  - Errors: every entry point returns a trplk_status; on anything but
 *    TRPLK_OK (and TRPLK_NOT_CONVERGED, whose outputs are still filled) the
 *    outputs are unspecified and trplk_last_error() says why.  Invalid
 *    arguments are detected before the computation starts (TRPLK_EINVAL):
 *    sizes and parameters on the host, the structure of a solver matrix
 *    (row pointers in order and within nnz, column indices in [0, n)) by a
 *    validation kernel whose result is read before any other kernel uses
 *    the rows.
 */
#ifndef TRPLK_H_
#define TRPLK_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TRPLK_ABI_VERSION 2

typedef enum {
  TRPLK_OK = 0,
  TRPLK_EINVAL = 1,         /* bad argument or CSR structure                 */
  TRPLK_ENOMEM = 2,         /* device allocation failed                      */
  TRPLK_ECUDA = 3,          /* a CUDA call or kernel failed                  */
  TRPLK_NOT_CONVERGED = 4,  /* max_cycles reached; outputs hold the best pairs */
  TRPLK_BREAKDOWN = 5,      /* the Krylov space became invariant; no progress */
  TRPLK_NOT_SPD_B = 6,      /* x^T B x <= 0 was observed                     */
  TRPLK_NAN = 7,            /* a NaN or Inf reached a reduction              */
  TRPLK_ETIMEOUT = 8        /* a bounded device-side wait ran out            */
} trplk_status;

enum { TRPLK_F64 = 0, TRPLK_F32 = 1 };
enum { TRPLK_SMALLEST = 0 };
enum {
  TRPLK_PRECOND_NONE = 0,          /* M = I                                   */
  TRPLK_PRECOND_JACOBI = 1,        /* M = diag(A)^-1                          */
  TRPLK_PRECOND_FSAI = 2,          /* M = G^T G, classical FSAI on tril(A)    */
  TRPLK_PRECOND_FSAI_LEARNED = 3,  /* M = G^T G, G predicted by the MLP       */
  TRPLK_PRECOND_JACOBI_SHIFTED = 4,/* M_i = diag(A - rho_i B)^-1, rebuilt every
                                      cycle (Sec. 3: M may change per cycle to
                                      approximate (A - rho_i B)^-1); each
                                      diagonal entry floored at 1e-3 a_jj     */
  TRPLK_PRECOND_IC0 = 5            /* no-fill incomplete Cholesky L L^T ~ A
                                      (the paper's incomplete factorizations,
                                      Sec. 5.4-5.5), each triangular solve
                                      applied by 2 Jacobi sweeps:
                                      M = P^T P, P ~ L^-1 (SPD)               */
};
enum {
  TRPLK_LOCKING_SOFT = 0,  /* Algorithm 1: converged pairs stay in the basis   */
  TRPLK_LOCKING_HARD = 1   /* converged pairs are locked out of the search
                              (Sec. 3: hard locking can replace soft locking) */
};

/* Packed MLP parameters of the learned FSAI (FP32, this order):
 * W1[64][8], b1[64], W2[64][64], b2[64], W3[7][64], b3[7] -- 5191 floats. */
#define TRPLK_MLP_PARAMS 5191
enum {
  TRPLK_PRECISION_FP64 = 0,  /* FP64 storage and arithmetic throughout        */
  TRPLK_PRECISION_MIXED = 1  /* FP32 storage/SpMV, FP64-class coefficients,
                                then FP64 refinement to tol                   */
};

typedef struct trplk_handle trplk_handle;

/* A sparse symmetric matrix in CSR form.  `val` holds nnz values of `dtype`.
 * on_device = 1: all three arrays are device pointers; 0: host pointers. */
typedef struct {
  int64_t n, nnz;
  const int64_t* rowptr;
  const int32_t* col;
  const void* val;
  int dtype;
  int on_device;
} trplk_csr;

/* Solver parameters (Algorithm 1's inputs, Sec. 3, with the paper's names):
 *  p          number of wanted (smallest) eigenpairs, 1 <= p <= k
 *  q          maximum basis size (the paper's q = maxBasisSize), q <= 64
 *  k          thick-restart size p_hat >= p (minRestartSize, Sec. 5), k <= 32
 *  l          maximum number of +K (previous Ritz) vectors, 0 <= l,
 *             q >= k + max(l, 1) + 1
 *  tol        residual tolerance: ||A x - theta B x||_2 <= tol ||A||_1 ||x||_2
 *  max_cycles maximum number of restart cycles (the paper's maxIter)
 *  seed       SplitMix64 seed of the start block when X0 is NULL
 *  which      TRPLK_SMALLEST (the only supported value)
 *  precond    TRPLK_PRECOND_*
 *  precision  TRPLK_PRECISION_*
 *  outputs_on_device  1: evals/evecs/resid are device pointers; 0: host
 *  mlp_weights  host FP32 packed MLP parameters (TRPLK_MLP_PARAMS) for
 *             precond = TRPLK_PRECOND_FSAI_LEARNED; grid = (nx, ny, nz) of the
 *             7-point operator it is applied to (x fastest); mlp_bf16 = 1
 *             runs the MLP with BF16 weights/activations (FP32 accumulation)
 *  mixed_tol  FP32-phase tolerance of the mixed path (0 = max(tol, 3e-8));
 *             the FP32 phase also stops when the target's relative residual,
 *             once below 1e-6, has not halved over 30 cycles (at any level:
 *             120 cycles); FP64 cycles from its Ritz vectors then finish to
 *             tol -- each starting from the preconditioned residuals of all
 *             pairs within 100x of tol, basis min(q, k + p + 4 + l) -- and
 *             info.refine_cycles counts them
 *  locking    TRPLK_LOCKING_SOFT or _HARD.  Hard: after each Rayleigh-Ritz
 *             step the leading run of converged pairs of the active basis is
 *             locked; locked vectors keep their place at the front of the
 *             basis (they count against q and k), every new basis vector is
 *             B-orthogonalised against them, and T, the Rayleigh-Ritz step and
 *             the restart cover the active columns only; the target is always
 *             the smallest active pair; the solve ends when p pairs are
 *             locked.  The mixed path locks in its FP32 phase; its FP64
 *             refinement polishes all p pairs with soft locking.
 *  block      block size b of block TRPL+K (0 or 1: Algorithm 1; the paper
 *             leaves a block TRPL+K to future work, Sec. 5.5).  A cycle
 *             works on the targets t .. t+b-1: its first b Lanczos vectors
 *             are their preconditioned residuals, and every later one is
 *             M(A g - rho_i B g) from the vector g of the same sequence b
 *             columns back (rho_i = theta_{t+i}), B-orthogonalised by CGS2
 *             against the whole basis.  Needs b <= k, k + b + l <= q and
 *             soft locking; the FP64 refinement of the mixed path uses b = 1. */
typedef struct {
  int p, q, k, l;
  double tol;
  int max_cycles;
  uint64_t seed;
  int which;
  int precond;
  int precision;
  int outputs_on_device;
  const float* mlp_weights;
  int grid[3];
  int mlp_bf16;
  double mixed_tol;
  int locking;
  int block;
} trplk_params;

/* Counters and timings of one solve. */
typedef struct {
  int cycles;             /* restart cycles of the main phase                 */
  int refine_cycles;      /* FP64 refinement cycles (mixed path)              */
  int64_t mv_A, mv_B;     /* matvecs with A and B (B = I counts none)         */
  int64_t prec_apply;     /* preconditioner applications                     */
  int64_t mv_check;       /* matvecs of the final FP64 residual check         */
  double seconds;         /* wall time of the call                            */
  int nconv;              /* pairs meeting tol in the final check             */
  double normA;           /* ||A||_1                                          */
  double max_resid;       /* largest final relative residual                  */
  int64_t launches;       /* kernel launches of this call                     */
  int locked;             /* pairs locked (hard locking; 0 with soft locking) */
} trplk_info;

/* Create a handle bound to CUDA device `device`.  cuda_stream: a
 * cudaStream_t to run on, or NULL for a stream the library creates and owns.
 * Returns TRPLK_EINVAL for a bad device, TRPLK_ECUDA if CUDA fails. */
trplk_status trplk_create(trplk_handle** h, int device, void* cuda_stream);

/* Destroy a handle and free its workspace.  NULL is accepted. */
trplk_status trplk_destroy(trplk_handle* h);

/* Text of the last error on this handle ("" if none).  Owned by the handle. */
const char* trplk_last_error(const trplk_handle* h);

/* ABI version of the loaded library (TRPLK_ABI_VERSION). */
int trplk_abi_version(void);

/* Solve A v = lambda B v for the p smallest eigenpairs by TRPL+K
 * (Algorithm 1, Sec. 3; generalized pencil as sketched at the end of Sec. 3
 * and in Algorithm 2, Sec. 4).
 *  A, B     CSR (B == NULL: B = I); F64 values; same n.
 *  X0       n x k column-major (ld = n) start block in host or device memory
 *           (unified addressing tells them apart), or NULL to draw it with
 *           SplitMix64 from params->seed
 *  evals    [p] ascending Ritz values
 *  evecs    n x p column-major (ld = n), B-orthonormal Ritz vectors
 *  resid    [p] final FP64 relative residuals ||A x - theta B x|| / (||A||_1 ||x||)
 *  info     counters (may be NULL)
 * Returns TRPLK_OK when every pair meets tol, TRPLK_NOT_CONVERGED (outputs
 * filled with the best pairs) after max_cycles, or an error code. */
trplk_status trplk_solve(trplk_handle* h, const trplk_csr* A, const trplk_csr* B,
                         const trplk_params* params, const double* X0, double* evals,
                         double* evecs, double* resid, trplk_info* info);

/* ------------------------------------------------------------------------
 * Step-level entry points: the kernels of the solver, one row of its hot
 * path each, for parity tests and for callers that drive their own loop.
 * All pointers are device pointers; `dtype` selects F64 or F32 storage of
 * every dense array of the call (coefficients, T, theta, Y, norms are always
 * double).  ld % 256 == 0, padding rows zero.
 * ---------------------------------------------------------------------- */

/* y = A x (the matvec of eq. (UpdateT)).  A on device, val of `A->dtype`;
 * x, y of that dtype, length n.  y must not alias x.  The storage form is
 * chosen from A's structure on each call, as in trplk_solve: diagonals (DIA,
 * at most 64 of them, <= 30% zero padding), SELL-32 slices (<= 25% padding),
 * or the hybrid of SELL slices and warp/CTA-per-row for long rows.  A's CSR
 * structure is not validated here (trplk_solve validates it). */
trplk_status trplk_spmv(trplk_handle* h, const trplk_csr* A, const void* x, void* y);

/* The fused T-column / preconditioner / first-projection pass of one inner
 * step (eq. (UpdateT) and the Lanczos step after it):
 *   tcol[0:w] = U[:, 0:w]^T z,  v = dinv .* (z - rho * bg),  h1[0:w] = BU[:, 0:w]^T v
 * U, BU: n x w (ld); BU may equal U (B = I).  dinv, z, bg, v: vectors (ld);
 * dinv == NULL means M = I.  tcol, h1: double[w].  v may not alias z or bg. */
trplk_status trplk_inner_project(trplk_handle* h, int dtype, int64_t n, int64_t ld, int w,
                                 const void* U, const void* BU, const void* z, const void* bg,
                                 const void* dinv, double rho, void* v, double* tcol, double* h1);

/* One classical Gram-Schmidt pass in the B-inner product: h = BU[:, 0:w]^T v
 * (double[w]).  (Sec. 3: the basis G is kept B-orthonormal to [X, G].) */
trplk_status trplk_project(trplk_handle* h, int dtype, int64_t n, int64_t ld, int w,
                           const void* BU, const void* v, double* hout);

/* CGS2 with B-normalisation (Sec. 3, the inner method's orthogonalisation):
 *   v <- v - U h1, h2 = BU^T v, v <- v - U h2, Bv = B v, beta = sqrt(v^T B v)
 * given h1 (double[w], from trplk_project or trplk_inner_project).  On
 * return v holds the orthogonalised, NOT normalised vector, Bv its B-image
 * (B == NULL: Bv may be NULL and Bv = v is implied), beta[0] = ||v||_B and
 * beta[1] = the B-norm before orthogonalisation (by Pythagoras). */
trplk_status trplk_cgs2(trplk_handle* h, int dtype, int64_t n, int64_t ld, int w, const void* U,
                        const void* BU, const trplk_csr* B, const double* h1, void* v, void* Bv,
                        double* beta);

/* Rayleigh-Ritz on the w x w projection (Algorithm 1, 'compute eigenpairs of
 * T'): T double, column-major (ldT), only the upper triangle is read.
 * theta: double[w] ascending; Y: double w x w column-major (ld = w), each
 * column signed so its largest-magnitude entry (first such) is positive.
 * One CTA: cyclic Jacobi sweeps in FP32, two FP64 Newton-Schulz steps that
 * make the accumulated rotations orthogonal to FP64 rounding, then FP64
 * Jacobi sweeps on the rotated T until its off-diagonal norm is below
 * 3e-15 ||T||_F (FP64 accuracy).  w <= 64. */
trplk_status trplk_rayleigh_ritz(trplk_handle* h, int w, const double* T, int ldT, double* theta,
                                 double* Y);

/* Thick-restart rotation (Algorithm 1, restart): Xout = U[:, 0:w] Y[:, 0:k]
 * with Y double w x k column-major (ldY).  Xout: n x k (ld), must not alias U. */
trplk_status trplk_rotate(trplk_handle* h, int dtype, int64_t n, int64_t ld, int w, int k,
                          const void* U, const double* Y, int ldY, void* Xout);

/* The same rotation on the tensor cores, FP32 U and Xout (trplk_rotate takes
 * this path for FP32 data when w k >= 480; the solver for B = I): each
 * 128-row tile of U is multiplied by Y on tcgen05.mma with FP32 accumulation
 * in tensor memory, BF16 operands from an exact three-way split of every FP32
 * value (and of Y to FP32 accuracy), the six products of parts whose order
 * adds up to at most two summed in FP32, so the result keeps FP32 accuracy.
 * ld a multiple of 128 (any ld the library allocates), U 16-byte aligned,
 * w <= 64, k <= 32; EINVAL otherwise. */
trplk_status trplk_rotate_tc(trplk_handle* h, int64_t n, int64_t ld, int w, int k, const float* U,
                             const double* Y, int ldY, float* Xout);

/* Residual norms from stored images: rnorm[i] = ||AX_i - theta_i BX_i||_2 and
 * xnorm[i] = ||X_i||_2, i < k.  BX == NULL means B = I (BX = X). */
trplk_status trplk_residual_norms(trplk_handle* h, int dtype, int64_t n, int64_t ld, int k,
                                  const void* X, const void* AX, const void* BX,
                                  const double* theta, double* rnorm, double* xnorm);

/* The counter-based start block: X(i, c) = 2 u - 1, u the top 53 bits of one
 * SplitMix64 step on state seed XOR (c n + i), for i < n, c < k; rows n..ld-1
 * zero.  X: double, ld. */
trplk_status trplk_start_block(trplk_handle* h, int64_t n, int64_t ld, int k, uint64_t seed,
                               double* X);

/* Final FP64 check (the residual form of the stopping test): for i < p,
 *   resid[i] = ||A x_i - theta_i B x_i||_2 / (normA ||x_i||_2)
 * with fresh FP64 matvecs.  X double n x p (ld); A, B F64 on device
 * (B == NULL: identity).  resid: double[p] (device). */
trplk_status trplk_check_residuals(trplk_handle* h, const trplk_csr* A, const trplk_csr* B,
                                   int64_t ld, int p, const double* X, const double* theta,
                                   double normA, double* resid);

/* The projection of trplk_project, h = BU[:, 0:w]^T v, for callers that
 * cannot let the library allocate device memory.  The paper has no
 * counterpart: this is an interface for two kinds of caller -- processes that
 * have already planned all device memory through their own pool (a
 * cudaMalloc here would fail or break that plan) and latency-critical loops
 * that cannot afford the device synchronisation an allocation may cause.
 * Needs no handle; runs on `cuda_stream` (NULL = legacy default stream) of
 * the current device and returns after it finished.  Arguments as for
 * trplk_project (dtype, n, ld % 256 == 0 with zero padding rows, 1 <= w <= 64,
 * device pointers, hout double[w]).
 * Scratch: one fixed __device__ array inside the library holding the partial
 * sums of at most 256 CTAs (256 KiB + 256 bytes), kept by every GPU that
 * loads the library until the process exits; the call never uses more CTAs,
 * so any n fits, and w > 64 returns TRPLK_EINVAL.  The array is shared by all
 * calls and keeps the last call's contents (the call clears the words that
 * must start at zero); calls whose kernels overlap on the GPU race on it and
 * must be serialised by the caller.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture.  No cudaMalloc, cudaFree or other allocating call.
 * Module loading: when the CUDA runtime loads modules lazily (its default
 * since CUDA 12.2), the first call on each device is what loads this part of
 * the library, and that load places the array (256 KiB) and the kernels'
 * code in device memory.  Make the first call before the caller's own pool
 * reserves the device's free memory, or set CUDA_MODULE_LOADING=EAGER so the
 * load happens when the context is created; later calls load nothing. */
trplk_status trplk_project_noalloc(int dtype, int64_t n, int64_t ld, int w, const void* BU,
                                   const void* v, double* hout, void* cuda_stream);

/* Failure-injection hook for tests (not part of the method).  Every
 * mbarrier wait of the streaming passes on this handle gives up after
 * `polls` polls: polls = 0 makes each wait give up at once, so the next call
 * that runs such a pass returns TRPLK_ETIMEOUT; polls < 0 restores the
 * default (2^22 polls).  A pass that gives up waits until every bulk copy it
 * issued has landed before its CTAs exit, so the handle stays usable.
 * EINVAL for a NULL handle. */
trplk_status trplk_set_wait_limit(trplk_handle* h, int64_t polls);

/* ------------------------------------------------------------------------
 * Learned FSAI preconditioner (not in the paper: the data-parallel
 * preconditioner of this library; the paper allows any M approximating
 * (A - rho I)^-1, Sec. 3).  G is lower triangular on the pattern of A's lower
 * triangle (with the diagonal, columns ascending); M = G^T G.
 * ---------------------------------------------------------------------- */

/* Number of packed MLP parameters (TRPLK_MLP_PARAMS). */
int trplk_mlp_param_count(void);

/* Starting weights for training (host, no GPU): W1, W2 He-normal
 * (variance 2/fan_in, SplitMix64 counter stream of `seed` through
 * Box-Muller), W3 = 0, biases 0 except b3[c] = log(e - 1), so that
 * softplus(o_c) = 1 and G = D^-1/2: training starts from Jacobi.
 * weights: host float[TRPLK_MLP_PARAMS]; EINVAL if NULL. */
trplk_status trplk_fsai_mlp_init(float* weights, uint64_t seed);

/* G's values in the order of A's lower pattern.  kind 0: classical FSAI
 * (row i solves A[P_i, P_i] g = e_i, scaled so (G A G^T)_ii = 1; rows of at
 * most 16 lower entries); kind 1: learned (dims = nx, ny, nz of a 7-point
 * operator, weights = host packed MLP parameters, bf16 = precision); kind 2:
 * the IC(0) factor L (L L^T = A on the lower pattern; fixed-point sweeps of
 * the left-looking recurrence run to convergence on the device).
 * A: device CSR, F64.  g: device double[nnz_lower], or NULL to only return
 * *nnz_lower.  EINVAL for a non-symmetric pattern or long rows, NOT_SPD_B if
 * a principal block is not SPD. */
trplk_status trplk_fsai_values(trplk_handle* h, const trplk_csr* A, int kind, const int32_t* dims,
                               const float* weights, int bf16, double* g, int64_t* nnz_lower);

/* The IC(0) preconditioner of TRPLK_PRECOND_IC0 applied to x (device, FP64,
 * length n): y = P^T (P x) where P x takes 2 Jacobi sweeps
 * x_{t+1} = x_t + D^-1 (x - L x_t) from x_0 = D^-1 x on the factor L given by
 * its values l on A's lower pattern (from trplk_fsai_values with kind 2;
 * D = diag(L)), and P^T the same sweeps on L^T.  y must not alias x. */
trplk_status trplk_ic0_apply(trplk_handle* h, const trplk_csr* A, const double* l, const double* x,
                             double* y);

/* y = G^T (G x) with G given by its values g on A's lower pattern (device,
 * FP64, length n; y must not alias x). */
trplk_status trplk_fsai_apply(trplk_handle* h, const trplk_csr* A, const double* g, const double* x,
                              double* y);

/* Training loss of the learned FSAI on one operator and its solver vectors
 * V (device, FP64, n x nv column-major, ld = n): loss[0] = E + gamma K,
 * loss[1] = E = mean_v [(Mv)^T A (Mv) - 2 ||Gv||^2] / (v^T D^-1 v),
 * loss[2] = K = log(mean_i (G A G^T)_ii) - (2/n) sum_i log g_ii;
 * grad: host double[TRPLK_MLP_PARAMS], d loss[0] / d weights. */
trplk_status trplk_fsai_loss_grad(trplk_handle* h, const trplk_csr* A, const int32_t* dims,
                                  const float* weights, int bf16, const double* V, int nv,
                                  double gamma, double* loss, double* grad);

/* Training parameters of trplk_fsai_train. */
typedef struct {
  int iters;            /* Adam steps (operators visited in turn)             */
  double lr;            /* Adam learning rate                                  */
  int vectors;          /* residual vectors harvested per operator             */
  int harvest_cycles;   /* TRPL+K cycles (Jacobi, mixed path) per harvest      */
  int q, k, l;          /* basis shape of the harvest solves                   */
  uint64_t seed;        /* start-block seed of operator o is seed + o          */
  int bf16;             /* 1: BF16 weights/activations, FP32 accumulation      */
  double gamma;         /* weight of the Kaporin term                          */
} trplk_train_params;

/* Train the MLP: harvest solver vectors -- the residuals A x - theta x of
 * the Ritz vectors of capped Jacobi TRPL+K runs -- on each operator (device
 * CSR, F64, 7-point, dims 3 per operator), then `iters`
 * Adam steps on the loss of trplk_fsai_loss_grad.  weights: host FP32 packed
 * parameters, updated in place; losses: host double[iters] or NULL. */
trplk_status trplk_fsai_train(trplk_handle* h, const trplk_csr* ops, const int32_t* dims, int nops,
                              const trplk_train_params* tp, float* weights, double* losses);

/* ------------------------------------------------------------------------
 * Per-kernel profiling (measurement support, not part of the method).
 * ---------------------------------------------------------------------- */

/* enable = 1: from now on bracket every kernel launch of this handle with
 * CUDA events on its stream and record the launch's algorithmic bytes
 * (every operand read once, every output written once); enable = 0: stop.
 * Either call clears what was recorded. */
trplk_status trplk_profile(trplk_handle* h, int enable);

/* Totals since the last trplk_profile(h, 1) for one kernel family `kind`
 * (0 <= kind < 24; see trplk_profile_kind_name; kinds 12..23 are the same
 * families on FP64 data, named with an "_f64" suffix): number of launches,
 * summed event time in milliseconds and summed algorithmic bytes.  EINVAL
 * for a bad kind or NULL output. */
trplk_status trplk_profile_read(trplk_handle* h, int kind, int64_t* launches, double* milliseconds,
                                double* bytes);

/* Name of kernel family `kind`, or NULL if out of range.  Static storage. */
const char* trplk_profile_kind_name(int kind);

#ifdef __cplusplus
}
#endif
#endif /* TRPLK_H_ */
