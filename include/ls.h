/*
 * ls.h -- C ABI of the GB300-native dense Krylov solver library.
 *
 * The library solves dense linear systems A x = b on one GPU, the problem
 * statement of Oancea, Andrei and Dragoescu, "Improving the performance of
 * the linear systems solvers using CUDA" (arXiv:1511.07207), section
 * "Serial iterative and direct methods ...": Krylov methods whose iterate
 * update x(i) = x(i-1) + d(i) needs only inner products, saxpy operations and
 * one dense matrix-vector product per step.  The methods are the conjugate
 * gradient (CG paragraph of that section) and restarted GMRES(m) (its GMRES
 * pseudocode and restart paragraph).  The host flow of the paper's section
 * "Parallel implementation ... using CUDA" (allocate, copy in, run kernels,
 * copy out) is kept, but every iteration runs on the device: no host
 * synchronisation per iteration.
 *
 * Conventions, for every entry point:
 *   - Matrices are dense and row-major: element (i, j) of A is A[i*lda + j],
 *     lda >= n.  Blocks of right-hand sides B and solutions X are n x nrhs,
 *     column-major (column j starts at B + j*ldb), ldb >= n.
 *   - Pointers may be host or device memory; the library tells them apart
 *     with cudaPointerGetAttributes.  Host inputs are copied to the device
 *     inside the call, host outputs copied back before it returns.  Device
 *     inputs are read in place (A is never modified).
 *   - The caller owns every buffer it passes.  Solve calls are synchronous:
 *     they return after the result is in x (or X) and in the info struct.
 *   - Every function returns an int status: 0 = LS_OK, > 0 = a numerical
 *     outcome (the result and info are still filled in), < 0 = an error
 *     (outputs untouched unless stated).  No function aborts, exits or
 *     throws.
 *   - One context per host thread; a context is not thread-safe, except for
 *     the server calls, which are.
 */
#ifndef LS_H
#define LS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define LS_OK               0   /* converged: ||b - A x|| <= rtol ||b|| (true residual) */
#define LS_NOT_CONVERGED    1   /* iteration limit reached; x is the last iterate        */
#define LS_BREAKDOWN        2   /* p.Ap <= 0 in CG (A not SPD), or a zero Givens pivot   */
#define LS_ERR_ARG         -1   /* invalid argument (size, stride, null pointer, opts)  */
#define LS_ERR_NOMEM       -2   /* device allocation failed or workspace too small      */
#define LS_ERR_CUDA        -3   /* a CUDA runtime call failed                           */
#define LS_ERR_TIMEOUT     -4   /* a bounded on-device wait ran out                     */
#define LS_ERR_BUSY        -5   /* server: no capacity / queue full                      */
#define LS_ERR_NAN         -6   /* a NaN or Inf appeared in b or in the iteration        */
#define LS_ERR_UNSUPPORTED -7   /* the combination of options is not supported           */

/* ---- methods and precisions ------------------------------------------- */
#define LS_METHOD_CG     0
#define LS_METHOD_GMRES  1
#define LS_METHOD_BICGSTAB 2   /* ls_bicgstab_solve only (not in the batched engine) */
#define LS_METHOD_JACOBI   3   /* ls_jacobi_solve only (not in the batched engine)   */
#define LS_METHOD_GAUSS_SEIDEL 4   /* ls_gauss_seidel_solve only (not in the batched engine) */
#define LS_METHOD_BLOCK_CG 5       /* ls_block_cg_solve only (not in the batched engine)   */
#define LS_BLOCK_CG_MAX_S 16       /* right-hand sides of one ls_block_cg_solve, at most   */
#define LS_METHOD_BLOCK_GMRES 6    /* ls_block_gmres_solve only                              */
#define LS_BLOCK_GMRES_MAX_MS 256  /* restart x right-hand sides of ls_block_gmres_solve     */
#define LS_METHOD_LU 7             /* ls_lu_solve (the direct method)                        */
#define LS_METHOD_CHOLESKY 8       /* ls_chol_solve (the direct method for SPD A)            */

#define LS_F64      0   /* plain FP64 solve                                            */
#define LS_F64_PAIR 4   /* kernel-level entry points only: FP64 A given as the FP32 pair
                           made by ls_split_f64 (hi rows, then lo rows), FP64 x and y,
                           products in double-single arithmetic                         */
#define LS_BF16_IR  1   /* A stored in BF16, FP32 inner CG, FP64 outer refinement        */
#define LS_FP8_IR   2   /* A stored in FP8-e4m3 with one FP32 scale per row, as above    */
#define LS_F32_IR   3   /* A stored in FP32, as above                                    */

#define LS_REFINE_FCG 0 /* outer loop = flexible CG preconditioned by the inner solve    */
#define LS_REFINE_IR  1 /* outer loop = classic refinement x += inner(b - A x)           */

/* ---- options and results ---------------------------------------------- */
typedef struct {
    double rtol;        /* stop when ||b - A x||_2 <= rtol ||b||_2 (default 1e-10)      */
    int max_iter;       /* matrix-vector products of the method (default 10 n + 10);
                           for LS_*_IR: outer iterations (default 60)                   */
    int restart;        /* GMRES restart length m, 1..LS_MAX_RESTART (default 30)       */
    int precision;      /* LS_F64 (default), LS_BF16_IR, LS_FP8_IR, LS_F32_IR (CG only) */
    int refine;         /* LS_REFINE_FCG (default) or LS_REFINE_IR                      */
    int inner_iters;    /* inner FP32 CG iterations per outer step (default 25)         */
    double inner_rtol;  /* inner relative tolerance, 0 = run inner_iters (default 0)    */
    int x0_given;       /* 1: x holds the initial guess; 0: start from x = 0 (default)  */
    int reorth;         /* GMRES: 0 = one Gram-Schmidt pass with a second pass when the
                           norm drops below 0.7x (default), 1 = always two passes       */
    int f64_matvec;     /* LS_F64 solves: 0 = split A once into the FP32 pair
                           hi = fp32(A), lo = fp32(A - hi) (about 48 bits) and form
                           every A v in double-single arithmetic on the FP32 pipe
                           (default: GB300 runs FP32 at 64x its FP64 FMA rate, so the
                           product becomes HBM-bound; extra workspace 8 n^2 bytes);
                           1 = native FP64 FMA                                          */
    int deflate;        /* ls_block_cg_solve: 1 = keep the search directions orthonormal and
                           of full rank, dropping dependent ones (no breakdown on dependent,
                           zero or converged columns; default), 0 = O'Leary's form;
                           ls_block_gmres_solve: 1 = replace the dependent columns of a
                           cycle's starting block (default), 0 = they are a breakdown       */
    int fused;          /* ls_cg_solve / ls_gmres_solve with f64_matvec = 0: 1 = when the rows
                           of A fit in the shared memory of the GPU's co-resident CTAs (n up
                           to about 1800 on 152 SMs), run the whole solve as one kernel that
                           reads A from HBM once and keeps it on chip (default); 0 = always
                           the general path (one graph, a product kernel per step).  The
                           iteration, its stop tests and results are the same up to
                           rounding                                                        */
} ls_opts;

#define LS_MAX_RESTART 128

typedef struct {
    int status;          /* same as the return value                                     */
    int iters;           /* matrix-vector products of the method (inner ones for LS_*_IR)*/
    int outer_iters;     /* LS_*_IR outer steps; GMRES restart cycles                    */
    double rel_res;      /* last recursive (or Givens-estimated) relative residual       */
    double true_rel_res; /* ||b - A x|| / ||b|| recomputed in FP64 at exit               */
    double time_ms;      /* device time of the solve (CUDA events on the context stream) */
    double bytes_moved;  /* algorithmic bytes of A streamed (sum over all products; a
                            fused solve streams A once)                                  */
    long long launches;  /* kernels executed on the device for this call                 */
} ls_info;

/* Fill *o with the defaults listed above.  Returns LS_OK, or LS_ERR_ARG for NULL. */
int ls_opts_default(ls_opts *o);

/* ---- context ------------------------------------------------------------ */
typedef struct ls_ctx ls_ctx;

/*
 * Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The stream may be a
 * PyTorch stream handle.  Returns LS_ERR_CUDA if the device is unusable,
 * LS_ERR_UNSUPPORTED if it is not an sm_103 GPU.
 */
int ls_create(ls_ctx **ctx, int device, void *cuda_stream);

/* Release the context and everything it allocated.  NULL is accepted. */
int ls_destroy(ls_ctx *ctx);

/*
 * Device workspace, in bytes, that a solve of size n (nrhs right-hand sides)
 * with `method` and options `o` (NULL = defaults) needs.  It excludes A
 * itself when A is a device pointer and includes a staging copy of A
 * otherwise (`a_on_device` = 0).
 */
int ls_workspace_size(ls_ctx *ctx, int method, int n, int nrhs, const ls_opts *o,
                      int a_on_device, size_t *bytes);

/*
 * Hand the context a caller-allocated device buffer (e.g. from PyTorch's
 * caching allocator) of `bytes` bytes, 256-byte aligned.  The library then
 * allocates nothing for solves that fit in it and returns LS_ERR_NOMEM for
 * those that do not.  dev_ptr = NULL returns to library-managed memory.
 */
int ls_set_workspace(ls_ctx *ctx, void *dev_ptr, size_t bytes);

/* ---- single-system solvers ----------------------------------------------- */
/*
 * Conjugate gradient (paper: CG paragraph; Hestenes-Stiefel form) for SPD A.
 * n >= 0, lda >= n; A row-major n x n (FP64); b and x vectors of n FP64.
 * With opts->precision = LS_BF16_IR / LS_FP8_IR / LS_F32_IR, A is quantised
 * on the device (BF16 round-to-nearest-even from FP64; FP8-e4m3 with
 * s_i = fp32(max_j |a_ij| / 448), q_ij = e4m3_rn_satfinite(a_ij / s_i)),
 * an FP32 CG on the stored matrix is the inner solver, and the outer loop
 * (opts->refine) runs in FP64 on the FP64 A.  x receives the solution on
 * status >= 0.
 */
int ls_cg_solve(ls_ctx *ctx, int n, const double *A, int64_t lda, const double *b,
                double *x, const ls_opts *opts, ls_info *info);

/*
 * Restarted GMRES(m), m = opts->restart (paper: GMRES pseudocode, Arnoldi
 * with classical Gram-Schmidt, and the restart paragraph), for general
 * nonsingular A.  The Hessenberg least-squares problem is updated with
 * Givens rotations, so the residual norm of every iterate is known without
 * forming it; each restart recomputes the true FP64 residual.  Arguments as
 * for ls_cg_solve; opts->precision must be LS_F64.
 */
int ls_gmres_solve(ls_ctx *ctx, int n, const double *A, int64_t lda, const double *b,
                   double *x, const ls_opts *opts, ls_info *info);

/*
 * BiCGSTAB (paper: BiCGSTAB listing, van der Vorst's stabilised BiCG) for
 * general nonsingular A: two matrix-vector products, four inner products and
 * six vector updates per step, shadow residual r^ = r(0).  The steps the
 * listing leaves out are: omega = (t.s) / (t.t), r = s - omega t,
 * rho_{k+1} = r^.r, and the stop test ||r|| <= rtol ||b|| (confirmed on the
 * true residual; when it fails the iteration restarts from it with r^ = r).
 * When ||s|| already passes, x += alpha p ends the step.  info->iters counts
 * matrix-vector products (two per full step).  Breakdown (r^.v = 0,
 * rho = 0, t.t = 0 or omega = 0 before convergence) returns LS_BREAKDOWN with
 * the last iterate in x.  Arguments as for ls_cg_solve; opts->precision must
 * be LS_F64 (else LS_ERR_UNSUPPORTED).
 */
int ls_bicgstab_solve(ls_ctx *ctx, int n, const double *A, int64_t lda, const double *b,
                      double *x, const ls_opts *opts, ls_info *info);

/*
 * Jacobi iteration (paper: introduction, the classical stationary methods it
 * takes from the textbooks; one of the iterative methods the library
 * implements and times in its speed-up tables): x(k+1) = x(k) + D^-1 (b - A x(k)),
 * D the diagonal of A.  Each step is one matrix-vector product whose
 * epilogue forms the next iterate and ||b - A x(k)||; the iteration stops
 * when ||b - A x(k)|| <= rtol ||b|| (status LS_OK) or after max_iter products
 * (LS_NOT_CONVERGED; default max_iter 10 n + 10) and returns in x the last
 * iterate whose residual it measured, so info->rel_res is that iterate's
 * true relative residual.  info->iters counts products.  It converges when
 * the spectral radius of I - D^-1 A is below one (e.g. A strictly
 * diagonally dominant).  A zero diagonal entry returns LS_BREAKDOWN with x
 * unchanged (x0, or 0) and its residual; a residual that overflows returns
 * LS_ERR_NAN.  Arguments as for ls_cg_solve; opts->precision must be LS_F64
 * (else LS_ERR_UNSUPPORTED); opts->f64_matvec selects the product as there.
 */
int ls_jacobi_solve(ls_ctx *ctx, int n, const double *A, int64_t lda, const double *b,
                    double *x, const ls_opts *opts, ls_info *info);

/*
 * Forward Gauss-Seidel (paper: the same passage as Jacobi): each sweep
 * recomputes x_0, x_1, ... in turn from the newest values of the others,
 * i.e. (D + L) x(k+1) = b - U x(k) with D + L the lower triangle of A
 * including the diagonal and U the strict upper triangle.  The device runs
 * it as a correction: r = b - A x(k) (one product, whose norm is the stop
 * test), then the triangular solve (D + L) d = r over row blocks of 64 and
 * x(k+1) = x(k) + d, so a sweep streams A once and its lower half once more.
 * Stopping rule, the iterate returned, info->iters (residual evaluations),
 * the breakdown on a zero diagonal entry and the errors are those of
 * ls_jacobi_solve.  It converges for every SPD A and for strictly
 * diagonally dominant A.  Arguments as for ls_cg_solve; opts->precision must
 * be LS_F64; opts->f64_matvec selects the residual product's kernel (the
 * sweep always reads the FP32 pair of A, formed once per solve).  n is at
 * most 64 x 8 x (SMs - 1) (77,312 on GB300), else LS_ERR_UNSUPPORTED.
 */
int ls_gauss_seidel_solve(ls_ctx *ctx, int n, const double *A, int64_t lda, const double *b,
                          double *x, const ls_opts *opts, ls_info *info);

/*
 * Block CG (paper: the CG paragraph's method, for s right-hand sides at once
 * in block form) for SPD A: A X = B with B and X n x s, column-major (column
 * j at B + j*ldb, X + j*ldx), 1 <= s <= 16.  Every step forms the block
 * product Q = A P (A streamed once for all columns, as its FP32 pair unless
 * opts->f64_matvec).  Two forms:
 *   opts->deflate = 1 (default): the search directions are kept orthonormal
 *   and of full rank r <= s, dependent ones dropped: gamma = P^T Q (r x r),
 *   alpha = gamma^-1 (P^T R), X += P alpha, R -= Q alpha, beta =
 *   -gamma^-1 (Q^T R), P = orth(R + P beta), where orth keeps a column only
 *   if its part outside the span of the columns kept before it exceeds 1e-8
 *   of its norm (Gram matrix of the normalized columns, Cholesky with
 *   diagonal pivoting, then a second pass).  Dependent, zero or converged
 *   residual columns only lower r: no breakdown for SPD A.
 *   opts->deflate = 0: O'Leary's form, gamma = P^T Q, alpha = gamma^-1
 *   (R^T R), beta = (R^T R)^-1 (R^T R)', P = R + P beta; a rank-deficient
 *   residual block (linearly dependent or zero columns of B, or of R during
 *   the iteration) makes a Cholesky factor fail: LS_BREAKDOWN with the last
 *   iterate in X.
 * With a full-rank block both iterates minimise the A-norm error over the
 * block Krylov space, so they need at most as many steps as single-vector CG
 * on any column.  Stops when every column has ||R_j|| <= rtol ||B_j||,
 * confirmed on the true residual (a failed confirmation restarts from it).
 * info->iters counts block steps (one block product each); info->rel_res and
 * true_rel_res are the largest true relative residual over the columns.  The
 * deflating form returns LS_BREAKDOWN only when gamma is not positive
 * definite (A not SPD).  X0 is read when opts->x0_given.  opts->precision
 * must be LS_F64 (else LS_ERR_UNSUPPORTED); s outside 1..16 or ld < n is
 * LS_ERR_ARG.  Host or device pointers, as for ls_cg_solve.
 */
int ls_block_cg_solve(ls_ctx *ctx, int n, int s, const double *A, int64_t lda, const double *B,
                      int64_t ldb, double *X, int64_t ldx, const ls_opts *opts, ls_info *info);

/*
 * Restarted block GMRES(m), m = opts->restart block steps per cycle (paper:
 * the GMRES pseudocode and restart paragraph, with a block Arnoldi process
 * over s right-hand sides at once) for general nonsingular A: A X = B with B
 * and X n x s, column-major (column j at B + j*ldb, X + j*ldx), 1 <= s <= 16,
 * m * s <= 256.  Each block step forms W = A V_j (one pass over the FP32 pair
 * of A for all s columns), orthogonalises it against the basis by two
 * passes of block classical Gram-Schmidt and factors it by CholQR2 into
 * V_{j+1} H_{j+1,j}; the band Hessenberg matrix is reduced by Givens
 * rotations, so every right-hand side's residual is known without forming
 * it; a cycle ends when all of them pass rtol ||B_c||, after m steps, or on a
 * block that lost rank; then X += V Y.  Each cycle starts from the true
 * residual and the solve stops when every column's true residual passes.
 * info->iters counts block steps, info->outer_iters cycles, rel_res the
 * largest true relative residual over the columns.  A cycle's starting
 * block R = B - A X may be rank-deficient (zero, repeated or dependent
 * columns: a column whose part orthogonal to the columns before it is at
 * most 1e-6 of its norm).  With opts->deflate (the default) each such
 * column is replaced by a fixed pseudo-random vector (entry i of column c:
 * 2u - 1, u the top 53 bits of output c 2^32 + i of SplitMix64 seeded with
 * 0, over 2^53), the block is orthonormalised into V_1 and S = V_1^T R, so
 * every right-hand side, the dependent ones included, is solved; with
 * opts->deflate = 0 such a block returns LS_BREAKDOWN.  A zero rotation
 * pivot returns LS_BREAKDOWN with the last iterate in X.  opts->precision
 * must be LS_F64 and opts->f64_matvec 0 (else LS_ERR_UNSUPPORTED); s or m
 * outside the limits or ld < n is LS_ERR_ARG.  Host or device pointers.
 */
int ls_block_gmres_solve(ls_ctx *ctx, int n, int s, const double *A, int64_t lda, const double *B,
                         int64_t ldb, double *X, int64_t ldx, const ls_opts *opts, ls_info *info);

/*
 * The direct method (paper: the right-looking LU with partial pivoting of
 * the direct-methods section): at step k the row v >= k with the largest
 * |a_vk| (the first one on ties) is swapped with row k, the sub-column is
 * divided by the pivot and the rank-1 update is subtracted from the trailing
 * block; b is carried along as an extra column, so L y = P b is done during
 * the elimination; then U x = y.  FP64, run by panels of 32 columns (the
 * panel's pivot steps, its row swaps on the other columns, the pivot rows
 * right of it, the trailing update), which only regroups the elimination's
 * operations: every element of L, U and y is bit for bit what the plain
 * elimination gives in FP64 (IEEE division, multiply and subtract not
 * fused, the updates of each element in step order).  After the solve the true
 * residual ||b - A x|| is formed (info->rel_res, true_rel_res; info->iters =
 * 0).  A zero pivot returns LS_BREAKDOWN with x unchanged; a residual that
 * is not finite returns LS_ERR_NAN.  A row-major n x n (host or device), b
 * and x n vectors; opts may be NULL; opts->precision must be LS_F64.  The
 * elimination is n^3 / 3 updates of two FP64 instructions each, bound by the
 * FP64 pipe; the trailing block crosses HBM once per panel.
 */
int ls_lu_solve(ls_ctx *ctx, int n, const double *A, int64_t lda, const double *b, double *x,
                const ls_opts *opts, ls_info *info);

/*
 * The factorization of ls_lu_solve alone: LU (n x n, row-major, leading
 * dimension ldlu >= n) receives the unit lower factor L below the diagonal
 * and U on and above it, rows in pivoted order; ipiv[k] the row swapped with
 * row k at step k; y = L^-1 P b.  Outputs may be host or device memory.
 * Returns LS_BREAKDOWN on a zero pivot at step k; then only the columns and
 * ipiv entries of the panels of 32 steps completed before k are final (the
 * rest of LU, ipiv and y is partial work).  LS_ERR_ARG on bad sizes or NULL
 * pointers.
 */
int ls_lu_factor(ls_ctx *ctx, int n, const double *A, int64_t lda, const double *b, double *LU,
                 int64_t ldlu, int *ipiv, double *y);

/*
 * Self-test of the bounded on-device waits (no paper passage: the library's
 * own failure detection).  which = 0: a kernel waits on an mbarrier that
 * nothing completes; which = 1: one CTA of a two-CTA kernel waits at a grid
 * barrier (a private one) that the other CTA never reaches.  Each wait gives
 * up after the library's limit (2 s), records the timeout and returns.
 * Returns LS_ERR_TIMEOUT when that happened, which is the expected result;
 * the context stays usable.  LS_ERR_ARG for a NULL context or another
 * `which`.  Synchronous on the context's stream.
 */
int ls_selftest_waits(ls_ctx *ctx, int which);

/* ---- batched solver -------------------------------------------------------- */
typedef struct {
    int method;          /* LS_METHOD_CG (SPD A) or LS_METHOD_GMRES                     */
    int n;               /* 1 .. LS_BATCH_MAX_N                                          */
    int nrhs;            /* 1 .. LS_BATCH_MAX_RHS                                        */
    const double *A;     /* row-major n x n, leading dimension lda (host or device)      */
    int64_t lda;
    const double *B;     /* n x nrhs column-major, leading dimension ldb                 */
    int64_t ldb;
    double *X;           /* n x nrhs column-major, leading dimension ldx (output)        */
    int64_t ldx;
    ls_opts opts;        /* rtol, max_iter, restart used per system; precision ignored  */
} ls_system;

#define LS_BATCH_MAX_N   8192
#define LS_BATCH_MAX_RHS 32

/*
 * Solve `count` independent systems in one persistent device launch.  Every
 * right-hand side column is solved on its own (column-independent CG or
 * GMRES(m) sharing each matrix product A*P across the columns of a system),
 * with FP32 products on the tensor cores inside an FP64 refinement loop on
 * the FP64 residual B - A X.  infos[i] receives the outcome of system i
 * (worst column).  Returns the worst status over the systems.
 */
int ls_batch_solve(ls_ctx *ctx, int count, const ls_system *sys, ls_info *infos);

/* ---- server (continuous batching) ----------------------------------------- */
typedef struct {
    size_t hbm_budget_bytes;   /* device memory the server may hold for requests      */
    int max_slots;             /* requests resident on the device at once             */
    int step_iters;            /* iterations each resident request advances per step  */
    int queue_capacity;        /* pending requests before submit returns LS_ERR_BUSY  */
    int merge_rhs;             /* 1: queued requests that share their matrix (the same
                                  device A, lda, n, method and options) are admitted
                                  together as right-hand-side columns of one slot (at
                                  most 32), so A is read once per step for all of them.
                                  Each column still runs its own iteration, but the
                                  shared reductions round in an order that depends on
                                  the slot's width, so a merged result matches a solo
                                  solve within the tolerance, not bit for bit; the
                                  slot's status (NaN, iteration limit) is shared.
                                  0: one request per slot                              */
} ls_server_cfg;

typedef struct ls_server ls_server;

/*
 * Start a server on the context's device with its own scheduler thread.
 * Requests are admitted when their device bytes fit in the budget and a slot
 * is free; every scheduler step advances all resident requests on the
 * device; finished requests retire and free their memory.
 */
int ls_server_start(ls_ctx *ctx, const ls_server_cfg *cfg, ls_server **srv);

/*
 * Queue one system (n <= LS_BATCH_MAX_N, nrhs <= LS_BATCH_MAX_RHS).  B is
 * copied before the call returns.  A in host memory is copied too; A in
 * device memory is read in place, so that a set of matrices kept resident on
 * the device can be served without copies -- it must stay valid and unchanged
 * until the ticket is done.  X (host or device) must stay valid until
 * ls_server_poll reports the ticket done.  Thread-safe.  LS_ERR_BUSY when the
 * queue is full or the server is stopping, LS_ERR_NOMEM when the request
 * alone exceeds the budget.
 */
int ls_server_submit(ls_server *srv, const ls_system *req, uint64_t *ticket);

/*
 * Non-blocking: *done = 1 once X has been written and *info filled in
 * (info->time_ms is the latency from submit to completion).  Thread-safe.
 * The call that reports done = 1 also forgets the ticket: a later poll of it,
 * like a poll of a ticket never issued, returns LS_ERR_ARG.
 */
int ls_server_poll(ls_server *srv, uint64_t ticket, int *done, ls_info *info);

/* Stop the scheduler: resident requests finish or are cancelled
 * (status LS_NOT_CONVERGED), pending ones are cancelled.  Never hangs. */
int ls_server_stop(ls_server *srv);

/* ---- kernel-level entry points (used by the tests and the benchmark) ------ */
/*
 * y = A x for a row-major rows x cols matrix stored as `dtype`
 * (LS_F64: double A, double x and y; LS_BF16_IR: uint16 BF16 codes;
 * LS_FP8_IR: uint8 e4m3 codes with FP32 row scales `scale`, y_i = s_i (Q x)_i;
 * LS_F32_IR: float A; LS_F64_PAIR: the FP32 pair of ls_split_f64 with lda = its
 * ldp, double x and y).  For the low-precision formats x and y are FP32.
 * All pointers are device pointers.
 */
int ls_gemv(ls_ctx *ctx, int dtype, int rows, int cols, const void *A, int64_t lda,
            const float *scale, const void *x, void *y);

/*
 * Split a row-major FP64 matrix (device) into the FP32 pair used by the FP64
 * solvers' products: pair[i * ldp + j] = hi_ij = fp32(a_ij) (round to nearest
 * even), pair[(rows + i) * ldp + j] = lo_ij = fp32(a_ij - hi_ij); hi + lo equals
 * a_ij to within 2^-48 |a_ij|.  ldp >= cols and a multiple of 4 (16-byte rows);
 * `pair` holds 2 rows ldp floats.  Device pointers; LS_ERR_ARG on bad sizes.
 */
int ls_split_f64(ls_ctx *ctx, int rows, int cols, const double *A, int64_t lda, float *pair, int64_t ldp);

/*
 * Quantise a row-major FP64 matrix on the device: LS_BF16_IR -> uint16 codes,
 * LS_FP8_IR -> uint8 codes plus FP32 row scales, LS_F32_IR -> float.
 * Roundings as described for ls_cg_solve.  Device pointers.
 */
int ls_quantize(ls_ctx *ctx, int dtype, int rows, int cols, const double *A, int64_t lda,
                void *Q, int64_t ldq, float *scale);

/*
 * Benchmark helper: launch the y = A x kernel of ls_gemv `reps` times back to
 * back on the context stream (same kernel, grid and tiles as inside the
 * solvers) and return in *ms_per_launch the mean device time of one launch,
 * measured with CUDA events recorded on that stream.
 */
int ls_gemv_timed(ls_ctx *ctx, int dtype, int rows, int cols, const void *A, int64_t lda,
                  const float *scale, const void *x, void *y, int reps, double *ms_per_launch);

/*
 * y = A x without any device allocation and without a context.  The paper has
 * no counterpart: this is a library service for callers that cannot allocate
 * device memory -- a process whose device memory is already fully reserved by
 * a framework's caching allocator or a memory pool (a direct cudaMalloc would
 * fail or fragment the pool), or a latency-bound loop that must not pay for
 * cudaMalloc / cudaFree, which can synchronise the whole device.  (ls_gemv
 * needs a context, and ls_create allocates the context's device block.)
 *
 * Arguments are those of ls_gemv (every format, LS_F64_PAIR included), plus
 * the cudaStream_t to run on (NULL = the legacy default stream); the current
 * device is used.  The call copies the matrix descriptor from host memory,
 * launches, reads the kernel's status back and synchronises the stream, so it
 * returns after y is written and must not be called while the stream is being
 * captured into a CUDA graph.  Every piece of scratch the kernel needs (matrix descriptor,
 * state block, completion ticket, per-CTA and per-row-tile partial sums)
 * lives in one static device array of LS_NOALLOC_SCRATCH_BYTES that every GPU
 * loading this library holds until the process exits; it has room for the
 * partial sums of LS_NOALLOC_MAX_CTAS CTAs (the kernel runs 2 CTAs per SM), so
 * on a device with more than LS_NOALLOC_MAX_CTAS / 2 SMs the call returns
 * LS_ERR_UNSUPPORTED.  The array is shared by every call on a device and keeps
 * the last call's contents (each call clears what must start at zero), so
 * calls whose work overlaps on the GPU -- from several host threads, or on
 * several streams -- race and must be serialised by the caller.  The first
 * call on each device looks up the device address of the array
 * (cudaGetSymbolAddress) and raises the kernel's shared-memory limit on that
 * device.  LS_ERR_ARG for bad sizes or pointers (LS_F64_PAIR also needs lda a
 * multiple of 4); LS_ERR_CUDA if a CUDA call fails; LS_ERR_TIMEOUT if a
 * bounded on-device wait gave up.
 */
#define LS_NOALLOC_MAX_CTAS 512
#define LS_NOALLOC_SCRATCH_BYTES (576 * 1024)
int ls_gemv_noalloc(int dtype, int rows, int cols, const void *A, int64_t lda,
                    const float *scale, const void *x, void *y, void *cuda_stream);

/*
 * Tile shapes of the batched engine (ls_batch_solve and the server), chosen
 * by timing.  The paper has no counterpart: its CUBLAS calls have fixed
 * shapes.  Each system of a batch, with s right-hand sides padded to sp in
 * {4, 8, 16, 32} columns, streams A in product tasks of 256 rows x ks32
 * columns and forms its FP32 inner block products on the tensor cores or on
 * the FP32 pipe (sp >= 16 only).  The choice for a system depends only on its
 * own n, s and the GPU's SM count, so a system gives the same bits alone or
 * in any batch.  Defaults without a cache: ks32 = 512, tensor cores for
 * sp >= 16.
 *
 * ls_autotune times every candidate (ks32 in {256, 512, 1024}, tensor cores
 * or FP32 pipe) on synthetic batches of each size bucket [2^b, 2^(b+1)),
 * b = 6..13, and each sp, keeps the fastest in this process, and writes them
 * to `path` (may be NULL) as a JSON cache keyed by (bucket, sp, precision of
 * the inner products, SM count).  flags: LS_TUNE_QUICK times only buckets 9
 * and 10 and sp 16 and 32.  It allocates its synthetic systems itself and
 * runs for seconds (tens of seconds for the full set); synchronous on the
 * context's stream.  LS_ERR_ARG for a NULL context or an unwritable path.
 *
 * ls_tune_load reads a cache written by ls_autotune (entries timed on a GPU
 * with another SM count are ignored at lookup); LS_ERR_ARG if the file is
 * missing or malformed (the current choices stay).  Without a call, the
 * first lookup of the process reads the file named by the environment
 * variable LS_TUNE_CACHE, if set.  ls_tune_reset returns to the defaults.
 * ls_tune_lookup reports the choice for an n x n system with nrhs columns on
 * a GPU of num_sms SMs.  These three touch no GPU and are thread-safe.
 */
#define LS_TUNE_QUICK 1
int ls_autotune(ls_ctx *ctx, const char *path, int flags);
int ls_tune_load(const char *path);
int ls_tune_reset(void);
int ls_tune_lookup(int n, int nrhs, int num_sms, int *ks32, int *tensor_cores);

/*
 * The direct method for symmetric positive definite A (paper: the Cholesky
 * factorization A = L L^T of the direct-methods section, Fig. 3 and the block
 * relations after it; then L y = b and L^T x = y).  Column by column: l_kk =
 * sqrt(a_kk), l_ik = a_ik / l_kk, a_ij -= l_ik l_jk (k < j <= i); only the
 * lower triangle of A is read.  b is carried along as an extra row, so L y =
 * b is done during the factorization.  FP64, run by panels of 32 columns (the
 * panel's steps, then the trailing lower triangle), which only regroups the
 * operations: every element of L and y is bit for bit what the plain column
 * factorization and forward substitution give in FP64 (IEEE square root and
 * division, multiply and subtract not fused, the updates of each element in
 * step order); x differs from a scalar back substitution by the order of its
 * sums.  After the solve the true residual ||b - A x|| is formed
 * (info->rel_res, true_rel_res; info->iters = 0).  A pivot a_kk <= 0 (A not
 * positive definite) or NaN returns LS_BREAKDOWN with x unchanged; a residual
 * that is not finite returns LS_ERR_NAN.  A row-major n x n (host or device),
 * b and x n vectors; opts may be NULL; opts->precision must be LS_F64.  The
 * factorization is n^3 / 6 updates of two FP64 instructions each, bound by
 * the FP64 pipe.
 */
int ls_chol_solve(ls_ctx *ctx, int n, const double *A, int64_t lda, const double *b, double *x,
                  const ls_opts *opts, ls_info *info);

/*
 * The factorization of ls_chol_solve alone: L (n x n, row-major, leading
 * dimension ldl >= n) receives the lower factor with zeros above the
 * diagonal, y = L^-1 b.  Outputs may be host or device memory.  Returns
 * LS_BREAKDOWN when a pivot is not positive and then sets *step (if not NULL)
 * to that step k; only the panels of 32 steps completed before k are final
 * in L and y.  *step is -1 otherwise.  LS_ERR_ARG on bad sizes or NULL
 * pointers.
 */
int ls_chol_factor(ls_ctx *ctx, int n, const double *A, int64_t lda, const double *b, double *L,
                   int64_t ldl, double *y, int *step);

/* Kernels the context has executed on the device since it was created. */
long long ls_kernel_launches(ls_ctx *ctx);

/* Static description of a status code. */
const char *ls_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* LS_H */
