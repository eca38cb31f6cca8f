/*
 * ls_oracle.c -- the ORACLE for the dense Krylov solvers.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously-correct
 * FP64 CPU statement of what the GPU library computes.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or helper with the CUDA library, and the
 * library never calls it.
 *
 * Paper: Oancea, Andrei, Dragoescu, "Improving the performance of the linear
 * systems solvers using CUDA" (arXiv:1511.07207).
 *   - Krylov frame x(i) = x(i-1) + d(i), inner products / saxpy / matvec:
 *     section "Serial iterative and direct methods", opening paragraphs.
 *   - Conjugate gradient: same section, CG paragraph (prose only; the paper
 *     points to Golub & Van Loan for the full statement, which is the
 *     Hestenes-Stiefel form written out below).
 *   - GMRES: same section, GMRES pseudocode (Arnoldi with Gram-Schmidt) and
 *     the restart paragraph that follows it.  The paper stops before the
 *     least-squares step; the Givens-rotation update used here is the
 *     standard one from Saad's book, which the paper cites for GMRES.
 *   - Jacobi: same section, first paragraph (the stationary methods, which
 *     the paper takes from the textbooks): x(k+1) = x(k) + D^-1 (b - A x(k)).
 *   - Gauss-Seidel: same passage; the forward sweep in place, each x_i
 *     recomputed from the newest values of the others.
 *   - Block CG: the CG paragraph's method for several right-hand sides at
 *     once in O'Leary's block form (s x s step matrices instead of scalars).
 *   - Block GMRES: the GMRES pseudocode and restart paragraph with a block
 *     Arnoldi process over the s right-hand sides at once.
 *   - BiCGSTAB: same section, BiCGSTAB listing, with the steps the listing
 *     leaves out written in (see or_bicgstab).
 *   - Gaussian elimination with partial pivoting: same section,
 *     "Right-looking LU factorization", then forward/back substitution.
 *   - Cholesky factorization A = L L^T of an SPD matrix: same section, the
 *     Cholesky paragraph (Figure 3 and the three computations that follow
 *     it), taken one column at a time, then L y = b and L^T x = y.
 *   - Mixed precision (BF16 / FP8-e4m3 storage of A, FP32 inner CG, FP64
 *     outer refinement) extends the paper's single/double precision axis
 *     (section "Results").
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py
 * against mathematics that does not depend on this file (numpy/LAPACK
 * solves and least squares, Krylov optimality, Arnoldi relation,
 * finite termination, nearest-value brute force for the roundings).
 *
 * Conventions: A is row-major with leading dimension lda >= n (element
 * (i,j) at A[i*lda + j]).  Status codes: 0 converged, 1 not converged,
 * 2 breakdown, -1 bad argument.
 *
 * Build: plain C99, -O2 -ffp-contract=off (no fused multiply-add, no
 * reassociation), optional -fopenmp which only splits the rows of a
 * matrix-vector product across threads (each row's sum keeps its order,
 * so results do not depend on the thread count).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_NOT_CONVERGED 1
#define OR_BREAKDOWN 2
#define OR_ERR_ARG (-1)

/* ------------------------------------------------------------------ */
/* BLAS-1/2 in plain loops                                             */
/* ------------------------------------------------------------------ */

static double dot(int n, const double *x, const double *y) {
    double s = 0.0;
    for (int i = 0; i < n; i++) s += x[i] * y[i];
    return s;
}

static double nrm2(int n, const double *x) { return sqrt(dot(n, x, x)); }

/* y = A x, row by row, each row summed left to right. */
static void gemv(int nrows, int ncols, const double *A, long lda,
                 const double *x, double *y, int nthreads) {
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(static)
#else
    (void)nthreads;
#endif
    for (int i = 0; i < nrows; i++) {
        const double *a = A + (long)i * lda;
        double s = 0.0;
        for (int j = 0; j < ncols; j++) s += a[j] * x[j];
        y[i] = s;
    }
}

int or_gemv(int nrows, int ncols, const double *A, long lda, const double *x,
            double *y, int nthreads) {
    if (nrows < 0 || ncols < 0 || lda < ncols) return OR_ERR_ARG;
    gemv(nrows, ncols, A, lda, x, y, nthreads);
    return OR_OK;
}

/* r = b - A x */
static void residual(int n, const double *A, long lda, const double *b,
                     const double *x, double *r, int nthreads) {
    gemv(n, n, A, lda, x, r, nthreads);
    for (int i = 0; i < n; i++) r[i] = b[i] - r[i];
}

int or_residual(int n, const double *A, long lda, const double *b,
                const double *x, double *r, int nthreads) {
    if (n < 0 || lda < n) return OR_ERR_ARG;
    residual(n, A, lda, b, x, r, nthreads);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Conjugate gradient (Hestenes-Stiefel), FP64                         */
/* ------------------------------------------------------------------ */
/*
 * Solves A x = b for SPD A.  Stops when the recursively updated residual
 * satisfies ||r|| <= rtol ||b||; the true residual b - A x is then
 * recomputed and, if it does not pass, the iteration restarts from it
 * (r = b - A x, p = r).  iters counts the matrix-vector products inside the
 * loop.  Optional histories (for tests on small n): R_hist and P_hist are
 * column-major n x (max_iter+1) arrays receiving r_k and p_k, res_hist
 * receives ||r_k|| for k = 0..iters.
 */
int or_cg(int n, const double *A, long lda, const double *b, double *x,
          double rtol, int max_iter, int x0_given, int nthreads,
          int *iters_out, double *rel_res_out,
          double *res_hist, double *R_hist, double *P_hist) {
    if (n < 0 || lda < n || max_iter < 0) return OR_ERR_ARG;
    double *r = malloc(sizeof(double) * (n ? n : 1));
    double *p = malloc(sizeof(double) * (n ? n : 1));
    double *q = malloc(sizeof(double) * (n ? n : 1));
    int status = OR_NOT_CONVERGED, k = 0;
    double nb = nrm2(n, b), rho;

    if (!x0_given) {
        for (int i = 0; i < n; i++) { x[i] = 0.0; r[i] = b[i]; }
    } else {
        residual(n, A, lda, b, x, r, nthreads);
    }
    if (nb == 0.0) {                      /* b = 0: x = 0 solves exactly */
        for (int i = 0; i < n; i++) x[i] = 0.0;
        *iters_out = 0; *rel_res_out = 0.0;
        free(r); free(p); free(q);
        return OR_OK;
    }
    memcpy(p, r, sizeof(double) * n);
    rho = dot(n, r, r);
    if (res_hist) res_hist[0] = sqrt(rho);
    if (R_hist) memcpy(R_hist, r, sizeof(double) * n);
    if (P_hist) memcpy(P_hist, p, sizeof(double) * n);

    int check = sqrt(rho) <= rtol * nb;
    for (;;) {
        if (check) {
            /* recursive residual passed: confirm with the true residual */
            residual(n, A, lda, b, x, q, nthreads);
            double t = nrm2(n, q);
            if (t <= rtol * nb) { status = OR_OK; break; }
            memcpy(r, q, sizeof(double) * n);
            memcpy(p, r, sizeof(double) * n);
            rho = dot(n, r, r);
            check = 0;
        }
        if (k >= max_iter) break;
        gemv(n, n, A, lda, p, q, nthreads);          /* q = A p */
        double pq = dot(n, p, q);
        if (!(pq > 0.0)) { status = OR_BREAKDOWN; break; }  /* not SPD, or NaN */
        double alpha = rho / pq;
        for (int i = 0; i < n; i++) x[i] += alpha * p[i];
        for (int i = 0; i < n; i++) r[i] -= alpha * q[i];
        double rho_new = dot(n, r, r);
        k++;
        if (res_hist) res_hist[k] = sqrt(rho_new);
        if (sqrt(rho_new) <= rtol * nb) {
            check = 1;
            rho = rho_new;
            if (R_hist) memcpy(R_hist + (long)k * n, r, sizeof(double) * n);
            continue;
        }
        double beta = rho_new / rho;
        for (int i = 0; i < n; i++) p[i] = r[i] + beta * p[i];
        rho = rho_new;
        if (R_hist) memcpy(R_hist + (long)k * n, r, sizeof(double) * n);
        if (P_hist) memcpy(P_hist + (long)k * n, p, sizeof(double) * n);
    }
    residual(n, A, lda, b, x, q, nthreads);
    *rel_res_out = nrm2(n, q) / nb;
    *iters_out = k;
    free(r); free(p); free(q);
    return status;
}

/* ------------------------------------------------------------------ */
/* Block CG (O'Leary), FP64                                            */
/* ------------------------------------------------------------------ */
/* Cholesky G = L L^T of an s x s SPD matrix (column-major, in place:
 * L in the lower triangle).  0 on success, 1 if a pivot is not positive. */
static int chol(int s, double *G) {
    for (int j = 0; j < s; j++) {
        double d = G[j + j * s];
        for (int k = 0; k < j; k++) d -= G[j + k * s] * G[j + k * s];
        if (!(d > 0.0)) return 1;
        d = sqrt(d);
        G[j + j * s] = d;
        for (int i = j + 1; i < s; i++) {
            double v = G[i + j * s];
            for (int k = 0; k < j; k++) v -= G[i + k * s] * G[j + k * s];
            G[i + j * s] = v / d;
        }
    }
    return 0;
}

/* Y = G^-1 Y for s x s matrices, G = L L^T factored by chol. */
static void chol_solve(int s, const double *L, double *Y) {
    for (int c = 0; c < s; c++) {
        double *y = Y + c * s;
        for (int i = 0; i < s; i++) {                 /* L z = y */
            double v = y[i];
            for (int k = 0; k < i; k++) v -= L[i + k * s] * y[k];
            y[i] = v / L[i + i * s];
        }
        for (int i = s - 1; i >= 0; i--) {            /* L^T w = z */
            double v = y[i];
            for (int k = i + 1; k < s; k++) v -= L[k + i * s] * y[k];
            y[i] = v / L[i + i * s];
        }
    }
}

/* Y = G^-1 Y for an r x r G = L L^T factored by chol and Y r x c (column-major). */
static void chol_solve_rect(int r, int c, const double *L, double *Y) {
    for (int j = 0; j < c; j++) {
        double *y = Y + (long)j * r;
        for (int i = 0; i < r; i++) {
            double v = y[i];
            for (int k = 0; k < i; k++) v -= L[i + k * r] * y[k];
            y[i] = v / L[i + i * r];
        }
        for (int i = r - 1; i >= 0; i--) {
            double v = y[i];
            for (int k = i + 1; k < r; k++) v -= L[k + i * r] * y[k];
            y[i] = v / L[i + i * r];
        }
    }
}

/* G = U^T V for n x s column-major blocks (s x s, column-major). */
static void gram(int n, int s, const double *U, const double *V, double *G) {
    for (int j = 0; j < s; j++)
        for (int i = 0; i < s; i++) G[i + j * s] = dot(n, U + (long)i * n, V + (long)j * n);
}

/*
 * Block conjugate gradient (O'Leary) for SPD A and s right-hand sides B
 * (n x s, column-major), X (n x s) in/out:
 *   R = B - A X, P = R, rho = R^T R
 *   loop: Q = A P; gamma = P^T Q; alpha = gamma^-1 rho;
 *         X += P alpha; R -= Q alpha; rho' = R^T R;
 *         stop when every column has ||R_j|| <= rtol ||B_j|| (confirmed on
 *         the true residual; a failed confirmation restarts from it);
 *         beta = rho^-1 rho'; P = R + P beta; rho = rho'.
 * iters counts block products.  gamma or rho not positive definite (a
 * rank-deficient residual block: linearly dependent or zero columns of B, or
 * columns that converged exactly) is a breakdown (status 2).  rel_res_out is
 * the largest true relative residual over the columns.
 */
int or_block_cg(int n, int s, const double *A, long lda, const double *B, double *X,
                double rtol, int max_iter, int x0_given, int nthreads,
                int *iters_out, double *rel_res_out) {
    if (n < 0 || s < 1 || lda < n || max_iter < 0) return OR_ERR_ARG;
    const size_t nb = sizeof(double) * (size_t)(n ? n : 1) * s, sb = sizeof(double) * s * s;
    double *R = malloc(nb), *P = malloc(nb), *Q = malloc(nb), *T = malloc(nb);
    double *rho = malloc(sb), *rhon = malloc(sb), *Lr = malloc(sb), *g = malloc(sb), *al = malloc(sb);
    double *bn = malloc(sizeof(double) * s);
    int status = OR_NOT_CONVERGED, k = 0;
    for (int j = 0; j < s; j++) bn[j] = nrm2(n, B + (long)j * n);

    /* R = B - A X (or B), P = R, rho = R^T R and its factor */
    #define RESTART()                                                              \
        do {                                                                       \
            for (int j = 0; j < s; j++)                                            \
                residual(n, A, lda, B + (long)j * n, X + (long)j * n, R + (long)j * n, nthreads); \
            memcpy(P, R, nb);                                                      \
            gram(n, s, R, R, rho);                                                 \
        } while (0)
    if (!x0_given) memset(X, 0, nb);
    RESTART();
    int check = 1;
    for (int j = 0; j < s; j++) check = check && sqrt(rho[j + j * s]) <= rtol * bn[j];
    for (;;) {
        if (check) {
            int ok = 1;
            for (int j = 0; j < s && ok; j++) {
                residual(n, A, lda, B + (long)j * n, X + (long)j * n, T, nthreads);
                ok = nrm2(n, T) <= rtol * bn[j];
            }
            if (ok) { status = OR_OK; break; }
            RESTART();
            check = 0;
        }
        if (k >= max_iter) break;
        memcpy(Lr, rho, sb);
        if (chol(s, Lr)) { status = OR_BREAKDOWN; break; }
        for (int j = 0; j < s; j++) gemv(n, n, A, lda, P + (long)j * n, Q + (long)j * n, nthreads);
        gram(n, s, P, Q, g);                                  /* gamma = P^T Q */
        if (chol(s, g)) { status = OR_BREAKDOWN; break; }
        memcpy(al, rho, sb);
        chol_solve(s, g, al);                                  /* alpha = gamma^-1 rho */
        for (int j = 0; j < s; j++)
            for (int c = 0; c < s; c++) {
                const double a = al[c + j * s];
                for (int i = 0; i < n; i++) {
                    X[i + (long)j * n] += P[i + (long)c * n] * a;
                    R[i + (long)j * n] -= Q[i + (long)c * n] * a;
                }
            }
        k++;
        gram(n, s, R, R, rhon);
        int conv = 1;
        for (int j = 0; j < s; j++) conv = conv && sqrt(rhon[j + j * s]) <= rtol * bn[j];
        if (conv) {
            check = 1;
            memcpy(rho, rhon, sb);
            continue;
        }
        memcpy(al, rhon, sb);
        chol_solve(s, Lr, al);                                 /* beta = rho^-1 rho' */
        for (int j = 0; j < s; j++) {                          /* P = R + P beta */
            for (int i = 0; i < n; i++) {
                double v = R[i + (long)j * n];
                for (int c = 0; c < s; c++) v += P[i + (long)c * n] * al[c + j * s];
                T[i + (long)j * n] = v;
            }
        }
        memcpy(P, T, nb);
        memcpy(rho, rhon, sb);
    }
    #undef RESTART
    double worst = 0.0;
    for (int j = 0; j < s; j++) {
        residual(n, A, lda, B + (long)j * n, X + (long)j * n, T, nthreads);
        const double rr = bn[j] > 0.0 ? nrm2(n, T) / bn[j] : nrm2(n, T);
        if (rr > worst || rr != rr) worst = rr;
    }
    *rel_res_out = worst;
    *iters_out = k;
    free(R); free(P); free(Q); free(T); free(rho); free(rhon); free(Lr); free(g); free(al); free(bn);
    return status;
}

/*
 * Orthonormal basis of the range of W (n x s, column-major) with the
 * dependent columns dropped: modified Gram-Schmidt with column pivoting.
 * Each step takes, among the columns not yet taken or dropped, the one with
 * the largest remaining norm, orthogonalizes it once more against the basis
 * so far, and keeps it as the next basis vector; every remaining column then
 * loses its component along that vector.  A column whose part outside the
 * span of the basis is at most tau times its own norm (a zero column
 * included) is dependent and dropped.  Q receives the rank orthonormal
 * columns, then zero columns.  Returns the rank.
 */
static int orth_rr(int n, int s, const double *W, double *Q, double tau) {
    double *Wc = malloc(sizeof(double) * (size_t)(n ? n : 1) * s);
    double *n0 = malloc(sizeof(double) * s), *cur = malloc(sizeof(double) * s);
    int *state = calloc((size_t)s, sizeof(int));          /* 0 open, 1 taken, 2 dropped */
    memcpy(Wc, W, sizeof(double) * (size_t)n * s);
    for (int j = 0; j < s; j++) n0[j] = cur[j] = nrm2(n, Wc + (long)j * n);
    int r = 0;
    for (;;) {
        int p = -1;
        for (int j = 0; j < s; j++) {
            if (state[j]) continue;
            if (!(cur[j] > tau * n0[j])) { state[j] = 2; continue; }
            if (p < 0 || cur[j] > cur[p]) p = j;
        }
        if (p < 0) break;
        double *w = Wc + (long)p * n;
        for (int i = 0; i < r; i++) {                      /* the second pass */
            const double *q = Q + (long)i * n;
            const double h = dot(n, q, w);
            for (int t = 0; t < n; t++) w[t] -= h * q[t];
        }
        const double nw = nrm2(n, w);
        if (!(nw > tau * n0[p])) { state[p] = 2; continue; }
        double *q = Q + (long)r * n;
        for (int t = 0; t < n; t++) q[t] = w[t] / nw;
        state[p] = 1;
        r++;
        for (int j = 0; j < s; j++) {                      /* the first pass of the others */
            if (state[j]) continue;
            double *v = Wc + (long)j * n;
            const double h = dot(n, q, v);
            for (int t = 0; t < n; t++) v[t] -= h * q[t];
            cur[j] = nrm2(n, v);
        }
    }
    for (int j = r; j < s; j++) memset(Q + (long)j * n, 0, sizeof(double) * (size_t)n);
    free(Wc); free(n0); free(cur); free(state);
    return r;
}

/*
 * Block CG that drops dependent directions instead of breaking down (the
 * block form of the paper's CG with the search directions kept orthonormal
 * and of full rank, as in the breakdown-free block CG of Ji and Li):
 *   R = B - A X;  P = orth(R)                  (rank r <= s)
 *   loop: Q = A P;  gamma = P^T Q (r x r);  alpha = gamma^-1 (P^T R);
 *         X += P alpha;  R -= Q alpha;
 *         stop when every column has ||R_j|| <= rtol ||B_j|| (confirmed on
 *         the true residual; a failed confirmation restarts from it);
 *         beta = -gamma^-1 (Q^T R);  P = orth(R + P beta).
 * The new directions are A-conjugate to P (P^T A (R + P beta) = 0) and span
 * the same block Krylov space as O'Leary's, so with a full-rank block the
 * iterates are the same; but dependent, zero or converged residual columns
 * only lower the rank of P, and gamma stays positive definite for SPD A.
 * orth drops a column whose part outside the span of the others is at most
 * 1e-8 of its norm.  iters counts block products; rank_out receives the last
 * rank.  gamma not positive definite (A not SPD) is a breakdown (status 2).
 */
int or_block_cg_deflated(int n, int s, const double *A, long lda, const double *B, double *X,
                         double rtol, int max_iter, int x0_given, int nthreads,
                         int *iters_out, double *rel_res_out, int *rank_out) {
    if (n < 0 || s < 1 || lda < n || max_iter < 0) return OR_ERR_ARG;
    const double tau = 1e-8;
    const size_t nb = sizeof(double) * (size_t)(n ? n : 1) * s, sb = sizeof(double) * s * s;
    double *R = malloc(nb), *P = malloc(nb), *Q = malloc(nb), *T = malloc(nb);
    double *g = malloc(sb), *al = malloc(sb), *be = malloc(sb), *bn = malloc(sizeof(double) * s);
    int status = OR_NOT_CONVERGED, k = 0, r = 0;
    for (int j = 0; j < s; j++) bn[j] = nrm2(n, B + (long)j * n);
    if (!x0_given) memset(X, 0, nb);
    #define RESTART_D()                                                            \
        do {                                                                       \
            for (int j = 0; j < s; j++)                                            \
                residual(n, A, lda, B + (long)j * n, X + (long)j * n, R + (long)j * n, nthreads); \
            r = orth_rr(n, s, R, P, tau);                                          \
        } while (0)
    RESTART_D();
    int check = 1;
    for (int j = 0; j < s; j++) check = check && nrm2(n, R + (long)j * n) <= rtol * bn[j];
    for (;;) {
        if (check) {
            int ok = 1;
            for (int j = 0; j < s && ok; j++) {
                residual(n, A, lda, B + (long)j * n, X + (long)j * n, T, nthreads);
                ok = nrm2(n, T) <= rtol * bn[j];
            }
            if (ok) { status = OR_OK; break; }
            RESTART_D();
            check = 0;
        }
        if (k >= max_iter) break;
        if (r == 0) { status = OR_BREAKDOWN; break; }      /* nothing left to search, not converged */
        for (int j = 0; j < r; j++) gemv(n, n, A, lda, P + (long)j * n, Q + (long)j * n, nthreads);
        gram(n, r, P, Q, g);                                   /* gamma = P^T Q (r x r) */
        if (chol(r, g)) { status = OR_BREAKDOWN; break; }
        for (int j = 0; j < s; j++)                            /* alpha = gamma^-1 P^T R (r x s) */
            for (int i = 0; i < r; i++) al[i + j * r] = dot(n, P + (long)i * n, R + (long)j * n);
        chol_solve_rect(r, s, g, al);
        for (int j = 0; j < s; j++)
            for (int c = 0; c < r; c++) {
                const double a = al[c + j * r];
                for (int i = 0; i < n; i++) {
                    X[i + (long)j * n] += P[i + (long)c * n] * a;
                    R[i + (long)j * n] -= Q[i + (long)c * n] * a;
                }
            }
        k++;
        int conv = 1;
        for (int j = 0; j < s; j++) conv = conv && nrm2(n, R + (long)j * n) <= rtol * bn[j];
        if (conv) { check = 1; continue; }
        for (int j = 0; j < s; j++)                            /* beta = -gamma^-1 Q^T R (r x s) */
            for (int i = 0; i < r; i++) be[i + j * r] = -dot(n, Q + (long)i * n, R + (long)j * n);
        chol_solve_rect(r, s, g, be);
        for (int j = 0; j < s; j++)                            /* T = R + P beta */
            for (int i = 0; i < n; i++) {
                double v = R[i + (long)j * n];
                for (int c = 0; c < r; c++) v += P[i + (long)c * n] * be[c + j * r];
                T[i + (long)j * n] = v;
            }
        r = orth_rr(n, s, T, P, tau);                           /* P = orth(R + P beta) */
    }
    #undef RESTART_D
    double worst = 0.0;
    for (int j = 0; j < s; j++) {
        residual(n, A, lda, B + (long)j * n, X + (long)j * n, T, nthreads);
        const double rr = bn[j] > 0.0 ? nrm2(n, T) / bn[j] : nrm2(n, T);
        if (rr > worst || rr != rr) worst = rr;
    }
    *rel_res_out = worst;
    *iters_out = k;
    if (rank_out) *rank_out = r;
    free(R); free(P); free(Q); free(T); free(g); free(al); free(be); free(bn);
    return status;
}

/* ------------------------------------------------------------------ */
/* Jacobi, FP64                                                        */
/* ------------------------------------------------------------------ */
/*
 * The stationary Jacobi iteration x(k+1) = x(k) + D^-1 (b - A x(k)), D the
 * diagonal of A.  Every product gives the residual of the current iterate;
 * the iteration stops when ||b - A x(k)|| <= rtol ||b||, or after max_iter
 * products, and returns the last iterate it measured, so the residual it
 * reports is that iterate's true one.  iters counts the products.  A zero
 * diagonal entry is a breakdown (status 2).  res_hist (optional, length
 * max_iter + 1) receives ||b - A x(k)|| for k = 0 .. iters - 1.
 */
int or_jacobi(int n, const double *A, long lda, const double *b, double *x,
              double rtol, int max_iter, int x0_given, int nthreads,
              int *iters_out, double *rel_res_out, double *res_hist) {
    if (n < 0 || lda < n || max_iter < 0) return OR_ERR_ARG;
    const size_t sz = sizeof(double) * (n ? n : 1);
    double *r = malloc(sz);
    int status = OR_NOT_CONVERGED, k = 0;
    const double nb = nrm2(n, b), tol = rtol * nrm2(n, b);
    if (!x0_given)
        for (int i = 0; i < n; i++) x[i] = 0.0;
    for (int i = 0; i < n; i++)
        if (A[(long)i * lda + i] == 0.0) { status = OR_BREAKDOWN; goto done; }
    if (nb == 0.0) {
        for (int i = 0; i < n; i++) x[i] = 0.0;
        status = OR_OK;
        goto done;
    }
    while (k < max_iter) {
        residual(n, A, lda, b, x, r, nthreads);          /* r = b - A x(k) */
        const double nr = nrm2(n, r);
        if (res_hist) res_hist[k] = nr;
        k++;
        if (!isfinite(nr)) break;
        if (nr <= tol) { status = OR_OK; break; }
        if (k == max_iter) break;
        for (int i = 0; i < n; i++) x[i] += r[i] / A[(long)i * lda + i];
    }
done:
    residual(n, A, lda, b, x, r, nthreads);
    *rel_res_out = nb > 0.0 ? nrm2(n, r) / nb : 0.0;
    *iters_out = k;
    free(r);
    return status;
}

/* ------------------------------------------------------------------ */
/* Gauss-Seidel, FP64                                                  */
/* ------------------------------------------------------------------ */
/*
 * The forward Gauss-Seidel sweep: for i = 0 .. n-1 in turn,
 *   x_i = (b_i - sum_{j != i} a_ij x_j) / a_ii,
 * with x_j already updated in this sweep for j < i and not yet for j > i.
 * The stopping rule, the iterate returned, iters, the breakdown on a zero
 * a_ii and res_hist are those of or_jacobi.
 */
int or_gauss_seidel(int n, const double *A, long lda, const double *b, double *x,
                    double rtol, int max_iter, int x0_given, int nthreads,
                    int *iters_out, double *rel_res_out, double *res_hist) {
    if (n < 0 || lda < n || max_iter < 0) return OR_ERR_ARG;
    const size_t sz = sizeof(double) * (n ? n : 1);
    double *r = malloc(sz);
    int status = OR_NOT_CONVERGED, k = 0;
    const double nb = nrm2(n, b), tol = rtol * nrm2(n, b);
    if (!x0_given)
        for (int i = 0; i < n; i++) x[i] = 0.0;
    for (int i = 0; i < n; i++)
        if (A[(long)i * lda + i] == 0.0) { status = OR_BREAKDOWN; goto done; }
    if (nb == 0.0) {
        for (int i = 0; i < n; i++) x[i] = 0.0;
        status = OR_OK;
        goto done;
    }
    while (k < max_iter) {
        residual(n, A, lda, b, x, r, nthreads);          /* r = b - A x(k) */
        const double nr = nrm2(n, r);
        if (res_hist) res_hist[k] = nr;
        k++;
        if (!isfinite(nr)) break;
        if (nr <= tol) { status = OR_OK; break; }
        if (k == max_iter) break;
        for (int i = 0; i < n; i++) {                    /* the sweep, in place */
            const double *a = A + (long)i * lda;
            double s = b[i];
            for (int j = 0; j < n; j++)
                if (j != i) s -= a[j] * x[j];
            x[i] = s / a[i];
        }
    }
done:
    residual(n, A, lda, b, x, r, nthreads);
    *rel_res_out = nb > 0.0 ? nrm2(n, r) / nb : 0.0;
    *iters_out = k;
    free(r);
    return status;
}

/* ------------------------------------------------------------------ */
/* BiCGSTAB, FP64                                                      */
/* ------------------------------------------------------------------ */
/*
 * The paper's BiCGSTAB (van der Vorst's stabilised BiCG), in the order of its
 * listing: rho_0 = 1, rho_1 = r^.r with the shadow residual r^ = r(0),
 * alpha = omega = 1, p = v = 0; per step beta = (rho_k / rho_{k-1})
 * (alpha / omega), p = r + beta (p - omega v), v = A p, alpha = rho_k /
 * (r^.v), s = r - alpha v, t = A s, omega, x += alpha p + omega s.  The
 * listing prints omega as a product and leaves out three steps, written in
 * here: omega = (t.s) / (t.t); r = s - omega t; rho_{k+1} = r^.r; and the
 * stop test ||r|| <= rtol ||b||, confirmed on the true residual b - A x (when
 * it fails, the iteration restarts from it with r^ = r).  When ||s|| already
 * passes the test the step ends with x += alpha p (no second product).
 * Breakdown (status 2): rho = 0, r^.v = 0, or t.t = 0 / omega = 0 with s != 0.
 * iters counts the matrix-vector products inside the loop (two per full
 * step).  Optional traces for tests, one entry per step (length max_iter):
 * shs[k] = (r^.s) / (|r^| |s|) and rt[k] = (r_new.t) / (|r_new| |t|); both
 * are zero in exact arithmetic (alpha makes s orthogonal to r^, omega
 * minimises ||s - omega t||, so r_new is orthogonal to t); alphas[k] = alpha of
 * the step (equal to BiCG's in exact arithmetic).  steps_out receives the
 * number of traced steps.
 */
int or_bicgstab(int n, const double *A, long lda, const double *b, double *x,
                double rtol, int max_iter, int x0_given, int nthreads,
                int *iters_out, double *rel_res_out, double *shs, double *rt, double *alphas,
                int *steps_out) {
    if (n < 0 || lda < n || max_iter < 0) return OR_ERR_ARG;
    const size_t sz = sizeof(double) * (n ? n : 1);
    double *r = malloc(sz), *rh = malloc(sz), *p = malloc(sz), *v = malloc(sz);
    double *s = malloc(sz), *t = malloc(sz), *q = malloc(sz);
    int status = OR_NOT_CONVERGED, k = 0, steps = 0;
    const double nb = nrm2(n, b), tol = rtol * nrm2(n, b);
    double rho_prev, rho, alpha, omega;

    if (!x0_given) {
        for (int i = 0; i < n; i++) { x[i] = 0.0; r[i] = b[i]; }
    } else {
        residual(n, A, lda, b, x, r, nthreads);
    }
    if (nb == 0.0) {                      /* b = 0: x = 0 solves exactly */
        for (int i = 0; i < n; i++) x[i] = 0.0;
        *iters_out = 0; *rel_res_out = 0.0;
        if (steps_out) *steps_out = 0;
        free(r); free(rh); free(p); free(v); free(s); free(t); free(q);
        return OR_OK;
    }
    int check = nrm2(n, r) <= tol, fresh = 1;
    for (;;) {
        if (fresh) {                      /* (re)start: r^ = r, rho_0 = 1, p = v = 0 */
            memcpy(rh, r, sizeof(double) * n);
            for (int i = 0; i < n; i++) { p[i] = 0.0; v[i] = 0.0; }
            rho_prev = 1.0;
            rho = dot(n, rh, r);
            alpha = 1.0;
            omega = 1.0;
            fresh = 0;
        }
        if (check) {
            residual(n, A, lda, b, x, q, nthreads);
            if (nrm2(n, q) <= tol) { status = OR_OK; break; }
            memcpy(r, q, sizeof(double) * n);
            check = 0;
            fresh = 1;
            continue;
        }
        if (k >= max_iter) break;
        if (rho == 0.0 || !isfinite(rho)) { status = OR_BREAKDOWN; break; }
        const double beta = (rho / rho_prev) * (alpha / omega);
        for (int i = 0; i < n; i++) p[i] = r[i] + beta * (p[i] - omega * v[i]);
        gemv(n, n, A, lda, p, v, nthreads);          /* v = A p */
        k++;
        const double rv = dot(n, rh, v);
        if (rv == 0.0 || !isfinite(rv)) { status = OR_BREAKDOWN; break; }
        alpha = rho / rv;
        if (alphas) alphas[steps] = alpha;
        for (int i = 0; i < n; i++) s[i] = r[i] - alpha * v[i];
        const double ns = nrm2(n, s);
        if (shs) shs[steps] = dot(n, rh, s) / (nrm2(n, rh) * (ns > 0.0 ? ns : 1.0));
        if (ns <= tol) {                  /* s passes: x += alpha p ends the step */
            for (int i = 0; i < n; i++) x[i] += alpha * p[i];
            memcpy(r, s, sizeof(double) * n);
            if (rt) rt[steps] = 0.0;
            steps++;
            check = 1;
            continue;
        }
        if (k >= max_iter) {
            for (int i = 0; i < n; i++) x[i] += alpha * p[i];
            memcpy(r, s, sizeof(double) * n);
            steps++;
            break;
        }
        gemv(n, n, A, lda, s, t, nthreads);          /* t = A s */
        k++;
        const double tt = dot(n, t, t);
        if (tt == 0.0 || !isfinite(tt)) { status = OR_BREAKDOWN; break; }
        omega = dot(n, t, s) / tt;
        for (int i = 0; i < n; i++) x[i] += alpha * p[i] + omega * s[i];
        for (int i = 0; i < n; i++) r[i] = s[i] - omega * t[i];
        if (rt) {
            const double nr = nrm2(n, r), nt = sqrt(tt);
            rt[steps] = dot(n, r, t) / ((nr > 0.0 ? nr : 1.0) * nt);
        }
        steps++;
        rho_prev = rho;
        rho = dot(n, rh, r);
        if (omega == 0.0) { status = OR_BREAKDOWN; break; }
        check = nrm2(n, r) <= tol;
    }
    residual(n, A, lda, b, x, q, nthreads);
    *rel_res_out = nrm2(n, q) / nb;
    *iters_out = k;
    if (steps_out) *steps_out = steps;
    free(r); free(rh); free(p); free(v); free(s); free(t); free(q);
    return status;
}

/* ------------------------------------------------------------------ */
/* Restarted GMRES(m), FP64                                            */
/* ------------------------------------------------------------------ */
/*
 * Each cycle: r = b - A x, beta = ||r||, v_1 = r / beta, g = beta e_1.
 * Arnoldi step k: w = A v_k; modified Gram-Schmidt against v_1..v_k
 * (h_jk = w . v_j, w -= h_jk v_j), with one more full pass when
 * ||w|| < 0.7 ||A v_k|| (its coefficients are added to h); h_{k+1,k} = ||w||;
 * v_{k+1} = w / h_{k+1,k}.  The previous Givens rotations are applied to
 * column k, a new rotation (c, s) = (h_kk, h_{k+1,k}) / hypot(...) zeroes
 * h_{k+1,k}, and g_{k+1} = -s g_k, g_k = c g_k, so |g_{k+1}| is the residual
 * norm of the current cycle iterate.  The cycle ends when
 * |g_{k+1}| <= rtol ||b||, when k = m, when the total step count reaches
 * max_iter, or on a (lucky) breakdown h_{k+1,k} <= 1e-14 ||A v_k||.  Then
 * R y = g is back-solved and x += V_k y.  The outer loop stops when the true
 * residual passes.  iters counts Arnoldi steps over all cycles.
 *
 * Optional first-cycle outputs for tests: V1 (column-major n x (m+1)),
 * H1 (column-major (m+1) x m, the unrotated Hessenberg matrix) and k1 (the
 * number of Arnoldi steps of the first cycle).  est_out receives the last
 * |g_{k+1}| / ||b||.
 */
int or_gmres(int n, const double *A, long lda, const double *b, double *x,
             int m, double rtol, int max_iter, int x0_given, int nthreads,
             int *iters_out, int *cycles_out, double *rel_res_out,
             double *est_out, double *V1, double *H1, int *k1) {
    if (n < 0 || lda < n || m < 1 || max_iter < 0) return OR_ERR_ARG;
    long ln = n ? n : 1;
    double *V = calloc((size_t)ln * (m + 1), sizeof(double));
    double *H = calloc((size_t)(m + 1) * m, sizeof(double));  /* rotated, col-major */
    double *Hraw = calloc((size_t)(m + 1) * m, sizeof(double));
    double *cs = calloc(m, sizeof(double)), *sn = calloc(m, sizeof(double));
    double *g = calloc(m + 1, sizeof(double)), *y = calloc(m, sizeof(double));
    double *w = malloc(sizeof(double) * ln), *r = malloc(sizeof(double) * ln);
    int status = OR_NOT_CONVERGED, total = 0, cycles = 0;
    double nb = nrm2(n, b), est = 0.0;
#define HR(i, j) H[(long)(j) * (m + 1) + (i)]
#define HW(i, j) Hraw[(long)(j) * (m + 1) + (i)]

    if (!x0_given) for (int i = 0; i < n; i++) x[i] = 0.0;
    if (k1) *k1 = 0;
    if (nb == 0.0) {
        for (int i = 0; i < n; i++) x[i] = 0.0;
        *iters_out = 0; *cycles_out = 0; *rel_res_out = 0.0;
        if (est_out) *est_out = 0.0;
        status = OR_OK;
        goto done;
    }
    for (;;) {
        residual(n, A, lda, b, x, r, nthreads);
        double beta = nrm2(n, r);
        if (beta <= rtol * nb) { status = OR_OK; break; }
        if (total >= max_iter) break;
        cycles++;
        for (int i = 0; i < n; i++) V[i] = r[i] / beta;
        memset(g, 0, sizeof(double) * (m + 1));
        memset(H, 0, sizeof(double) * (m + 1) * m);
        memset(Hraw, 0, sizeof(double) * (m + 1) * m);
        g[0] = beta;
        int k = 0, stop = 0;
        while (k < m && total < max_iter && !stop) {
            double *vk = V + (long)k * n, *vn = V + (long)(k + 1) * n;
            gemv(n, n, A, lda, vk, w, nthreads);
            double wnorm0 = nrm2(n, w);
            for (int j = 0; j <= k; j++) {                  /* MGS */
                double h = dot(n, w, V + (long)j * n);
                HR(j, k) = h;
                for (int i = 0; i < n; i++) w[i] -= h * V[(long)j * n + i];
            }
            double wnorm = nrm2(n, w);
            if (wnorm < 0.7 * wnorm0) {                     /* second pass */
                for (int j = 0; j <= k; j++) {
                    double h = dot(n, w, V + (long)j * n);
                    HR(j, k) += h;
                    for (int i = 0; i < n; i++) w[i] -= h * V[(long)j * n + i];
                }
                wnorm = nrm2(n, w);
            }
            HR(k + 1, k) = wnorm;
            for (int j = 0; j <= k + 1; j++) HW(j, k) = HR(j, k);
            int lucky = !(wnorm > 1e-14 * wnorm0);
            if (!lucky) for (int i = 0; i < n; i++) vn[i] = w[i] / wnorm;
            /* apply the earlier rotations to column k */
            for (int j = 0; j < k; j++) {
                double a = HR(j, k), c = HR(j + 1, k);
                HR(j, k) = cs[j] * a + sn[j] * c;
                HR(j + 1, k) = -sn[j] * a + cs[j] * c;
            }
            double den = hypot(HR(k, k), HR(k + 1, k));
            if (den == 0.0) { status = OR_BREAKDOWN; stop = 2; break; }
            cs[k] = HR(k, k) / den;
            sn[k] = HR(k + 1, k) / den;
            HR(k, k) = den;
            HR(k + 1, k) = 0.0;
            g[k + 1] = -sn[k] * g[k];
            g[k] = cs[k] * g[k];
            k++;
            total++;
            est = fabs(g[k]) / nb;
            if (fabs(g[k]) <= rtol * nb || lucky) stop = 1;
        }
        if (cycles == 1) {
            if (V1) memcpy(V1, V, sizeof(double) * n * (k + 1 <= m + 1 ? k + 1 : m + 1));
            if (H1) memcpy(H1, Hraw, sizeof(double) * (m + 1) * m);
            if (k1) *k1 = k;
        }
        if (stop == 2) break;
        /* back-solve R y = g on the leading k x k block */
        for (int i = k - 1; i >= 0; i--) {
            double s = g[i];
            for (int j = i + 1; j < k; j++) s -= HR(i, j) * y[j];
            y[i] = s / HR(i, i);
        }
        for (int j = 0; j < k; j++)
            for (int i = 0; i < n; i++) x[i] += V[(long)j * n + i] * y[j];
    }
    residual(n, A, lda, b, x, r, nthreads);
    *rel_res_out = nrm2(n, r) / nb;
    *iters_out = total;
    *cycles_out = cycles;
    if (est_out) *est_out = est;
done:
    free(V); free(H); free(Hraw); free(cs); free(sn); free(g); free(y);
    free(w); free(r);
#undef HR
#undef HW
    return status;
}

/* ------------------------------------------------------------------ */
/* Restarted block GMRES(m), FP64                                      */
/* ------------------------------------------------------------------ */
/*
 * Block GMRES for s right-hand sides B (n x s, column-major), X (n x s)
 * in/out.  A cycle orthonormalises R = B - A X column by column (modified
 * Gram-Schmidt, two passes) into V_1 with R = V_1 S; then for j = 1..m:
 * W = A V_j, and each column of W is orthogonalised (MGS, two passes)
 * against every basis vector so far and normalised, which gives the
 * columns of the band Hessenberg matrix H ((m+1)s x ms, s subdiagonals).
 * Each new column of H is reduced by the earlier Givens rotations and then
 * by s new ones (its subdiagonal entries from the bottom up), applied also
 * to G = [S; 0]; after a block step with k columns the residual of
 * right-hand side c is the norm of rows k..k+s-1 of G's column c.  The
 * cycle ends when every column passes (<= rtol ||B_c||), after m block steps,
 * when total block steps reach max_iter, or after a step whose block lost
 * rank (a column norm at most 1e-14 of its norm before orthogonalisation:
 * that basis vector is zero); then R Y = G (the leading k x k triangle, back
 * substitution) and X += V Y.  The iteration stops when the true residual
 * of every column passes.  iters counts block steps, cycles the restarts.
 *
 * The starting block of a cycle may be rank-deficient (a zero column, two
 * equal columns, a column that combines others).  Column c is dependent
 * when its part orthogonal to the columns kept before it has a norm of at
 * most 1e-6 of its own (the first Gram-Schmidt pass over R is then a
 * rank-revealing QR that keeps the columns in order).  With deflate = 0
 * that is a breakdown.  With deflate = 1 each dependent column c is
 * replaced by the vector z_c (z_c[i] = 2 u - 1, u = the top 53 bits of
 * output k = c 2^32 + i of SplitMix64 seeded with 0, over 2^53; see
 * splitmix64_out), the block with the replacements is orthonormalised
 * into V_1 as above, and S = V_1^T R, so that R = V_1 S holds for every
 * column up to the dependent columns' remainders (at most 1e-6 of them).
 * The block Krylov space then grows from the kept directions and the
 * replacements, and the block width stays s.  A zero rotation pivot is a
 * breakdown.
 */

/* Output k (counted from 0) of SplitMix64 seeded with 0 (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
 * the state after k + 1 steps of the Weyl sequence, then the mixing
 * function. */
static uint64_t splitmix64_out(uint64_t k) {
    uint64_t x = (k + 1u) * 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

/* The replacement vector z_c of a dependent column c (see or_block_gmres). */
static void replacement_vector(int n, int c, double *z) {
    for (int i = 0; i < n; i++) {
        const uint64_t k = ((uint64_t)c << 32) | (uint64_t)i;
        z[i] = 2.0 * ((double)(splitmix64_out(k) >> 11) * 0x1.0p-53) - 1.0;
    }
}

/* The replacement vector z_c, exported for its pin. */
void or_block_gmres_replacement(int n, int c, double *z) {
    if (n > 0 && c >= 0 && z) replacement_vector(n, c, z);
}

/* Two-pass modified Gram-Schmidt of the n x s block M (column-major, in
 * place) in column order, accumulating the coefficients into Gc (ld rows).
 * Column c counts as dependent when its norm after orthogonalisation is at
 * most tol times its norm before; it is then set to zero (a zero column
 * adds nothing to the later projections) and dead[c] = 1.  Returns the
 * number of dependent columns. */
static int mgs2_block(int n, int s, double *M, double *Gc, int ld, double tol, int *dead) {
    int ndead = 0;
    for (int c = 0; c < s; c++) {
        double *v = M + (long)c * n;
        const double before = nrm2(n, v);
        for (int pass2 = 0; pass2 < 2; pass2++)
            for (int q = 0; q < c; q++) {
                const double h = dot(n, M + (long)q * n, v);
                Gc[(long)c * ld + q] += h;
                for (int i = 0; i < n; i++) v[i] -= h * M[(long)q * n + i];
            }
        const double nv = nrm2(n, v);
        dead[c] = !(nv > tol * before);
        if (dead[c]) {
            ndead++;
            memset(v, 0, sizeof(double) * n);
            continue;
        }
        Gc[(long)c * ld + c] = nv;
        for (int i = 0; i < n; i++) v[i] /= nv;
    }
    return ndead;
}
int or_block_gmres(int n, int s, const double *A, long lda, const double *B, double *X, int m,
                   double rtol, int max_iter, int x0_given, int deflate, int nthreads,
                   int *iters_out, int *cycles_out, double *rel_res_out) {
    if (n < 0 || s < 1 || lda < n || m < 1 || max_iter < 0) return OR_ERR_ARG;
    const long ln = n ? n : 1;
    const int ld = (m + 1) * s, ncol = m * s;
    double *V = calloc((size_t)ln * ld, sizeof(double));
    double *H = calloc((size_t)ld * ncol, sizeof(double));
    double *G = calloc((size_t)ld * s, sizeof(double));
    double *Y = calloc((size_t)ncol * s, sizeof(double));
    double *cs = calloc((size_t)ncol * s, sizeof(double)), *sn = calloc((size_t)ncol * s, sizeof(double));
    int *rr = calloc((size_t)ncol * s, sizeof(int));
    double *bn = calloc(s, sizeof(double)), *w = malloc(sizeof(double) * ln);
    double *R0 = malloc(sizeof(double) * ln * s);
    int *dead = calloc(s, sizeof(int));
    int status = OR_NOT_CONVERGED, total = 0, cycles = 0;
#define HB(i, k) H[(long)(k) * ld + (i)]
#define GB(i, c) G[(long)(c) * ld + (i)]
    for (int c = 0; c < s; c++) bn[c] = nrm2(n, B + (long)c * n);
    if (!x0_given) memset(X, 0, sizeof(double) * ln * s);
    for (;;) {
        /* R = B - A X into the first s basis columns; every column passes? */
        int pass = 1;
        for (int c = 0; c < s; c++) {
            residual(n, A, lda, B + (long)c * n, X + (long)c * n, V + (long)c * n, nthreads);
            pass = pass && nrm2(n, V + (long)c * n) <= rtol * bn[c];
        }
        if (pass) { status = OR_OK; break; }
        if (total >= max_iter) break;
        cycles++;
        memset(H, 0, sizeof(double) * ld * ncol);
        memset(G, 0, sizeof(double) * ld * s);
        /* R = V_1 S; the first pass is the rank-revealing QR of R */
        memcpy(R0, V, sizeof(double) * n * s);
        if (mgs2_block(n, s, V, G, ld, deflate ? 1e-6 : 1e-14, dead)) {
            if (!deflate) { status = OR_BREAKDOWN; break; }
            memcpy(V, R0, sizeof(double) * n * s);
            for (int c = 0; c < s; c++)
                if (dead[c]) replacement_vector(n, c, V + (long)c * n);
            memset(G, 0, sizeof(double) * ld * s);
            if (mgs2_block(n, s, V, G, ld, 1e-14, dead)) { status = OR_BREAKDOWN; break; }
            memset(G, 0, sizeof(double) * ld * s);           /* S = V_1^T R */
            for (int c = 0; c < s; c++)
                for (int q = 0; q < s; q++) GB(q, c) = dot(n, V + (long)q * n, R0 + (long)c * n);
        }
        int k = 0, nrot = 0, stop = 0;
        for (int j = 0; j < m && total < max_iter && !stop; j++) {
            int lucky = 0;
            for (int c = 0; c < s; c++) {
                const int col = j * s + c, nb_idx = (j + 1) * s + c;   /* column of H, new basis vector */
                gemv(n, n, A, lda, V + (long)col * n, w, nthreads);     /* w = A v_col */
                const double before = nrm2(n, w);
                for (int pass2 = 0; pass2 < 2; pass2++)
                    for (int q = 0; q < nb_idx; q++) {
                        const double h = dot(n, V + (long)q * n, w);
                        HB(q, col) += h;
                        for (int i = 0; i < n; i++) w[i] -= h * V[(long)q * n + i];
                    }
                const double nw = nrm2(n, w);
                double *vn = V + (long)nb_idx * n;
                if (nw > 1e-14 * before) {
                    HB(nb_idx, col) = nw;
                    for (int i = 0; i < n; i++) vn[i] = w[i] / nw;
                } else {
                    HB(nb_idx, col) = 0.0;
                    memset(vn, 0, sizeof(double) * n);
                    lucky = 1;
                }
            }
            /* Givens: the block's s columns in order */
            for (int c = 0; c < s && !stop; c++) {
                const int col = j * s + c;
                for (int t = 0; t < nrot; t++) {
                    const int r = rr[t];
                    const double a = HB(r, col), b = HB(r + 1, col);
                    HB(r, col) = cs[t] * a + sn[t] * b;
                    HB(r + 1, col) = -sn[t] * a + cs[t] * b;
                }
                for (int r = col + s - 1; r >= col; r--) {      /* zero row r + 1 */
                    const double a = HB(r, col), b = HB(r + 1, col);
                    const double den = hypot(a, b);
                    const double cc = den > 0.0 ? a / den : 1.0, ss = den > 0.0 ? b / den : 0.0;
                    HB(r, col) = den > 0.0 ? den : a;
                    HB(r + 1, col) = 0.0;
                    for (int q = 0; q < s; q++) {
                        const double ga = GB(r, q), gb = GB(r + 1, q);
                        GB(r, q) = cc * ga + ss * gb;
                        GB(r + 1, q) = -ss * ga + cc * gb;
                    }
                    rr[nrot] = r; cs[nrot] = cc; sn[nrot] = ss; nrot++;
                }
                if (HB(col, col) == 0.0) { status = OR_BREAKDOWN; stop = 2; }
            }
            if (stop == 2) break;
            k = (j + 1) * s;
            total++;
            int conv = 1;
            for (int c = 0; c < s; c++) {
                double e2 = 0.0;
                for (int r = k; r < k + s; r++) e2 += GB(r, c) * GB(r, c);
                conv = conv && sqrt(e2) <= rtol * bn[c];
            }
            if (conv || lucky) stop = 1;
        }
        if (stop == 2) break;
        /* R Y = G on the leading k x k triangle, X += V Y */
        for (int c = 0; c < s; c++) {
            double *y = Y + (long)c * ncol;
            for (int i = k - 1; i >= 0; i--) {
                double v = GB(i, c);
                for (int q = i + 1; q < k; q++) v -= HB(i, q) * y[q];
                y[i] = v / HB(i, i);
            }
            for (int q = 0; q < k; q++)
                for (int i = 0; i < n; i++) X[(long)c * n + i] += V[(long)q * n + i] * y[q];
        }
    }
    double worst = 0.0;
    for (int c = 0; c < s; c++) {
        residual(n, A, lda, B + (long)c * n, X + (long)c * n, w, nthreads);
        const double r = bn[c] > 0.0 ? nrm2(n, w) / bn[c] : nrm2(n, w);
        if (!(r <= worst)) worst = r;
    }
    *rel_res_out = worst;
    *iters_out = total;
    *cycles_out = cycles;
    free(V); free(H); free(G); free(Y); free(cs); free(sn); free(rr); free(bn); free(w);
    free(R0); free(dead);
#undef HB
#undef GB
    return status;
}

/* ------------------------------------------------------------------ */
/* Gaussian elimination with partial pivoting (check solve, tiny n)    */
/* ------------------------------------------------------------------ */
/*
 * Right-looking LU with partial pivoting: at step k pick the row v >= k
 * with the largest |A(v,k)| (first one on ties), swap rows k and v (and the
 * right-hand side), divide the sub-column by the pivot and subtract the
 * rank-1 update from the trailing block.  Then L y = P b (unit lower,
 * forward) and U x = y (back).  Returns OR_BREAKDOWN on a zero pivot.
 */
/* The elimination on W (n x n, row-major) and y, in place; ipiv[k] = the
 * row swapped with row k (NULL: not recorded).  Returns OR_BREAKDOWN on a
 * zero pivot (W, y as far as the elimination got). */
static int ge_eliminate(int n, double *W, double *y, int *ipiv) {
    for (int k = 0; k < n; k++) {
        int v = k;
        double best = fabs(W[(long)k * n + k]);
        for (int i = k + 1; i < n; i++) {
            double a = fabs(W[(long)i * n + k]);
            if (a > best) { best = a; v = i; }
        }
        if (ipiv) ipiv[k] = v;
        if (v != k) {
            for (int j = 0; j < n; j++) {
                double t = W[(long)k * n + j];
                W[(long)k * n + j] = W[(long)v * n + j];
                W[(long)v * n + j] = t;
            }
            double t = y[k]; y[k] = y[v]; y[v] = t;
        }
        double piv = W[(long)k * n + k];
        if (piv == 0.0) return OR_BREAKDOWN;
        for (int i = k + 1; i < n; i++) {
            double l = W[(long)i * n + k] / piv;
            W[(long)i * n + k] = l;
            for (int j = k + 1; j < n; j++) W[(long)i * n + j] -= l * W[(long)k * n + j];
            y[i] -= l * y[k];                     /* forward substitution, fused */
        }
    }
    return OR_OK;
}

int or_ge_solve(int n, const double *A, long lda, const double *b, double *x) {
    if (n < 0 || lda < n) return OR_ERR_ARG;
    double *W = malloc(sizeof(double) * (size_t)(n ? n : 1) * (n ? n : 1));
    double *y = malloc(sizeof(double) * (n ? n : 1));
    for (int i = 0; i < n; i++) {
        memcpy(W + (long)i * n, A + (long)i * lda, sizeof(double) * n);
        y[i] = b[i];
    }
    int status = ge_eliminate(n, W, y, NULL);
    if (status == OR_OK) {
        for (int i = n - 1; i >= 0; i--) {        /* back substitution */
            double s = y[i];
            for (int j = i + 1; j < n; j++) s -= W[(long)i * n + j] * x[j];
            x[i] = s / W[(long)i * n + i];
        }
    }
    free(W); free(y);
    return status;
}

/* The factorization alone: LU (n x n, row-major: unit L below the diagonal,
 * U on and above it, rows in pivoted order), ipiv (the row swapped with row
 * k at step k) and y = L^-1 P b (the fused forward substitution). */
int or_ge_factor(int n, const double *A, long lda, const double *b, double *LU, int *ipiv, double *y) {
    if (n < 0 || lda < n) return OR_ERR_ARG;
    for (int i = 0; i < n; i++) {
        memcpy(LU + (long)i * n, A + (long)i * lda, sizeof(double) * n);
        y[i] = b[i];
    }
    return ge_eliminate(n, LU, y, ipiv);
}

/* ------------------------------------------------------------------ */
/* Cholesky factorization, FP64                                        */
/* ------------------------------------------------------------------ */
/*
 * The paper's Cholesky relations (A11 = L11 L11^T, L21 L11^T = A21,
 * A22 - L21 L21^T = L22 L22^T, L overwriting the lower triangle of A)
 * taken with a 1 x 1 leading block, i.e. right-looking by columns: at step
 * k, l_kk = sqrt(a_kk); l_ik = a_ik / l_kk for i > k; then
 * a_ij -= l_ik l_jk for k < j <= i (the lower triangle of the trailing
 * block).  Every element a_ij receives its updates for k = 0, 1, ... in
 * order, each as a rounded product and a rounded difference.  A pivot
 * a_kk <= 0 (or not a number) means A is not SPD: OR_BREAKDOWN, with L as
 * far as the factorization got.  L is n x n row-major, the strict upper
 * triangle set to zero.
 */
static int chol_columns(int n, double *W) {
    for (int k = 0; k < n; k++) {
        double akk = W[(long)k * n + k];
        if (!(akk > 0.0)) return OR_BREAKDOWN;
        double lkk = sqrt(akk);
        W[(long)k * n + k] = lkk;
        for (int i = k + 1; i < n; i++) W[(long)i * n + k] /= lkk;
        for (int i = k + 1; i < n; i++) {
            double lik = W[(long)i * n + k];
            for (int j = k + 1; j <= i; j++) W[(long)i * n + j] -= lik * W[(long)j * n + k];
        }
    }
    return OR_OK;
}

int or_chol_factor(int n, const double *A, long lda, double *L) {
    if (n < 0 || lda < n) return OR_ERR_ARG;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) L[(long)i * n + j] = j <= i ? A[(long)i * lda + j] : 0.0;
    return chol_columns(n, L);
}

/* L y = b by forward substitution (L n x n row-major, lower): y_i =
 * (b_i - sum_{j < i} l_ij y_j) / l_ii, the sum taken in increasing j. */
void or_chol_forward(int n, const double *L, const double *b, double *y) {
    for (int i = 0; i < n; i++) {
        double s = b[i];
        for (int j = 0; j < i; j++) s -= L[(long)i * n + j] * y[j];
        y[i] = s / L[(long)i * n + i];
    }
}

/* A x = b by the factorization, then L y = b (forward) and L^T x = y (back). */
int or_chol_solve(int n, const double *A, long lda, const double *b, double *x) {
    if (n < 0 || lda < n) return OR_ERR_ARG;
    double *L = malloc(sizeof(double) * (size_t)(n ? n : 1) * (n ? n : 1));
    int st = or_chol_factor(n, A, lda, L);
    if (st == OR_OK) {
        or_chol_forward(n, L, b, x);             /* y in x */
        for (int i = n - 1; i >= 0; i--) {       /* L^T x = y */
            double s = x[i];
            for (int j = i + 1; j < n; j++) s -= L[(long)j * n + i] * x[j];
            x[i] = s / L[(long)i * n + i];
        }
    }
    free(L);
    return st;
}

/* ------------------------------------------------------------------ */
/* Low-precision storage formats                                       */
/* ------------------------------------------------------------------ */
/*
 * Both roundings are written from the format definitions: the value is
 * scaled by its quantum (the spacing of the format at that magnitude),
 * rounded to the nearest integer with ties to even (rint under the
 * default rounding mode), and scaled back.
 *
 * BF16: 1 sign, 8 exponent (bias 127), 7 fraction bits; normal numbers
 * carry 8 significant bits, so the quantum at |d| in [2^e, 2^(e+1)) is
 * 2^(e-7); below 2^-126 the quantum is 2^-133.  Overflow goes to infinity.
 */
static double round_to_quantum(double d, double q) { return rint(d / q) * q; }

double or_bf16_round(double d) {
    if (isnan(d) || isinf(d) || d == 0.0) return d;
    int e;
    frexp(d, &e);                /* |d| in [2^(e-1), 2^e) */
    int ex = e - 1;
    double q = ex < -126 ? ldexp(1.0, -133) : ldexp(1.0, ex - 7);
    double v = round_to_quantum(d, q);
    const double maxv = ldexp(255.0, 120);           /* (2 - 2^-7) 2^127 */
    if (fabs(v) > maxv) return copysign(INFINITY, d);
    return v;
}

static uint16_t bf16_bits(double v) {
    if (isnan(v)) return 0x7FC0;
    float f = (float)v;                               /* exact: v is a BF16 value */
    uint32_t u;
    memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);
}

/*
 * FP8 E4M3 (the "fn" variant: no infinities, one NaN pattern per sign):
 * 1 sign, 4 exponent (bias 7), 3 fraction bits.  Normal numbers (>= 2^-6)
 * carry 4 significant bits, quantum 2^(e-3); subnormals have quantum 2^-9.
 * Largest finite value 448 = 1.75 * 2^8.  Saturating conversion: results
 * beyond 448 in magnitude become +-448.
 */
double or_e4m3_round(double d) {
    if (isnan(d)) return d;
    if (isinf(d)) return copysign(448.0, d);
    if (d == 0.0) return d;
    int e;
    frexp(d, &e);
    int ex = e - 1;
    double q = ex < -6 ? ldexp(1.0, -9) : ldexp(1.0, ex - 3);
    double v = round_to_quantum(d, q);
    if (fabs(v) > 448.0) v = copysign(448.0, d);
    return v;
}

static uint8_t e4m3_bits(double v) {
    if (isnan(v)) return 0x7F;
    uint8_t s = signbit(v) ? 0x80 : 0x00;
    double a = fabs(v);
    if (a == 0.0) return s;
    if (a < ldexp(1.0, -6)) return s | (uint8_t)(a / ldexp(1.0, -9));   /* subnormal */
    int e;
    double f = frexp(a, &e);                           /* a = f 2^e, f in [0.5,1) */
    int ex = e - 1;                                    /* a = (2f) 2^ex */
    int mant = (int)((2.0 * f - 1.0) * 8.0);
    return s | (uint8_t)((ex + 7) << 3) | (uint8_t)mant;
}

double or_e4m3_decode(uint8_t c) {
    int s = c >> 7, ex = (c >> 3) & 15, m = c & 7;
    if (ex == 15 && m == 7) return NAN;
    double v = ex == 0 ? ldexp((double)m, -9) : ldexp(1.0 + m / 8.0, ex - 7);
    return s ? -v : v;
}

double or_bf16_decode(uint16_t c) {
    uint32_t u = (uint32_t)c << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

/* Quantise a row-major n x n matrix to BF16 codes (row-major, ldq). */
int or_quant_bf16(int nrows, int ncols, const double *A, long lda,
                  uint16_t *Q, long ldq) {
    if (nrows < 0 || ncols < 0 || lda < ncols || ldq < ncols) return OR_ERR_ARG;
    for (int i = 0; i < nrows; i++)
        for (int j = 0; j < ncols; j++)
            Q[(long)i * ldq + j] = bf16_bits(or_bf16_round(A[(long)i * lda + j]));
    return OR_OK;
}

/*
 * Quantise to FP8-e4m3 with one FP32 scale per row:
 * s_i = fp32(max_j |a_ij| / 448) (1 when that is zero), and
 * q_ij = e4m3_sat(a_ij / s_i) with the division done in FP64.
 * The stored matrix represents s_i * q_ij.
 */
int or_quant_fp8(int nrows, int ncols, const double *A, long lda,
                 uint8_t *Q, long ldq, float *scale) {
    if (nrows < 0 || ncols < 0 || lda < ncols || ldq < ncols) return OR_ERR_ARG;
    for (int i = 0; i < nrows; i++) {
        const double *a = A + (long)i * lda;
        double mx = 0.0;
        for (int j = 0; j < ncols; j++) if (fabs(a[j]) > mx) mx = fabs(a[j]);
        float s = (float)(mx / 448.0);
        if (!(s > 0.0f)) s = 1.0f;          /* all-zero row, or scale underflow */
        scale[i] = s;
        for (int j = 0; j < ncols; j++)
            Q[(long)i * ldq + j] = e4m3_bits(or_e4m3_round(a[j] / (double)s));
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Mixed precision: FP32 inner CG on the stored matrix, FP64 outer      */
/* ------------------------------------------------------------------ */
/*
 * The stored matrix is given dequantised as FP32 values Af (row-major,
 * ldf) -- exact for BF16 codes -- plus an optional FP32 row scale: the
 * inner product is y_i = s_i * sum_j Af_ij p_j in FP32 arithmetic
 * (s = NULL means s_i = 1).  For FP8 storage Af holds the decoded e4m3
 * codes, exact in FP32.
 */
static void gemv_f32(int n, const float *Af, long ldf, const float *scale,
                     const float *p, float *y, int nthreads) {
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(static)
#else
    (void)nthreads;
#endif
    for (int i = 0; i < n; i++) {
        const float *a = Af + (long)i * ldf;
        float s = 0.0f;
        for (int j = 0; j < n; j++) s += a[j] * p[j];
        y[i] = scale ? scale[i] * s : s;
    }
}

static float dot_f32(int n, const float *x, const float *y) {
    float s = 0.0f;
    for (int i = 0; i < n; i++) s += x[i] * y[i];
    return s;
}

/*
 * Inner solve: z ~ Ahat^{-1} rhs by CG in FP32 from z = 0, for at most
 * `iters` iterations or until ||r|| <= inner_rtol ||rhs|| (inner_rtol <= 0
 * disables the tolerance test).  A non-positive curvature stops the inner
 * loop (z keeps its last value; if that is the first iteration z = rhs).
 * Returns the number of iterations done.
 */
int or_cg_f32(int n, const float *Af, long ldf, const float *scale,
              const float *rhs, float *z, int iters, float inner_rtol,
              int nthreads) {
    float *r = malloc(sizeof(float) * (n ? n : 1));
    float *p = malloc(sizeof(float) * (n ? n : 1));
    float *q = malloc(sizeof(float) * (n ? n : 1));
    for (int i = 0; i < n; i++) { z[i] = 0.0f; r[i] = rhs[i]; p[i] = rhs[i]; }
    float rho = dot_f32(n, r, r);
    float stop = inner_rtol > 0.0f ? inner_rtol * inner_rtol * rho : -1.0f;
    int k = 0;
    for (; k < iters; k++) {
        if (rho <= stop || rho == 0.0f) break;
        gemv_f32(n, Af, ldf, scale, p, q, nthreads);
        float pq = dot_f32(n, p, q);
        if (!(pq > 0.0f)) {
            if (k == 0) for (int i = 0; i < n; i++) z[i] = rhs[i];
            break;
        }
        float alpha = rho / pq;
        for (int i = 0; i < n; i++) z[i] += alpha * p[i];
        for (int i = 0; i < n; i++) r[i] -= alpha * q[i];
        float rho_new = dot_f32(n, r, r);
        float beta = rho_new / rho;
        for (int i = 0; i < n; i++) p[i] = r[i] + beta * p[i];
        rho = rho_new;
    }
    free(r); free(p); free(q);
    return k;
}

/*
 * Outer FP64 loop driven by the FP64 residual.
 *   mode 0 (flexible CG, Notay 2000): z_k = ||r|| * inner(r / ||r||);
 *     p_k = z_k - sum_{j<k} (z_k . w_j / p_j . w_j) p_j with w_j = A p_j
 *     (FP64), alpha = (p_k . r) / (p_k . w_k), x += alpha p_k,
 *     r -= alpha w_k.  Every stored direction is kept (full
 *     A-orthogonalisation).
 *   mode 1 (classic refinement): r = b - A x (FP64), x += ||r|| inner(r/||r||).
 * Stops when ||r|| <= rtol ||b||, confirmed on the true residual (the
 * recursive FCG residual is replaced by the true one when it is not).
 * outer_out counts outer steps, inner_out the inner CG iterations.
 * P_out (optional, n x max_outer column-major) receives the FCG directions.
 */
int or_mixed_cg(int n, const double *A, long lda, const float *Af, long ldf,
                const float *scale, const double *b, double *x, double rtol,
                int max_outer, int inner_iters, double inner_rtol, int mode,
                int nthreads, int *outer_out, int *inner_out,
                double *rel_res_out, double *res_hist, double *P_out) {
    if (n < 0 || lda < n || ldf < n || max_outer < 0) return OR_ERR_ARG;
    long ln = n ? n : 1;
    double *r = malloc(sizeof(double) * ln), *z = malloc(sizeof(double) * ln);
    double *P = malloc(sizeof(double) * ln * (max_outer + 1));
    double *W = malloc(sizeof(double) * ln * (max_outer + 1));
    double *pw = malloc(sizeof(double) * (max_outer + 1));
    float *rf = malloc(sizeof(float) * ln), *zf = malloc(sizeof(float) * ln);
    int status = OR_NOT_CONVERGED, outer = 0, inner = 0, nstored = 0;
    double nb = nrm2(n, b);
    for (int i = 0; i < n; i++) x[i] = 0.0;
    if (nb == 0.0) {
        *outer_out = 0; *inner_out = 0; *rel_res_out = 0.0;
        status = OR_OK;
        goto done;
    }
    for (int i = 0; i < n; i++) r[i] = b[i];
    int recursive = 0;          /* r is a recursively updated residual */
    for (;;) {
        double rn = nrm2(n, r);
        if (res_hist) res_hist[outer] = rn / nb;
        if (rn <= rtol * nb) {
            if (!recursive) { status = OR_OK; break; }
            residual(n, A, lda, b, x, r, nthreads);   /* confirm */
            recursive = 0;
            continue;
        }
        if (!(rn == rn)) { status = OR_BREAKDOWN; break; }
        if (outer >= max_outer) break;
        for (int i = 0; i < n; i++) rf[i] = (float)(r[i] / rn);
        inner += or_cg_f32(n, Af, ldf, scale, rf, zf, inner_iters,
                           (float)inner_rtol, nthreads);
        for (int i = 0; i < n; i++) z[i] = rn * (double)zf[i];
        outer++;
        if (mode == 1) {
            for (int i = 0; i < n; i++) x[i] += z[i];
            residual(n, A, lda, b, x, r, nthreads);
            continue;
        }
        double *p = P + (long)nstored * n, *w = W + (long)nstored * n;
        memcpy(p, z, sizeof(double) * n);
        for (int j = 0; j < nstored; j++) {
            double c = dot(n, z, W + (long)j * n) / pw[j];
            for (int i = 0; i < n; i++) p[i] -= c * P[(long)j * n + i];
        }
        gemv(n, n, A, lda, p, w, nthreads);
        double d = dot(n, p, w);
        if (!(d > 0.0)) { status = OR_BREAKDOWN; break; }
        double alpha = dot(n, p, r) / d;
        for (int i = 0; i < n; i++) x[i] += alpha * p[i];
        for (int i = 0; i < n; i++) r[i] -= alpha * w[i];
        pw[nstored++] = d;
        recursive = 1;
    }
    residual(n, A, lda, b, x, r, nthreads);
    *rel_res_out = nrm2(n, r) / nb;
    *outer_out = outer;
    *inner_out = inner;
    if (P_out) memcpy(P_out, P, sizeof(double) * n * nstored);
done:
    free(r); free(z); free(P); free(W); free(pw); free(rf); free(zf);
    return status;
}

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
