// k_bcg.cu -- block conjugate gradient for s right-hand sides: O'Leary's form
// and a deflating form with orthonormal, rank-revealed search directions (the
// second half of this file).
//
// Block CG (the paper's CG paragraph, for several right-hand sides at once
// in O'Leary's block form) replaces CG's scalars by s x s matrices:
//   Q = A P;  gamma = P^T Q;  alpha = gamma^-1 rho;  X += P alpha;
//   R -= Q alpha;  rho' = R^T R;  beta = rho^-1 rho';  P = R + P beta.
// The products Q = A P are s launches of the solvers' GEMV (one per column,
// each streaming A once as the FP32 pair); everything else of a step is
// one cooperative kernel:
//   bcg_step   gamma (per-CTA partial Gram matrices over row ranges, reduced
//              in CTA order), one warp factors gamma (Cholesky) and solves
//              for alpha; every CTA updates its rows of X and R and forms
//              its partial R^T R; one warp tests every column, factors rho'
//              and solves for beta; every CTA forms P = R + P beta row by
//              row.  Three bounded grid barriers.
//   bcg_init   X = 0 (or keep X0, R from the residual GEMVs), P = R,
//              rho = R^T R and its factor, ||B_j||, the loop conditions.
//   bcg_check  after the loop: accept when every column's true residual
//              passes, or restart from it (P = R, rho = R^T R).
// The s x s algebra is FP64 on one warp (s <= 16): Cholesky column by column
// with the lanes over rows, triangular solves with the lanes over right-hand
// sides.  A factor that meets a non-positive pivot (a rank-deficient block)
// is a breakdown.  Blocks are column-major n x s with column stride ld.
#include <cuda_runtime.h>

#include "ls_device.cuh"
#include "ls_internal.h"

namespace lsi {

constexpr int BK = 256;   // threads per CTA

// ---- one warp: s x s Cholesky and solves (column-major, shared memory) ------------
// G = L L^T in place (L in the lower triangle); false on a non-positive pivot.
__device__ bool warp_chol(int s, double *G) {
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < s; j++) {
        double d = G[j + j * s];
        for (int k = 0; k < j; k++) d -= G[j + k * s] * G[j + k * s];
        if (!(d > 0.0)) return false;          // same value in every lane
        d = sqrt(d);
        __syncwarp();
        if (lane > j && lane < s) {
            double v = G[lane + j * s];
            for (int k = 0; k < j; k++) v -= G[lane + k * s] * G[j + k * s];
            G[lane + j * s] = v / d;
        }
        if (lane == 0) G[j + j * s] = d;
        __syncwarp();
    }
    return true;
}

// Y = (L L^T)^-1 Y, one right-hand side per lane.
__device__ void warp_chol_solve(int s, const double *L, double *Y) {
    const int c = threadIdx.x & 31;
    if (c < s) {
        double *y = Y + c * s;
        for (int i = 0; i < s; i++) {
            double v = y[i];
            for (int k = 0; k < i; k++) v -= L[i + k * s] * y[k];
            y[i] = v / L[i + i * s];
        }
        for (int i = s - 1; i >= 0; i--) {
            double v = y[i];
            for (int k = i + 1; k < s; k++) v -= L[k + i * s] * y[k];
            y[i] = v / L[i + i * s];
        }
    }
    __syncwarp();
}

// ---- Gram matrices -------------------------------------------------------------------
// This CTA's partial U^T V over rows [lo, hi) into part[cta][s*s]: T =
// BK / s^2 threads per entry, thread q summing rows lo + q, lo + q + T, ...,
// the T sums added in q order (all threads of the CTA call it).
__device__ __forceinline__ void gram_partial(const BcgVecs &v, const double *U, const double *V, long long lo,
                                             long long hi) {
    __shared__ double red[BK];
    const int s = v.s, E = s * s, T = BK / E;
    const int e = threadIdx.x / T, q = threadIdx.x - e * T;
    double acc = 0.0;
    if (e < E) {
        const int a = e % s, b = e / s;
        const double *u = U + (long long)a * v.ld, *w = V + (long long)b * v.ld;
        for (long long i = lo + q; i < hi; i += T) acc += u[i] * w[i];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    if (e < E && q == 0) {
        double sum = 0.0;
        for (int t = 0; t < T; t++) sum += red[threadIdx.x + t];
        v.part[(size_t)blockIdx.x * BCG_MAX_S * BCG_MAX_S + e] = sum;
    }
    __syncthreads();
}

// One warp: G = sum of the partials, entry by entry, as eight interleaved
// sums over the CTAs added pairwise (a fixed order).
__device__ __forceinline__ void gram_reduce(const BcgVecs &v, double *G) {
    const int s = v.s, nc = (int)gridDim.x;
    for (int e = threadIdx.x & 31; e < s * s; e += 32) {
        double t[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int c = 0; c < nc; c++) t[c & 7] += __ldcg(&v.part[(size_t)c * BCG_MAX_S * BCG_MAX_S + e]);
        G[e] = ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
    }
    __syncwarp();
}

__device__ __forceinline__ bool all_pass(const BcgVecs &v, const double *rho) {
    bool ok = true;
    for (int j = 0; j < v.s; j++) ok = ok && sqrt(rho[j + j * v.s]) <= v.rtol * v.sm->bn[j];
    return ok;
}

// ---- init ----------------------------------------------------------------------------
__global__ void __launch_bounds__(BK) bcg_init_kernel(BcgVecs v, int x0_given, cudaGraphConditionalHandle h_outer,
                                                      cudaGraphConditionalHandle h_inner) {
    __shared__ double G[BCG_MAX_S * BCG_MAX_S];
    State *st = v.st;
    BcgSmall *sm = v.sm;
    count_launch(st);
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    for (int j = 0; j < v.s; j++)
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const long long o = (long long)j * v.ld + i;
            if (!x0_given) {
                v.X[o] = 0.0;
                v.R[o] = v.B[o];
            }
            v.P[o] = v.R[o];
        }
    __syncthreads();
    gram_partial(v, v.R, v.R, lo, hi);
    // partial ||B_j||^2
    for (int j = threadIdx.x; j < v.s; j += blockDim.x) {
        const double *b = v.B + (long long)j * v.ld;
        double acc = 0.0;
        for (long long i = lo; i < hi; i++) acc += b[i] * b[i];
        v.part2[(size_t)blockIdx.x * BCG_MAX_S + j] = acc;
    }
    if (!grid_sync(v.bar, st)) return;
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        gram_reduce(v, G);
        const int lane = threadIdx.x;
        if (lane < v.s) {
            double acc = 0.0;
            for (int c = 0; c < (int)gridDim.x; c++) acc += __ldcg(&v.part2[(size_t)c * BCG_MAX_S + lane]);
            sm->bn[lane] = sqrt(acc);
        }
        __syncwarp();
        for (int e = lane; e < v.s * v.s; e += 32) sm->rho[e] = G[e];
        bool nan = false;
        for (int e = 0; e < v.s * v.s; e++) nan = nan || !isfinite(G[e]);
        for (int j = 0; j < v.s; j++) nan = nan || !isfinite(sm->bn[j]);
        const bool pass = !nan && all_pass(v, G);
        bool factored = false;
        if (!nan && !pass) factored = warp_chol(v.s, G);
        for (int e = lane; e < v.s * v.s; e += 32) sm->L[e] = G[e];
        if (lane == 0) {
            int go = 1;
            if (nan) {
                set_err(st, ERRB_NAN);
                go = 0;
            } else if (pass) {
                go = 0;                               // confirm on the true residual
            } else if (!factored) {
                st->status = LS_BREAKDOWN;            // rank-deficient residual block
                go = 0;
            } else if (st->max_iter <= 0) {
                go = 0;
            }
            set_cond(st, h_inner, go);
            set_cond(st, h_outer, 1u);
        }
    }
}

// ---- one step after Q = A P ---------------------------------------------------------------
__global__ void __launch_bounds__(BK) bcg_step_kernel(BcgVecs v, cudaGraphConditionalHandle h_inner) {
    __shared__ double G[BCG_MAX_S * BCG_MAX_S], Y[BCG_MAX_S * BCG_MAX_S];
    __shared__ double coef[BCG_MAX_S * BCG_MAX_S];
    __shared__ int flag_s;
    State *st = v.st;
    BcgSmall *sm = v.sm;
    count_launch(st);
    const int s = v.s;
    if (*(volatile int *)&st->err || *(volatile int *)&st->status == LS_BREAKDOWN) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(st, h_inner, 0u);
        return;
    }
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    // gamma = P^T Q
    gram_partial(v, v.P, v.Q, lo, hi);
    if (!grid_sync(v.bar, st)) return;
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        gram_reduce(v, G);
        const bool ok = warp_chol(s, G);
        if (ok) {
            for (int e = threadIdx.x; e < s * s; e += 32) Y[e] = sm->rho[e];
            __syncwarp();
            warp_chol_solve(s, G, Y);                    // alpha = gamma^-1 rho
            for (int e = threadIdx.x; e < s * s; e += 32) sm->alpha[e] = Y[e];
        }
        if (threadIdx.x == 0) {
            sm->ok = ok ? 1 : 0;
            if (!ok) st->status = LS_BREAKDOWN;
        }
    }
    if (!grid_sync(v.bar, st)) return;
    if (threadIdx.x == 0) flag_s = *(volatile int *)&sm->ok;
    __syncthreads();
    if (!flag_s) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(st, h_inner, 0u);
        return;
    }
    // X += P alpha, R -= Q alpha (row by row, all s columns), partial R^T R
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) coef[e] = __ldcg(&sm->alpha[e]);
    __syncthreads();
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        double p[BCG_MAX_S], q[BCG_MAX_S];
#pragma unroll
        for (int c = 0; c < BCG_MAX_S; c++) {
            p[c] = c < s ? v.P[(long long)c * v.ld + i] : 0.0;
            q[c] = c < s ? v.Q[(long long)c * v.ld + i] : 0.0;
        }
        for (int j = 0; j < s; j++) {
            double dx = 0.0, dr = 0.0;
#pragma unroll
            for (int c = 0; c < BCG_MAX_S; c++)
                if (c < s) {
                    dx += p[c] * coef[c + j * s];
                    dr += q[c] * coef[c + j * s];
                }
            v.X[(long long)j * v.ld + i] += dx;
            v.R[(long long)j * v.ld + i] -= dr;
        }
    }
    __syncthreads();
    gram_partial(v, v.R, v.R, lo, hi);
    if (!grid_sync(v.bar, st)) return;
    // rho' = R^T R: stop test, or beta = rho^-1 rho' and the factor of rho'
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        gram_reduce(v, G);                                // rho'
        bool nan = false;
        for (int e = 0; e < s * s; e++) nan = nan || !isfinite(G[e]);
        const bool pass = !nan && all_pass(v, G);
        int go = 0;
        if (!nan && !pass) {
            for (int e = threadIdx.x; e < s * s; e += 32) Y[e] = G[e];
            for (int e = threadIdx.x; e < s * s; e += 32) coef[e] = sm->L[e];
            __syncwarp();
            warp_chol_solve(s, coef, Y);                  // beta = rho^-1 rho'
            for (int e = threadIdx.x; e < s * s; e += 32) sm->beta[e] = Y[e];
            for (int e = threadIdx.x; e < s * s; e += 32) sm->rho[e] = G[e];
            __syncwarp();
            const bool ok = warp_chol(s, G);              // factor of rho' for the next step
            for (int e = threadIdx.x; e < s * s; e += 32) sm->L[e] = G[e];
            go = ok ? 1 : 0;
            if (threadIdx.x == 0 && !ok) st->status = LS_BREAKDOWN;
        } else {
            for (int e = threadIdx.x; e < s * s; e += 32) sm->rho[e] = G[e];
        }
        if (threadIdx.x == 0) {
            st->iter++;
            if (nan) set_err(st, ERRB_NAN);
            if (go && st->iter >= st->max_iter) go = 0;
            sm->ok = go;
            sm->update_p = (!nan && !pass && *(volatile int *)&st->status != LS_BREAKDOWN) ? 1 : 0;
            set_cond(st, h_inner, go ? 1u : 0u);
        }
    }
    if (!grid_sync(v.bar, st)) return;
    if (threadIdx.x == 0) flag_s = *(volatile int *)&sm->update_p;
    __syncthreads();
    if (!flag_s) return;
    // P = R + P beta (row by row)
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) coef[e] = __ldcg(&sm->beta[e]);
    __syncthreads();
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        double p[BCG_MAX_S];
#pragma unroll
        for (int c = 0; c < BCG_MAX_S; c++) p[c] = c < s ? v.P[(long long)c * v.ld + i] : 0.0;
        for (int j = 0; j < s; j++) {
            double acc = v.R[(long long)j * v.ld + i];
#pragma unroll
            for (int c = 0; c < BCG_MAX_S; c++)
                if (c < s) acc += p[c] * coef[c + j * s];
            v.P[(long long)j * v.ld + i] = acc;
        }
    }
}

// ---- after the loop: the true residual R = B - A X (written by the residual
// GEMVs, with ||R_j||^2 in sm->r2) -----------------------------------------------------------
__global__ void __launch_bounds__(BK) bcg_check_kernel(BcgVecs v, cudaGraphConditionalHandle h_outer,
                                                       cudaGraphConditionalHandle h_inner) {
    __shared__ double G[BCG_MAX_S * BCG_MAX_S];
    __shared__ int restart_s;
    State *st = v.st;
    BcgSmall *sm = v.sm;
    count_launch(st);
    const int s = v.s;
    if (threadIdx.x == 0) {
        bool pass = true, nan = false;
        for (int j = 0; j < s; j++) {
            const double r2 = *(volatile double *)&sm->r2[j];
            nan = nan || !isfinite(r2);
            pass = pass && sqrt(r2) <= v.rtol * sm->bn[j];
        }
        int restart = 0;
        if (*(volatile int *)&st->err || nan) {
            if (nan) set_err(st, ERRB_NAN);
        } else if (*(volatile int *)&st->status == LS_BREAKDOWN) {
            // a factor failed: stop with the last iterate
        } else if (pass) {
            if (blockIdx.x == 0) st->status = LS_OK;
        } else if (*(volatile int *)&st->iter >= st->max_iter) {
            if (blockIdx.x == 0) st->status = LS_NOT_CONVERGED;
        } else {
            restart = 1;
        }
        restart_s = restart;
    }
    __syncthreads();
    if (!restart_s) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            set_cond(st, h_outer, 0u);
            set_cond(st, h_inner, 0u);
        }
        return;
    }
    // restart from the true residual: P = R, rho = R^T R and its factor
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    for (int j = 0; j < s; j++)
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x)
            v.P[(long long)j * v.ld + i] = v.R[(long long)j * v.ld + i];
    __syncthreads();
    gram_partial(v, v.R, v.R, lo, hi);
    if (!grid_sync(v.bar, st)) return;
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        gram_reduce(v, G);
        for (int e = threadIdx.x; e < s * s; e += 32) sm->rho[e] = G[e];
        __syncwarp();
        const bool ok = warp_chol(s, G);
        for (int e = threadIdx.x; e < s * s; e += 32) sm->L[e] = G[e];
        if (threadIdx.x == 0) {
            if (!ok) st->status = LS_BREAKDOWN;
            st->cycles++;
            set_cond(st, h_inner, ok ? 1u : 0u);
            set_cond(st, h_outer, 1u);
        }
    }
}

// ============================================================================
// The deflating form: the search directions P are kept orthonormal and of
// full rank r <= s by a rank-revealing orthogonalization, dependent ones
// dropped, so dependent, zero or converged residual columns never make a
// step matrix singular (block CG with orthonormalized directions, as in the
// breakdown-free block CG of Ji and Li):
//   Q = A P;  gamma = P^T Q (r x r);  alpha = gamma^-1 (P^T R);
//   X += P alpha;  R -= Q alpha;  per-column stop test;
//   beta = -gamma^-1 (Q^T R);  P = orth(R + P beta).
// The new directions are A-conjugate to P and span the same block Krylov
// space as O'Leary's, so with a full-rank block the iterates are the same.
// orth(W): W^T W, columns normalized to unit norm, Cholesky with diagonal
// pivoting (largest remaining diagonal first) that stops when the remaining
// diagonal is at most tau^2 = 1e-16 (the column's part outside the span of
// the taken ones is at most 1e-8 of its norm: dependent), then P = W T with
// T = D^-1 Pi L^-T, and a second pass (Gram of P, Cholesky, P = P L2^-T).
// Small matrices use leading dimension BCG_MAX_S; the s x s algebra (at most
// 16 x 16) runs on one thread.
// ============================================================================
constexpr int SL = BCG_MAX_S;              // leading dimension of the small matrices
constexpr double BCGD_TAU2 = 1e-16;        // (1e-8)^2 on the normalized diagonal

// This CTA's partial U[:, :nu]^T V[:, :nv] over rows [lo, hi) into
// buf[cta][SL*SL].  Every thread of the CTA takes part: T = BK / (nu nv)
// threads per entry, thread q of an entry summing rows lo + q, lo + q + T,
// ...; the T sums added in q order (a fixed order, so the result does not
// depend on timing).  A warp's FP64 instruction takes about 64 cycles of
// its scheduler's FP64 unit on this GPU, so shorter chains spread over all
// warps (and all four schedulers) are what counts.
__device__ __forceinline__ void gram_partial_ld(const BcgVecs &v, double *buf, const double *U, int nu,
                                                const double *V, int nv, long long lo, long long hi) {
    __shared__ double red[BK];
    const int E = nu * nv;
    if (E == 0) return;
    const int T = BK / E;
    const int e = threadIdx.x / T, q = threadIdx.x - e * T;
    double acc = 0.0;
    if (e < E) {
        const int a = e % nu, b = e / nu;
        const double *u = U + (long long)a * v.ld, *w = V + (long long)b * v.ld;
        for (long long i = lo + q; i < hi; i += T) acc += u[i] * w[i];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    if (e < E && q == 0) {
        double sum = 0.0;
        for (int t = 0; t < T; t++) sum += red[threadIdx.x + t];
        const int a = e % nu, b = e / nu;
        buf[(size_t)blockIdx.x * SL * SL + a + b * SL] = sum;
    }
    __syncthreads();
}
// G = the sum of the CTAs' partials, entry by entry, by all threads of the
// calling CTA: eight interleaved sums over the CTAs (CTA c into sum c % 8),
// added pairwise; a fixed order.
__device__ __forceinline__ void gram_reduce_ld(const double *buf, int nu, int nv, double *G) {
    const int nc = (int)gridDim.x;
    for (int e = threadIdx.x; e < nu * nv; e += blockDim.x) {
        const int a = e % nu, b = e / nu;
        const double *p = buf + a + b * SL;
        double t[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        int c = 0;
        for (; c + 8 <= nc; c += 8)
#pragma unroll
            for (int u = 0; u < 8; u++) t[u] += __ldcg(p + (size_t)(c + u) * SL * SL);
        for (int u = 0; c + u < nc; u++) t[u] += __ldcg(p + (size_t)(c + u) * SL * SL);
        G[a + b * SL] = ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
    }
}

// Cholesky of the leading r x r block (lower triangle, leading dimension SL);
// false on a pivot that is not positive.
__device__ bool small_chol(int r, double *G) {
    for (int j = 0; j < r; j++) {
        double d = G[j + j * SL];
        for (int k = 0; k < j; k++) d -= G[j + k * SL] * G[j + k * SL];
        if (!(d > 0.0)) return false;
        d = sqrt(d);
        G[j + j * SL] = d;
        const double dinv = 1.0 / d;   // one division per column (FP64 division is slow here)
        for (int i = j + 1; i < r; i++) {
            double x = G[i + j * SL];
            for (int k = 0; k < j; k++) x -= G[i + k * SL] * G[j + k * SL];
            G[i + j * SL] = x * dinv;
        }
    }
    return true;
}
// Y (r x c) = (L L^T)^-1 Y, column j of Y by thread j of the calling CTA
// (all threads call it), with the reciprocals of L's diagonal formed once.
__device__ void small_chol_solve(int r, int c, const double *L, double *Y) {
    __shared__ double dinv[SL];
    if (threadIdx.x < r) dinv[threadIdx.x] = 1.0 / L[threadIdx.x + threadIdx.x * SL];
    __syncthreads();
    for (int j = threadIdx.x; j < c; j += blockDim.x) {
        double *y = Y + j * SL;
        for (int i = 0; i < r; i++) {
            double x = y[i];
            for (int k = 0; k < i; k++) x -= L[i + k * SL] * y[k];
            y[i] = x * dinv[i];
        }
        for (int i = r - 1; i >= 0; i--) {
            double x = y[i];
            for (int k = i + 1; k < r; k++) x -= L[k + i * SL] * y[k];
            y[i] = x * dinv[i];
        }
    }
    __syncthreads();
}
// M = L^-T (upper triangular, r x r) for a lower-triangular L.
__device__ void small_inv_t(int r, const double *L, double *M) {
    for (int b = 0; b < SL; b++)
        for (int a = 0; a < SL; a++) M[a + b * SL] = 0.0;
    double dinv[SL];
    for (int a = 0; a < r; a++) dinv[a] = 1.0 / L[a + a * SL];
    for (int b = 0; b < r; b++) {                  // column b of M solves L^T m = e_b
        for (int a = r - 1; a >= 0; a--) {
            double x = a == b ? 1.0 : 0.0;
            for (int k = a + 1; k < r; k++) x -= L[k + a * SL] * M[k + b * SL];
            M[a + b * SL] = x * dinv[a];
        }
    }
}

// First pass of orth: from G = W^T W (s x s) the rank r and T (s x s) with
// W T = the r orthonormal-to-first-order columns (then zero columns).
// work: 3 SL^2 + 2 SL doubles, iwork: 2 SL ints (shared memory of the caller).
__device__ int rr_factor(int s, const double *G, double *T, double *work, int *iwork) {
    double *Lp = work, *M = work + SL * SL, *Lcm = work + 2 * SL * SL;
    double *d = work + 3 * SL * SL, *rem = d + SL;
    int *perm = iwork, *state = iwork + SL;
#define Lc(q, t) Lcm[(q) + (t) * SL]
    double dinv[SL];
    for (int j = 0; j < s; j++) {
        d[j] = sqrt(G[j + j * SL]);
        dinv[j] = 1.0 / d[j];
        state[j] = d[j] > 0.0 ? 0 : 2;             // 0 open, 1 taken, 2 dropped
        rem[j] = 1.0;
    }
    int r = 0;
    for (;;) {
        int p = -1;
        for (int j = 0; j < s; j++) {
            if (state[j]) continue;
            if (!(rem[j] > BCGD_TAU2)) { state[j] = 2; continue; }
            if (p < 0 || rem[j] > rem[p]) p = j;
        }
        if (p < 0) break;
        const double lpp = sqrt(rem[p]), linv = 1.0 / lpp;
        perm[r] = p;
        state[p] = 1;
        Lc(p, r) = lpp;
        for (int q = 0; q < s; q++) {
            if (state[q]) continue;
            double x = G[q + p * SL] * dinv[q] * dinv[p];
            for (int t = 0; t < r; t++) x -= Lc(q, t) * Lc(p, t);
            Lc(q, r) = x * linv;
            rem[q] -= Lc(q, r) * Lc(q, r);
        }
        r++;
    }
    for (int b = 0; b < SL; b++)
        for (int a = 0; a < SL; a++) Lp[a + b * SL] = 0.0;
    for (int a = 0; a < r; a++)
        for (int t = 0; t <= a; t++) Lp[a + t * SL] = Lc(perm[a], t);
    small_inv_t(r, Lp, M);
    for (int e = 0; e < SL * SL; e++) T[e] = 0.0;
    for (int a = 0; a < r; a++)
        for (int b = 0; b < r; b++) T[perm[a] + b * SL] = M[a + b * SL] * dinv[perm[a]];
#undef Lc
    return r;
}

// P = orth(W) over the whole grid (cooperative launch; W and P must differ).
// On return sm->rank holds r and sm->w2 the squared column norms of W.
// false if a grid barrier gave up or the second pass failed.
__device__ bool coop_orth(const BcgVecs &v, const double *W, long long lo, long long hi) {
    __shared__ double G[SL * SL], T[SL * SL], work[3 * SL * SL + 2 * SL];
    __shared__ int r_s, iwork[2 * SL];
    BcgSmall *sm = v.sm;
    const int s = v.s;
    gram_partial_ld(v, v.part, W, s, W, s, lo, hi);
    if (!grid_sync(v.bar, v.st)) return false;
    if (blockIdx.x == 0) {
        gram_reduce_ld(v.part, s, s, G);
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int j = 0; j < s; j++) sm->w2[j] = G[j + j * SL];
            bool nan = false;
            for (int j = 0; j < s; j++) nan = nan || !isfinite(G[j + j * SL]);
            const int r = nan ? 0 : rr_factor(s, G, T, work, iwork);
            for (int e = 0; e < SL * SL; e++) sm->T[e] = T[e];
            sm->rank = r;
        }
    }
    if (!grid_sync(v.bar, v.st)) return false;
    if (threadIdx.x == 0) r_s = *(volatile int *)&sm->rank;
    for (int e = threadIdx.x; e < SL * SL; e += blockDim.x) T[e] = __ldcg(&sm->T[e]);
    __syncthreads();
    const int r = r_s;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {     // P = W T
        double w[BCG_MAX_S];
#pragma unroll
        for (int c = 0; c < BCG_MAX_S; c++) w[c] = c < s ? W[(long long)c * v.ld + i] : 0.0;
        for (int b = 0; b < s; b++) {
            double acc = 0.0;
#pragma unroll
            for (int c = 0; c < BCG_MAX_S; c++)
                if (c < s) acc += w[c] * T[c + b * SL];
            v.P[(long long)b * v.ld + i] = acc;
        }
    }
    __syncthreads();
    gram_partial_ld(v, v.part, v.P, r, v.P, r, lo, hi);                 // second pass
    if (!grid_sync(v.bar, v.st)) return false;
    if (blockIdx.x == 0) {
        gram_reduce_ld(v.part, r, r, G);
        __syncthreads();
        if (threadIdx.x == 0) {
            const bool ok = small_chol(r, G);
            if (ok) small_inv_t(r, G, T);
            for (int e = 0; e < SL * SL; e++) sm->T[e] = ok ? T[e] : 0.0;
            if (!ok) sm->rank = -1;
        }
    }
    if (!grid_sync(v.bar, v.st)) return false;
    for (int e = threadIdx.x; e < SL * SL; e += blockDim.x) T[e] = __ldcg(&sm->T[e]);
    if (threadIdx.x == 0) r_s = *(volatile int *)&sm->rank;
    __syncthreads();
    if (r_s < 0) return false;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {     // P = P L2^-T (upper triangular)
        double p[BCG_MAX_S];
#pragma unroll
        for (int c = 0; c < BCG_MAX_S; c++) p[c] = c < r ? v.P[(long long)c * v.ld + i] : 0.0;
        for (int b = 0; b < r; b++) {
            double acc = 0.0;
#pragma unroll
            for (int c = 0; c < BCG_MAX_S; c++)
                if (c <= b) acc += p[c] * T[c + b * SL];
            v.P[(long long)b * v.ld + i] = acc;
        }
    }
    __syncthreads();
    return true;
}

// Every column's ||R_j|| <= rtol ||B_j|| (r2 = the squared norms).
__device__ __forceinline__ bool cols_pass(const BcgVecs &v, const double *r2) {
    bool ok = true;
    for (int j = 0; j < v.s; j++) ok = ok && sqrt(r2[j]) <= v.rtol * v.sm->bn[j];
    return ok;
}

// X = 0 and R = B (or R from the residual GEMVs), ||B_j||, P = orth(R), the
// loop conditions.
__global__ void __launch_bounds__(BK) bcgd_init_kernel(BcgVecs v, int x0_given, cudaGraphConditionalHandle h_outer,
                                                       cudaGraphConditionalHandle h_inner) {
    State *st = v.st;
    BcgSmall *sm = v.sm;
    count_launch(st);
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    for (int j = 0; j < v.s; j++)
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const long long o = (long long)j * v.ld + i;
            if (!x0_given) {
                v.X[o] = 0.0;
                v.R[o] = v.B[o];
            }
        }
    for (int j = threadIdx.x; j < v.s; j += blockDim.x) {
        const double *b = v.B + (long long)j * v.ld;
        double acc = 0.0;
        for (long long i = lo; i < hi; i++) acc += b[i] * b[i];
        v.part2[(size_t)blockIdx.x * BCG_MAX_S + j] = acc;
    }
    __syncthreads();
    if (!grid_sync(v.bar, st)) return;
    if (blockIdx.x == 0 && threadIdx.x < v.s) {   // eight interleaved sums over the CTAs
        double t[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int c = 0; c < (int)gridDim.x; c++) t[c & 7] += __ldcg(&v.part2[(size_t)c * BCG_MAX_S + threadIdx.x]);
        sm->bn[threadIdx.x] = sqrt(((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7])));
    }
    const bool ok = coop_orth(v, v.R, lo, hi);          // its first barrier publishes bn too
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        bool nan = false;
        for (int j = 0; j < v.s; j++) nan = nan || !isfinite(sm->w2[j]) || !isfinite(sm->bn[j]);
        const bool pass = !nan && cols_pass(v, sm->w2);
        int go = 1;
        if (!ok) {
            go = 0;
            if (!*(volatile int *)&st->err) st->status = LS_BREAKDOWN;
        } else if (nan) {
            set_err(st, ERRB_NAN);
            go = 0;
        } else if (pass || sm->rank == 0) {
            go = 0;                                     // confirm on the true residual
        } else if (st->max_iter <= 0) {
            go = 0;
        }
        set_cond(st, h_inner, go);
        set_cond(st, h_outer, 1u);
    }
}

// One step after Q = A P.
__global__ void __launch_bounds__(BK) bcgd_step_kernel(BcgVecs v, cudaGraphConditionalHandle h_inner) {
    __shared__ double G[SL * SL], H[SL * SL], coef[SL * SL];
    __shared__ int flag_s, r_s;
    State *st = v.st;
    BcgSmall *sm = v.sm;
    count_launch(st);
    const int s = v.s;
    if (*(volatile int *)&st->err || *(volatile int *)&st->status == LS_BREAKDOWN) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(st, h_inner, 0u);
        return;
    }
    if (threadIdx.x == 0) r_s = *(volatile int *)&sm->rank;
    __syncthreads();
    const int r = r_s;
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    // gamma = P^T Q and P^T R
    gram_partial_ld(v, v.part, v.P, r, v.Q, r, lo, hi);
    gram_partial_ld(v, v.partb, v.P, r, v.R, s, lo, hi);
    if (!grid_sync(v.bar, st)) return;
    if (blockIdx.x == 0) {
        gram_reduce_ld(v.part, r, r, G);
        gram_reduce_ld(v.partb, r, s, H);
        __syncthreads();
        if (threadIdx.x == 0) flag_s = small_chol(r, G) ? 1 : 0;   // positive definite for SPD A
        __syncthreads();
        if (flag_s) small_chol_solve(r, s, G, H);       // alpha = gamma^-1 P^T R (all threads)
        if (threadIdx.x == 0) {
            for (int e = 0; e < SL * SL; e++) {
                sm->Lg[e] = G[e];
                sm->alpha[e] = H[e];
            }
            sm->ok = flag_s;
            if (!flag_s) st->status = LS_BREAKDOWN;
        }
    }
    if (!grid_sync(v.bar, st)) return;
    if (threadIdx.x == 0) flag_s = *(volatile int *)&sm->ok;
    for (int e = threadIdx.x; e < SL * SL; e += blockDim.x) coef[e] = __ldcg(&sm->alpha[e]);
    __syncthreads();
    if (!flag_s) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(st, h_inner, 0u);
        return;
    }
    // X += P alpha, R -= Q alpha (row by row), then Q^T R and ||R_j||^2
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        double p[BCG_MAX_S], q[BCG_MAX_S];
#pragma unroll
        for (int c = 0; c < BCG_MAX_S; c++) {
            p[c] = c < r ? v.P[(long long)c * v.ld + i] : 0.0;
            q[c] = c < r ? v.Q[(long long)c * v.ld + i] : 0.0;
        }
        for (int j = 0; j < s; j++) {
            double dx = 0.0, dr = 0.0;
#pragma unroll
            for (int c = 0; c < BCG_MAX_S; c++)
                if (c < r) {
                    dx += p[c] * coef[c + j * SL];
                    dr += q[c] * coef[c + j * SL];
                }
            v.X[(long long)j * v.ld + i] += dx;
            v.R[(long long)j * v.ld + i] -= dr;
        }
    }
    __syncthreads();
    gram_partial_ld(v, v.part, v.Q, r, v.R, s, lo, hi);
    for (int j = threadIdx.x; j < s; j += blockDim.x) {
        const double *rr = v.R + (long long)j * v.ld;
        double acc = 0.0;
        for (long long i = lo; i < hi; i++) acc += rr[i] * rr[i];
        v.part2[(size_t)blockIdx.x * BCG_MAX_S + j] = acc;
    }
    if (!grid_sync(v.bar, st)) return;
    if (blockIdx.x == 0) {
        __shared__ double r2[BCG_MAX_S];
        __shared__ int nan_s, go_s;
        // ||R_j||^2: thread j, eight interleaved sums over the CTAs
        if (threadIdx.x < s) {
            double t[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            const int nc = (int)gridDim.x;
            for (int c = 0; c < nc; c++) t[c & 7] += __ldcg(&v.part2[(size_t)c * BCG_MAX_S + threadIdx.x]);
            r2[threadIdx.x] = ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            bool nan = false;
            for (int j = 0; j < s; j++) nan = nan || !isfinite(r2[j]);
            nan_s = nan;
            go_s = !nan && !cols_pass(v, r2);
        }
        __syncthreads();
        if (go_s) {
            gram_reduce_ld(v.part, r, s, H);
            for (int e = threadIdx.x; e < SL * SL; e += blockDim.x) G[e] = sm->Lg[e];
            __syncthreads();
            small_chol_solve(r, s, G, H);              // beta = -gamma^-1 Q^T R (all threads)
        }
        if (threadIdx.x == 0) {
            int go = go_s;
            if (go)
                for (int e = 0; e < SL * SL; e++) sm->beta[e] = -H[e];
            st->iter++;
            if (nan_s) set_err(st, ERRB_NAN);
            sm->update_p = go;
            if (go && st->iter >= st->max_iter) go = 0;
            sm->ok = go;
        }
    }
    if (!grid_sync(v.bar, st)) return;
    if (threadIdx.x == 0) flag_s = *(volatile int *)&sm->update_p;
    for (int e = threadIdx.x; e < SL * SL; e += blockDim.x) coef[e] = __ldcg(&sm->beta[e]);
    __syncthreads();
    if (!flag_s) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(st, h_inner, 0u);
        return;
    }
    // W = R + P beta into Q's storage, then P = orth(W)
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        double p[BCG_MAX_S];
#pragma unroll
        for (int c = 0; c < BCG_MAX_S; c++) p[c] = c < r ? v.P[(long long)c * v.ld + i] : 0.0;
        for (int j = 0; j < s; j++) {
            double acc = v.R[(long long)j * v.ld + i];
#pragma unroll
            for (int c = 0; c < BCG_MAX_S; c++)
                if (c < r) acc += p[c] * coef[c + j * SL];
            v.Q[(long long)j * v.ld + i] = acc;
        }
    }
    __syncthreads();
    const bool ok = coop_orth(v, v.Q, lo, hi);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int go = *(volatile int *)&sm->ok;
        if (!ok) {
            go = 0;
            if (!*(volatile int *)&st->err) st->status = LS_BREAKDOWN;
        } else if (sm->rank == 0) {
            go = 0;                                     // nothing left to search: confirm
        }
        set_cond(st, h_inner, go ? 1u : 0u);
    }
}

// After the loop: the true residual (residual GEMVs, ||R_j||^2 in sm->r2);
// accept, stop, or restart from it with P = orth(R).
__global__ void __launch_bounds__(BK) bcgd_check_kernel(BcgVecs v, cudaGraphConditionalHandle h_outer,
                                                        cudaGraphConditionalHandle h_inner) {
    __shared__ int restart_s;
    State *st = v.st;
    BcgSmall *sm = v.sm;
    count_launch(st);
    const int s = v.s;
    if (threadIdx.x == 0) {
        bool pass = true, nan = false;
        for (int j = 0; j < s; j++) {
            const double r2 = *(volatile double *)&sm->r2[j];
            nan = nan || !isfinite(r2);
            pass = pass && sqrt(r2) <= v.rtol * sm->bn[j];
        }
        int restart = 0;
        if (*(volatile int *)&st->err || nan) {
            if (nan) set_err(st, ERRB_NAN);
        } else if (*(volatile int *)&st->status == LS_BREAKDOWN) {
        } else if (pass) {
            if (blockIdx.x == 0) st->status = LS_OK;
        } else if (*(volatile int *)&st->iter >= st->max_iter) {
            if (blockIdx.x == 0) st->status = LS_NOT_CONVERGED;
        } else {
            restart = 1;
        }
        restart_s = restart;
    }
    __syncthreads();
    if (!restart_s) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            set_cond(st, h_outer, 0u);
            set_cond(st, h_inner, 0u);
        }
        return;
    }
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    const bool ok = coop_orth(v, v.R, lo, hi);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int go = 1;
        if (!ok) {
            go = 0;
            if (!*(volatile int *)&st->err) st->status = LS_BREAKDOWN;
        } else if (sm->rank == 0) {
            go = 0;
            st->status = LS_BREAKDOWN;                  // not converged and nothing left to search
        }
        st->cycles++;
        set_cond(st, h_inner, go ? 1u : 0u);
        set_cond(st, h_outer, go ? 1u : 0u);
    }
}

BcgKernels bcg_kernels() {
    BcgKernels K{};
    K.init = reinterpret_cast<void *>(&bcg_init_kernel);
    K.step = reinterpret_cast<void *>(&bcg_step_kernel);
    K.check = reinterpret_cast<void *>(&bcg_check_kernel);
    K.dinit = reinterpret_cast<void *>(&bcgd_init_kernel);
    K.dstep = reinterpret_cast<void *>(&bcgd_step_kernel);
    K.dcheck = reinterpret_cast<void *>(&bcgd_check_kernel);
    K.block = BK;
    return K;
}

}  // namespace lsi
