// k_bcg.cu -- O'Leary's block conjugate gradient for s right-hand sides.
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
// This CTA's partial U^T V over rows [lo, hi) into part[cta][s*s].
__device__ __forceinline__ void gram_partial(const BcgVecs &v, const double *U, const double *V, long long lo,
                                             long long hi) {
    const int s = v.s;
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
        const int a = e % s, b = e / s;
        const double *u = U + (long long)a * v.ld, *w = V + (long long)b * v.ld;
        double acc = 0.0;
        for (long long i = lo; i < hi; i++) acc += u[i] * w[i];
        v.part[(size_t)blockIdx.x * BCG_MAX_S * BCG_MAX_S + e] = acc;
    }
}

// One warp: G = sum of the partials in CTA order.
__device__ __forceinline__ void gram_reduce(const BcgVecs &v, double *G) {
    const int s = v.s;
    for (int e = threadIdx.x & 31; e < s * s; e += 32) {
        double acc = 0.0;
        for (int c = 0; c < (int)gridDim.x; c++) acc += __ldcg(&v.part[(size_t)c * BCG_MAX_S * BCG_MAX_S + e]);
        G[e] = acc;
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

BcgKernels bcg_kernels() {
    BcgKernels K{};
    K.init = reinterpret_cast<void *>(&bcg_init_kernel);
    K.step = reinterpret_cast<void *>(&bcg_step_kernel);
    K.check = reinterpret_cast<void *>(&bcg_check_kernel);
    K.block = BK;
    return K;
}

}  // namespace lsi
