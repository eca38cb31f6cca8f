// k_krylov.cu -- the vector work of the Krylov iterations, fused around the
// matrix-vector product and run without host synchronisation:
//
//   CG (paper, CG paragraph; Hestenes-Stiefel form):
//     cg_init    x = 0 (or keep x0), r = b (or b - A x0 from the GEMV), p = r,
//                rho = r.r, ||b||, the tolerance, and the loop conditions;
//     cg_update  x += alpha p, r -= alpha q, rho' = r.r (grid reduction),
//                stop test ||r|| <= rtol ||b||, beta = rho'/rho, p = r + beta p;
//                alpha itself is produced by the GEMV's last CTA (p.q);
//     cg_check   after the loop: accept on the true residual b - A x, or
//                restart from it (residual replacement) while iterations remain.
//   BiCGSTAB (paper, BiCGSTAB listing; the steps it leaves out -- omega =
//   t.s / t.t, r = s - omega t, the next rho = r^.r and the stop test -- are
//   written in):
//     bs_init    x = 0 (or keep x0), r = b (or b - A x0), r^ = r, p = r, v = 0,
//                rho = r^.r, ||b||, the tolerance, the loop conditions;
//     bs_s       s = r - alpha v (alpha from the first GEMV's last CTA: rho /
//                r^.v), ||s||; when ||s|| passes, x += alpha p ends the step;
//     bs_update  omega = t.s / t.t (t.s from the second GEMV), x += alpha p +
//                omega s, r = s - omega t, rho' = r^.r, stop test,
//                beta = (rho'/rho)(alpha/omega), p = r + beta (p - omega v);
//     bs_check   after the loop: accept on the true residual, or restart from
//                it with r^ = r while iterations remain.
//   GMRES(m) (paper, GMRES pseudocode and the restart paragraph; the
//   least-squares update by Givens rotations follows Saad's book):
//     gm_init    x = 0 (or keep x0), ||b|| and the tolerance;
//     gm_start   beta = ||b - A x|| (from the GEMV), v_1 = r / beta, g = beta e1;
//     gm_arnoldi classical Gram-Schmidt: h = V_k^T w and w -= V_k h (a second
//                pass when ||w|| falls below 0.7 ||A v_k||, or always when
//                asked), h_{k+1,k} = ||w||, v_{k+1} = w / h_{k+1,k}; then one
//                thread applies the old rotations to column k, forms the new
//                one, updates g and tests |g_{k+1}| <= rtol ||b||;
//     gm_finish  back-solve R y = g (one warp), x += V_k y.
//   Jacobi (paper, introduction: the classical stationary methods, taken from
//   the textbooks): x(k+1) = x(k) + D^-1 (b - A x(k)).  The step itself is the
//   GEMV's epilogue (next iterate into a second vector, ||b - A x(k)||^2
//   reduced, stop test in its last CTA); around it:
//     ja_diag    D^-1 from the FP64 diagonal of A, breakdown on a zero entry;
//     ja_init    x = 0 (or keep x0), ||b||, the tolerance, the loop condition;
//     ja_next    take the next iterate unless the GEMV's test stopped the loop.
//
// Cooperative kernels (launched with the cooperative attribute, grid =
// co-resident blocks) meet at a bounded grid barrier; every cross-block sum
// is done by every block in the same fixed order, so all blocks agree
// bit for bit and results are deterministic.  Loop control is on the
// device: the kernels set the graph's while-node conditions.
#include <cuda_runtime.h>

#include "ls_device.cuh"
#include "ls_internal.h"

namespace lsi {

constexpr int KB = 256;   // threads per block of the vector kernels

// Sum of one partial slot over all blocks, by one warp (fixed order).
__device__ __forceinline__ double reduce_slot(const double *part, int slot, int G) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < G; b += 32) s += __ldcg(&part[(size_t)slot * G + b]);
    return warp_sum(s);
}

// Block b publishes `v` into slot `slot`.
__device__ __forceinline__ void publish(double *part, int slot, double v) {
    if (threadIdx.x == 0) part[(size_t)slot * gridDim.x + blockIdx.x] = v;
}

// ============================================================================
// CG
// ============================================================================
__global__ void __launch_bounds__(KB) cg_init_kernel(Vecs v, int x0_given,
                                                     cudaGraphConditionalHandle h_outer,
                                                     cudaGraphConditionalHandle h_inner) {
    __shared__ double red[KB / 32];
    State *st = v.st;
    count_launch(st);
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    double bb = 0.0, rr = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double bi = v.b[i];
        double ri;
        if (!x0_given) {
            v.x[i] = 0.0;
            ri = bi;
            v.r[i] = ri;
        } else {
            ri = v.r[i];           // b - A x0, written by the residual GEMV
        }
        v.p[i] = ri;
        bb += bi * bi;
        rr += ri * ri;
    }
    bb = block_sum(bb, red);
    rr = block_sum(rr, red);
    publish(v.part, 0, bb);
    publish(v.part, 1, rr);
    if (!grid_sync(v.bar, st)) return;
    __shared__ double b2_s;
    if (threadIdx.x < 32) {
        const double t = reduce_slot(v.part, 0, gridDim.x);
        if (threadIdx.x == 0) b2_s = t;
    }
    __syncthreads();
    if (b2_s == 0.0 && x0_given)   // b = 0: x = 0 solves exactly, whatever x0 was
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) v.x[i] = 0.0;
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        const double b2 = b2_s;
        const double r2 = reduce_slot(v.part, 1, gridDim.x);
        if (threadIdx.x == 0) {
            const double bn = sqrt(b2);
            st->bnorm = bn;
            st->tol_abs = v.rtol * bn;
            st->rho = r2;
            st->rnorm = sqrt(r2);
            st->true_rnorm = sqrt(r2);
            int go = 1;
            if (!isfinite(b2) || !isfinite(r2)) {
                set_err(st, ERRB_NAN);
                go = 0;
            } else if (bn == 0.0 || sqrt(r2) <= st->tol_abs) {
                st->status = LS_OK;    // b = 0 (x = 0), or the start already solves
                go = 0;
            } else if (st->max_iter <= 0) {
                st->status = LS_NOT_CONVERGED;
                go = 0;
            }
            set_cond(v.st, h_outer, go);
            set_cond(v.st, h_inner, go);
        }
    }
}

__global__ void __launch_bounds__(KB) cg_update_kernel(Vecs v, cudaGraphConditionalHandle h_inner) {
    __shared__ double red[KB / 32];
    State *st = v.st;
    count_launch(st);
    const double alpha = st->alpha, rho = st->rho, tol = st->tol_abs;
    const int status = st->status, err = st->err;
    if (status == LS_BREAKDOWN || err) {   // the GEMV found p.Ap <= 0 (or a wait failed)
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(v.st, h_inner, 0);
        return;
    }
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    double rr = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        v.x[i] += alpha * v.p[i];
        const double ri = v.r[i] - alpha * v.q[i];
        v.r[i] = ri;
        rr += ri * ri;
    }
    rr = block_sum(rr, red);
    publish(v.part, 0, rr);
    if (!grid_sync(v.bar, st)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(v.st, h_inner, 0);
        return;
    }
    __shared__ double rho_new_s;
    if (threadIdx.x < 32) {
        const double t = reduce_slot(v.part, 0, gridDim.x);
        if (threadIdx.x == 0) rho_new_s = t;
    }
    __syncthreads();
    const double rho_new = rho_new_s;
    const bool finite = isfinite(rho_new);
    const bool conv = finite && sqrt(rho_new) <= tol;
    const double beta = rho_new / rho;
    if (finite && !conv) {
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x)
            v.p[i] = v.r[i] + beta * v.p[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->rho = rho_new;
        st->rnorm = sqrt(rho_new);
        st->beta = beta;
        st->iter += 1;
        st->conv = conv;
        if (!finite) set_err(st, ERRB_NAN);
        if (!finite || conv || st->iter >= st->max_iter) set_cond(v.st, h_inner, 0);
    }
}

// After the loop the GEMV has put q = b - A x and ||q|| (true_rnorm) in place.
__global__ void __launch_bounds__(KB) cg_check_kernel(Vecs v, cudaGraphConditionalHandle h_outer,
                                                      cudaGraphConditionalHandle h_inner) {
    State *st = v.st;
    count_launch(st);
    const double t = st->true_rnorm;
    int decision;   // 0 accept, 1 limit, 2 breakdown/error, 3 replace and continue
    if (st->err || !isfinite(t)) decision = 2;
    else if (st->status == LS_BREAKDOWN) decision = 2;
    else if (t <= st->tol_abs) decision = 0;
    else if (st->iter >= st->max_iter) decision = 1;
    else decision = 3;
    if (decision == 3) {
        long long lo, hi;
        block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const double qi = v.q[i];
            v.r[i] = qi;
            v.p[i] = qi;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (decision == 0) st->status = LS_OK;
        if (decision == 1) st->status = LS_NOT_CONVERGED;
        if (decision == 2 && !isfinite(t)) set_err(st, ERRB_NAN);
        st->cycles += 1;   // true-residual checks
        if (decision == 3) {
            st->rho = t * t;
            st->rnorm = t;
            st->conv = 0;
        }
        set_cond(v.st, h_outer, decision == 3);
        set_cond(v.st, h_inner, decision == 3);
    }
}

// ============================================================================
// GMRES(m)
// ============================================================================
__global__ void __launch_bounds__(KB) gm_init_kernel(Vecs v, int x0_given,
                                                     cudaGraphConditionalHandle h_outer) {
    __shared__ double red[KB / 32];
    State *st = v.st;
    count_launch(st);
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    double bb = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        if (!x0_given) v.x[i] = 0.0;
        const double bi = v.b[i];
        bb += bi * bi;
    }
    bb = block_sum(bb, red);
    publish(v.part, 0, bb);
    if (!grid_sync(v.bar, st)) return;
    __shared__ double b2_s;
    if (threadIdx.x < 32) {
        const double t = reduce_slot(v.part, 0, gridDim.x);
        if (threadIdx.x == 0) b2_s = t;
    }
    __syncthreads();
    if (b2_s == 0.0 && x0_given)   // b = 0: x = 0 solves exactly
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) v.x[i] = 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double b2 = b2_s;
        {
            const double bn = sqrt(b2);
            st->bnorm = bn;
            st->tol_abs = v.rtol * bn;
            int go = 1;
            if (!isfinite(b2)) {
                set_err(st, ERRB_NAN);
                go = 0;
            } else if (bn == 0.0) {
                st->status = LS_OK;
                st->true_rnorm = 0.0;
                go = 0;
            }
            set_cond(v.st, h_outer, go);
        }
    }
}

// A cycle starts: the residual GEMV has written q = b - A x, true_rnorm = ||q||.
__global__ void __launch_bounds__(KB) gm_start_kernel(Vecs v, cudaGraphConditionalHandle h_outer,
                                                      cudaGraphConditionalHandle h_inner) {
    State *st = v.st;
    count_launch(st);
    const double beta = st->true_rnorm;
    int go;
    if (st->err || !isfinite(beta)) go = -1;
    else if (st->status == LS_BREAKDOWN) go = -3;
    else if (beta <= st->tol_abs) go = 0;
    else if (st->total >= st->max_iter) go = -2;
    else go = 1;
    if (go == 1) {
        long long lo, hi;
        block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) v.V[i] = v.q[i] / beta;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (go == -1) set_err(st, ERRB_NAN);
        if (go == 0) st->status = LS_OK;
        if (go == -2) st->status = LS_NOT_CONVERGED;
        // no new cycle: the gm_finish node that follows in this body must not
        // apply the previous cycle's correction a second time
        if (go != 1) st->k = 0;
        if (go == 1) {
            GmresSmall *gm = v.gm;
            gm->g[0] = beta;
            st->k = 0;
            st->est = beta;
            st->cycles += 1;
        }
        set_cond(v.st, h_outer, go == 1);
        set_cond(v.st, h_inner, go == 1);
    }
}

// One Arnoldi step after the GEMV has written w = A v_k into column k+1 and
// ||w||^2 into wnorm0.
__global__ void __launch_bounds__(KB) gm_arnoldi_kernel(Vecs v, cudaGraphConditionalHandle h_inner) {
    __shared__ double red[KB / 32];
    __shared__ double h[LS_MAX_RESTART + 1];
    __shared__ double hsum[LS_MAX_RESTART + 1];
    __shared__ double wn_s;
    State *st = v.st;
    count_launch(st);
    const int k = st->k;                  // 0-based: w is column k+1, basis columns 0..k
    const double wnorm0 = st->wnorm0;
    const int always2 = st->reorth;
    const int G = gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    long long lo, hi;
    block_range(v.n, blockIdx.x, G, lo, hi);
    double *w = v.V + (long long)(k + 1) * v.ldv;
    for (int j = threadIdx.x; j <= k; j += blockDim.x) hsum[j] = 0.0;
    __syncthreads();

    double wn2 = 0.0;
    for (int pass = 0; pass < 2; pass++) {
        // h_j = v_j . w over this block's rows (warp per column), one slot per j
        for (int j = warp; j <= k; j += nw) {
            const double *vj = v.V + (long long)j * v.ldv;
            double s = 0.0;
            for (long long i = lo + lane; i < hi; i += 32) s += vj[i] * w[i];
            s = warp_sum(s);
            if (lane == 0) v.part[(size_t)j * G + blockIdx.x] = s;
        }
        if (!grid_sync(v.bar, st)) break;
        for (int j = warp; j <= k; j += nw) {
            const double t = reduce_slot(v.part, j, G);
            if (lane == 0) h[j] = t;
        }
        __syncthreads();
        // w -= V_k h on this block's rows, and ||w||^2
        double acc = 0.0;
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            double wi = w[i];
            for (int j = 0; j <= k; j++) wi -= h[j] * v.V[(long long)j * v.ldv + i];
            w[i] = wi;
            acc += wi * wi;
        }
        for (int j = threadIdx.x; j <= k; j += blockDim.x) hsum[j] += h[j];
        acc = block_sum(acc, red);
        // slot k+1 is free (h used slots 0..k); keep it separate from them
        publish(v.part, LS_MAX_RESTART + 1, acc);
        if (!grid_sync(v.bar, st)) break;
        if (threadIdx.x < 32) {
            const double t = reduce_slot(v.part, LS_MAX_RESTART + 1, G);
            if (threadIdx.x == 0) wn_s = t;
        }
        __syncthreads();
        wn2 = wn_s;
        // a second pass only when cancellation lost accuracy (or always if asked)
        if (pass == 0 && !always2 && !(wn2 < 0.49 * wnorm0)) break;
    }
    if (st->err) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(v.st, h_inner, 0);
        return;
    }
    const double wn = sqrt(wn2);
    const bool lucky = !(wn > 1e-14 * sqrt(wnorm0));
    if (!lucky)
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) w[i] = w[i] / wn;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        GmresSmall *gm = v.gm;
        const int m1 = LS_MAX_RESTART + 1;
        double *Hk = gm->H + (size_t)k * m1;
        for (int j = 0; j <= k; j++) Hk[j] = hsum[j];
        Hk[k + 1] = wn;
        for (int j = 0; j < k; j++) {          // earlier rotations
            const double a = Hk[j], c = Hk[j + 1];
            Hk[j] = gm->cs[j] * a + gm->sn[j] * c;
            Hk[j + 1] = -gm->sn[j] * a + gm->cs[j] * c;
        }
        const double den = hypot(Hk[k], Hk[k + 1]);
        bool stop = false;
        if (den == 0.0 || !isfinite(den)) {
            st->status = LS_BREAKDOWN;
            if (!isfinite(den)) set_err(st, ERRB_NAN);
            stop = true;
        } else {
            const double c = Hk[k] / den, s = Hk[k + 1] / den;
            gm->cs[k] = c;
            gm->sn[k] = s;
            Hk[k] = den;
            Hk[k + 1] = 0.0;
            gm->g[k + 1] = -s * gm->g[k];
            gm->g[k] = c * gm->g[k];
            st->k = k + 1;
            st->total += 1;
            st->est = fabs(gm->g[k + 1]);
            if (st->est <= st->tol_abs || lucky || k + 1 >= st->m || st->total >= st->max_iter)
                stop = true;
        }
        if (stop) set_cond(v.st, h_inner, 0);
    }
}

// End of a cycle: R y = g (upper triangular k x k), x += V_k y.
__global__ void __launch_bounds__(KB) gm_finish_kernel(Vecs v) {
    __shared__ double ys[LS_MAX_RESTART];
    State *st = v.st;
    count_launch(st);
    const int k = st->k;
    if (st->status == LS_BREAKDOWN || st->err || k == 0) return;
    GmresSmall *gm = v.gm;
    const int m1 = LS_MAX_RESTART + 1;
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        // back substitution by one warp: row i uses y_{i+1..k-1}
        const int lane = threadIdx.x;
        for (int i = k - 1; i >= 0; i--) {
            double s = 0.0;
            for (int j = i + 1 + lane; j < k; j += 32) s += gm->H[(size_t)j * m1 + i] * ys[j];
            s = warp_sum(s);
            if (lane == 0) ys[i] = (gm->g[i] - s) / gm->H[(size_t)i * m1 + i];
            __syncwarp();
        }
        for (int j = lane; j < k; j += 32) gm->y[j] = ys[j];
    }
    if (!grid_sync(v.bar, st)) return;
    for (int j = threadIdx.x; j < k; j += blockDim.x) ys[j] = __ldcg(&gm->y[j]);
    __syncthreads();
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        double xi = v.x[i];
        for (int j = 0; j < k; j++) xi += v.V[(long long)j * v.ldv + i] * ys[j];
        v.x[i] = xi;
    }
}

// ============================================================================
// BiCGSTAB
// ============================================================================
__global__ void __launch_bounds__(KB) bs_init_kernel(Vecs v, int x0_given,
                                                     cudaGraphConditionalHandle h_outer,
                                                     cudaGraphConditionalHandle h_inner) {
    __shared__ double red[KB / 32];
    State *st = v.st;
    count_launch(st);
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    double bb = 0.0, rr = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double bi = v.b[i];
        double ri;
        if (!x0_given) {
            v.x[i] = 0.0;
            ri = bi;
            v.r[i] = ri;
        } else {
            ri = v.r[i];           // b - A x0, written by the residual GEMV
        }
        v.rh[i] = ri;
        v.p[i] = ri;
        v.vv[i] = 0.0;
        bb += bi * bi;
        rr += ri * ri;
    }
    bb = block_sum(bb, red);
    rr = block_sum(rr, red);
    publish(v.part, 0, bb);
    publish(v.part, 1, rr);
    if (!grid_sync(v.bar, st)) return;
    __shared__ double b2_s;
    if (threadIdx.x < 32) {
        const double t = reduce_slot(v.part, 0, gridDim.x);
        if (threadIdx.x == 0) b2_s = t;
    }
    __syncthreads();
    if (b2_s == 0.0 && x0_given)   // b = 0: x = 0 solves exactly, whatever x0 was
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) v.x[i] = 0.0;
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        const double b2 = b2_s;
        const double r2 = reduce_slot(v.part, 1, gridDim.x);
        if (threadIdx.x == 0) {
            const double bn = sqrt(b2);
            st->bnorm = bn;
            st->tol_abs = v.rtol * bn;
            st->rho = r2;              // r^ = r
            st->alpha = 1.0;
            st->omega = 1.0;
            st->skip = 0;
            st->rnorm = sqrt(r2);
            st->true_rnorm = sqrt(r2);
            int go = 1;
            if (!isfinite(b2) || !isfinite(r2)) {
                set_err(st, ERRB_NAN);
                go = 0;
            } else if (bn == 0.0 || sqrt(r2) <= st->tol_abs) {
                st->status = LS_OK;
                go = 0;
            } else if (st->max_iter <= 0) {
                st->status = LS_NOT_CONVERGED;
                go = 0;
            }
            set_cond(v.st, h_outer, go);
            set_cond(v.st, h_inner, go);
        }
    }
}

// s = r - alpha v, ||s||^2; when ||s|| passes the test (or the next product
// would exceed the limit) x += alpha p, r = s and the step ends here.
__global__ void __launch_bounds__(KB) bs_s_kernel(Vecs v, cudaGraphConditionalHandle h_inner) {
    __shared__ double red[KB / 32];
    State *st = v.st;
    count_launch(st);
    if (st->status == LS_BREAKDOWN || st->err) {   // r^.v = 0 (or a wait failed)
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->skip = 1;
            set_cond(v.st, h_inner, 0);
        }
        return;
    }
    const double alpha = st->alpha, tol = st->tol_abs;
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    double ss = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double si = v.r[i] - alpha * v.vv[i];
        v.s[i] = si;
        ss += si * si;
    }
    ss = block_sum(ss, red);
    publish(v.part, 0, ss);
    if (!grid_sync(v.bar, st)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->skip = 1;
            set_cond(v.st, h_inner, 0);
        }
        return;
    }
    __shared__ double ss_s;
    if (threadIdx.x < 32) {
        const double t = reduce_slot(v.part, 0, gridDim.x);
        if (threadIdx.x == 0) ss_s = t;
    }
    __syncthreads();
    const double s2 = ss_s;
    const bool finite = isfinite(s2);
    const bool pass = finite && sqrt(s2) <= tol;
    const bool last = st->iter + 1 >= st->max_iter;   // no room for the second product
    if (finite && (pass || last)) {
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            v.x[i] += alpha * v.p[i];
            v.r[i] = v.s[i];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->iter += 1;                 // v = A p
        if (!finite) set_err(st, ERRB_NAN);
        const int stop = !finite || pass || last;
        st->skip = stop;
        if (pass) {
            st->conv = 1;
            st->rnorm = sqrt(s2);
        }
        if (stop) set_cond(v.st, h_inner, 0);
    }
}

// omega = t.s / t.t, x += alpha p + omega s, r = s - omega t, rho' = r^.r,
// stop test, beta = (rho'/rho)(alpha/omega), p = r + beta (p - omega v).
__global__ void __launch_bounds__(KB) bs_update_kernel(Vecs v, cudaGraphConditionalHandle h_inner) {
    __shared__ double red[KB / 32];
    State *st = v.st;
    count_launch(st);
    if (st->skip) return;
    const double alpha = st->alpha, rho = st->rho, tol = st->tol_abs, ts = st->dot;
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    double tt = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double ti = v.t[i];
        tt += ti * ti;
    }
    tt = block_sum(tt, red);
    publish(v.part, 0, tt);
    if (!grid_sync(v.bar, st)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(v.st, h_inner, 0);
        return;
    }
    __shared__ double tt_s;
    if (threadIdx.x < 32) {
        const double t = reduce_slot(v.part, 0, gridDim.x);
        if (threadIdx.x == 0) tt_s = t;
    }
    __syncthreads();
    const double t2 = tt_s;
    if (t2 == 0.0 || !isfinite(t2) || !isfinite(ts)) {   // t = A s = 0 with s != 0, or NaN
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->iter += 1;
            if (!isfinite(t2) || !isfinite(ts)) set_err(st, ERRB_NAN);
            else st->status = LS_BREAKDOWN;
            set_cond(v.st, h_inner, 0);
        }
        return;
    }
    const double omega = ts / t2;
    double rr = 0.0, rhr = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double si = v.s[i];
        v.x[i] += alpha * v.p[i] + omega * si;
        const double ri = si - omega * v.t[i];
        v.r[i] = ri;
        rr += ri * ri;
        rhr += v.rh[i] * ri;
    }
    rr = block_sum(rr, red);
    rhr = block_sum(rhr, red);
    publish(v.part, 1, rr);
    publish(v.part, 2, rhr);
    if (!grid_sync(v.bar, st)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(v.st, h_inner, 0);
        return;
    }
    __shared__ double rr_s, rhr_s;
    if (threadIdx.x < 32) {
        const double a = reduce_slot(v.part, 1, gridDim.x);
        const double b = reduce_slot(v.part, 2, gridDim.x);
        if (threadIdx.x == 0) {
            rr_s = a;
            rhr_s = b;
        }
    }
    __syncthreads();
    const double r2 = rr_s, rho_new = rhr_s;
    const bool finite = isfinite(r2) && isfinite(rho_new);
    const bool conv = finite && sqrt(r2) <= tol;
    const bool broke = omega == 0.0 || rho_new == 0.0;
    const int iter_new = st->iter + 1;                 // t = A s
    const bool go = finite && !conv && !broke && iter_new < st->max_iter;
    if (go) {
        const double beta = (rho_new / rho) * (alpha / omega);
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x)
            v.p[i] = v.r[i] + beta * (v.p[i] - omega * v.vv[i]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->omega = omega;
        st->beta = (rho_new / rho) * (alpha / omega);
        st->rho = rho_new;
        st->rnorm = sqrt(r2);
        st->iter = iter_new;
        st->conv = conv;
        if (!finite) set_err(st, ERRB_NAN);
        else if (broke && !conv) st->status = LS_BREAKDOWN;
        if (!go) set_cond(v.st, h_inner, 0);
    }
}

// After the loop the GEMV has put q = b - A x and ||q|| (true_rnorm) in place:
// accept, stop, or restart from q with a new shadow residual r^ = q.
__global__ void __launch_bounds__(KB) bs_check_kernel(Vecs v, cudaGraphConditionalHandle h_outer,
                                                      cudaGraphConditionalHandle h_inner) {
    State *st = v.st;
    count_launch(st);
    const double t = st->true_rnorm;
    int decision;   // 0 accept, 1 limit, 2 breakdown/error, 3 restart
    if (st->err || !isfinite(t)) decision = 2;
    else if (t <= st->tol_abs) decision = 0;
    else if (st->status == LS_BREAKDOWN) decision = 2;
    else if (st->iter >= st->max_iter) decision = 1;
    else decision = 3;
    if (decision == 3) {
        long long lo, hi;
        block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const double qi = v.q[i];
            v.r[i] = qi;
            v.rh[i] = qi;
            v.p[i] = qi;
            v.vv[i] = 0.0;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (decision == 0) st->status = LS_OK;
        if (decision == 1) st->status = LS_NOT_CONVERGED;
        if (decision == 2 && !isfinite(t)) set_err(st, ERRB_NAN);
        st->cycles += 1;   // true-residual checks
        if (decision == 3) {
            st->rho = t * t;
            st->rnorm = t;
            st->alpha = 1.0;
            st->omega = 1.0;
            st->conv = 0;
            st->skip = 0;
        }
        set_cond(v.st, h_outer, decision == 3);
        set_cond(v.st, h_inner, decision == 3);
    }
}

// ============================================================================
// Jacobi
// ============================================================================
// dinv = 1 / a_ii from the FP64 matrix (before the loop, outside the graph,
// since A may be borrowed per call); a zero a_ii marks the solve a breakdown.
__global__ void __launch_bounds__(KB) ja_diag_kernel(int n, const double *__restrict__ A, long long lda,
                                                     double *__restrict__ dinv, State *st) {
    count_launch(st);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double d = A[i * lda + i];
        if (d == 0.0) {
            st->status = LS_BREAKDOWN;   // every writer writes the same value
            dinv[i] = 0.0;
        } else {
            dinv[i] = 1.0 / d;
        }
    }
}

// x = 0 unless x0 was given; ||b|| and the tolerance; b = 0 ends the solve
// with x = 0 (unless the diagonal broke down first).  v.q holds the next
// iterate, v.p holds D^-1.
__global__ void __launch_bounds__(KB) ja_init_kernel(Vecs v, int x0_given,
                                                     cudaGraphConditionalHandle h_loop) {
    __shared__ double red[KB / 32];
    State *st = v.st;
    count_launch(st);
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    double bb = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double bi = v.b[i];
        if (!x0_given) v.x[i] = 0.0;
        bb += bi * bi;
    }
    bb = block_sum(bb, red);
    publish(v.part, 0, bb);
    if (!grid_sync(v.bar, st)) return;
    __shared__ double b2_s;
    if (threadIdx.x < 32) {
        const double t = reduce_slot(v.part, 0, gridDim.x);
        if (threadIdx.x == 0) b2_s = t;
    }
    __syncthreads();
    const bool broke = *(volatile int *)&st->status == LS_BREAKDOWN;
    const double b2 = b2_s;
    if (b2 == 0.0 && !broke && x0_given)
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) v.x[i] = 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double bn = sqrt(b2);
        st->bnorm = bn;
        st->tol_abs = v.rtol * bn;
        st->skip = 0;
        int go = 1;
        if (!isfinite(b2)) {
            set_err(st, ERRB_NAN);
            go = 0;
        } else if (broke) {
            go = 1;                  // one product measures the residual of x
        } else if (bn == 0.0) {
            st->status = LS_OK;
            st->rnorm = st->true_rnorm = 0.0;
            go = 0;
        }
        set_cond(st, h_loop, go);
    }
}

// After the Jacobi GEMV: x = x_next unless its last CTA stopped the loop
// (then x keeps the iterate whose residual was measured).
__global__ void __launch_bounds__(KB) ja_next_kernel(Vecs v, cudaGraphConditionalHandle h_loop) {
    State *st = v.st;
    count_launch(st);
    const int stop = *(volatile int *)&st->skip || st->err;
    if (!stop) {
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < v.n;
             i += (long long)gridDim.x * blockDim.x)
            v.x[i] = v.q[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(st, h_loop, stop ? 0u : 1u);
}

KrylovKernels krylov_kernels(int num_sms) {
    KrylovKernels K{};
    K.cg_init = reinterpret_cast<void *>(&cg_init_kernel);
    K.cg_update = reinterpret_cast<void *>(&cg_update_kernel);
    K.cg_check = reinterpret_cast<void *>(&cg_check_kernel);
    K.bs_init = reinterpret_cast<void *>(&bs_init_kernel);
    K.bs_s = reinterpret_cast<void *>(&bs_s_kernel);
    K.bs_update = reinterpret_cast<void *>(&bs_update_kernel);
    K.bs_check = reinterpret_cast<void *>(&bs_check_kernel);
    K.gm_init = reinterpret_cast<void *>(&gm_init_kernel);
    K.gm_start = reinterpret_cast<void *>(&gm_start_kernel);
    K.gm_arnoldi = reinterpret_cast<void *>(&gm_arnoldi_kernel);
    K.gm_finish = reinterpret_cast<void *>(&gm_finish_kernel);
    K.ja_diag = reinterpret_cast<void *>(&ja_diag_kernel);
    K.ja_init = reinterpret_cast<void *>(&ja_init_kernel);
    K.ja_next = reinterpret_cast<void *>(&ja_next_kernel);
    K.block = KB;
    K.coop_grid = num_sms;   // one block per SM: always co-resident
    return K;
}

}  // namespace lsi
