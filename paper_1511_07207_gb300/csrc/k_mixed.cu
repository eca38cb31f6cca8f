// k_mixed.cu -- kernels of the mixed-precision solve: A is stored in BF16,
// FP8-e4m3 (+ FP32 row scales) or FP32; an FP32 conjugate gradient on the
// stored matrix is the inner solver; the outer loop runs in FP64 on the FP64
// matrix and is driven by the FP64 residual.  This extends the paper's
// single / double precision axis (section "Results": every solver in both
// precisions) to the low-precision storage formats of GB300.
//
//   mx_init     x = 0 (or x0 via the residual GEMV), r = b - A x, ||b||, ||r||
//   in_init     rhs = r / ||r|| in FP32, z = 0, p = rhs, rho = rhs.rhs
//   (GEMV)      q = Ahat p in FP32 with FP32 accumulation, p.q -> alpha
//   in_update   z += alpha p, r_in -= alpha q, rho', beta, p = r_in + beta p
//   fcg_project flexible CG: z64 = ||r|| z; p_k = z64 - sum_j (z64.w_j / d_j) p_j
//               (full A-orthogonalisation against the stored directions)
//   (GEMV)      w_k = A p_k in FP64, d_k = p_k.w_k
//   fcg_update  alpha = p_k.r / d_k, x += alpha p_k, r -= alpha w_k, ||r||
//   mx_check    accept on the true FP64 residual, or continue from it
//   ir_start / ir_update  classic refinement: r = b - A x, x += ||r|| z.
#include <cuda_runtime.h>

#include "ls_device.cuh"
#include "ls_internal.h"

namespace lsi {

constexpr int MB = 256;
constexpr int SLOT_PR = PART_SLOTS - 1;   // p_k . r, published by fcg_project

__device__ __forceinline__ double reduce_slot_m(const double *part, int slot, int G) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < G; b += 32) s += __ldcg(&part[(size_t)slot * G + b]);
    return warp_sum(s);
}
__device__ __forceinline__ void publish_m(double *part, int slot, double v) {
    if (threadIdx.x == 0) part[(size_t)slot * gridDim.x + blockIdx.x] = v;
}
// every block reduces `slot` and gets the total
__device__ __forceinline__ double all_reduce_slot(const double *part, int slot) {
    __shared__ double t_s;
    if (threadIdx.x < 32) {
        const double t = reduce_slot_m(part, slot, gridDim.x);
        if (threadIdx.x == 0) t_s = t;
    }
    __syncthreads();
    const double t = t_s;
    __syncthreads();
    return t;
}

// x0 = 0: r = b.  x0 given: the residual GEMV has written r = b - A x0.
__global__ void __launch_bounds__(MB) mx_init_kernel(MixVecs v, int x0_given,
                                                     cudaGraphConditionalHandle h_super,
                                                     cudaGraphConditionalHandle h_outer) {
    __shared__ double red[MB / 32];
    State *st = v.st;
    count_launch(st);
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    double bb = 0.0, rr = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double bi = v.b[i];
        if (!x0_given) {
            v.x[i] = 0.0;
            v.r[i] = bi;
        }
        const double ri = v.r[i];
        bb += bi * bi;
        rr += ri * ri;
    }
    bb = block_sum(bb, red);
    rr = block_sum(rr, red);
    publish_m(v.part, 0, bb);
    publish_m(v.part, 1, rr);
    if (!grid_sync(v.bar, st)) return;
    const double b2 = all_reduce_slot(v.part, 0);
    const double r2 = all_reduce_slot(v.part, 1);
    if (b2 == 0.0 && x0_given)
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) v.x[i] = 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double bn = sqrt(b2);
        st->bnorm = bn;
        st->tol_abs = v.rtol * bn;
        st->rnorm = sqrt(r2);
        st->true_rnorm = sqrt(r2);
        int go = 1;
        if (!isfinite(b2) || !isfinite(r2)) {
            set_err(st, ERRB_NAN);
            go = 0;
        } else if (bn == 0.0 || sqrt(r2) <= st->tol_abs) {
            st->status = LS_OK;
            go = 0;
        } else if (st->max_outer <= 0) {
            st->status = LS_NOT_CONVERGED;
            go = 0;
        }
        set_cond(v.st, h_super, go);
        set_cond(v.st, h_outer, go);
    }
}

// Inner right-hand side r / ||r|| in FP32; z = 0; p = rhs; rho = rhs.rhs.
__device__ __forceinline__ void inner_setup(const MixVecs &v, double rn, double *red,
                                            cudaGraphConditionalHandle h_inner) {
    State *st = v.st;
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    float acc = 0.0f;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const float f = (float)(v.r[i] / rn);
        v.rf[i] = f;
        v.pf[i] = f;
        v.zf[i] = 0.0f;
        acc = fmaf(f, f, acc);
    }
    const double t = block_sum((double)acc, red);
    publish_m(v.part, 2, t);
    if (!grid_sync(v.bar, st)) return;
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        const double rho = reduce_slot_m(v.part, 2, gridDim.x);
        if (threadIdx.x == 0) {
            st->in_rho = rho;
            st->in_rho0 = rho;
            st->in_iter = 0;
            st->in_stop = 0;
            st->in_tol2 = st->in_tol2 > 0.0f ? st->in_tol2 : -1.0f;
            set_cond(v.st, h_inner, st->in_max > 0 && rho > 0.0);
        }
    }
}

__global__ void __launch_bounds__(MB) in_init_kernel(MixVecs v, cudaGraphConditionalHandle h_inner) {
    __shared__ double red[MB / 32];
    count_launch(v.st);
    const double rn = v.st->rnorm;
    inner_setup(v, rn, red, h_inner);
}

// One FP32 CG step on the stored matrix (alpha comes from the GEMV's last CTA).
__global__ void __launch_bounds__(MB) in_update_kernel(MixVecs v, cudaGraphConditionalHandle h_inner) {
    __shared__ double red[MB / 32];
    State *st = v.st;
    count_launch(st);
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    if (st->in_stop == 2) {   // p.Ahat p <= 0: keep the iterate (the rhs itself on step 0)
        if (st->in_iter == 0)
            for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) v.zf[i] = v.pf[i];
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(v.st, h_inner, 0);
        return;
    }
    const float alpha = (float)st->in_alpha;
    const double rho = st->in_rho;
    const int it = st->in_iter;
    float acc = 0.0f;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        v.zf[i] = fmaf(alpha, v.pf[i], v.zf[i]);
        const float ri = fmaf(-alpha, v.qf[i], v.rf[i]);
        v.rf[i] = ri;
        acc = fmaf(ri, ri, acc);
    }
    const double t = block_sum((double)acc, red);
    publish_m(v.part, 0, t);
    if (!grid_sync(v.bar, st)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(v.st, h_inner, 0);
        return;
    }
    const double rho_new = all_reduce_slot(v.part, 0);
    const bool stop = !(rho_new > (double)st->in_tol2) || !isfinite(rho_new) ||
                      it + 1 >= st->in_max || rho_new == 0.0;
    if (!stop) {
        const float beta = (float)(rho_new / rho);
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x)
            v.pf[i] = fmaf(beta, v.pf[i], v.rf[i]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->in_rho = rho_new;
        st->in_iter = it + 1;
        if (stop) set_cond(v.st, h_inner, 0);
    }
}

// Flexible-CG direction: z64 = ||r|| z into column k of P, then
// p_k = z64 - sum_j (z64 . w_j / d_j) p_j; publishes p_k . r.
__global__ void __launch_bounds__(MB) fcg_project_kernel(MixVecs v) {
    __shared__ double red[MB / 32];
    __shared__ double coef[LS_MAX_RESTART];
    State *st = v.st;
    count_launch(st);
    const int k = st->nstored;
    const double rn = st->rnorm;
    const int G = gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    long long lo, hi;
    block_range(v.n, blockIdx.x, G, lo, hi);
    double *pk = v.P + (long long)k * v.ldp;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) pk[i] = rn * (double)v.zf[i];
    if (v.mode == LS_REFINE_FCG && k > 0) {
        __syncthreads();
        for (int j = warp; j < k; j += nw) {
            const double *wj = v.W + (long long)j * v.ldp;
            double s = 0.0;
            for (long long i = lo + lane; i < hi; i += 32) s += pk[i] * wj[i];
            s = warp_sum(s);
            if (lane == 0) v.part[(size_t)j * G + blockIdx.x] = s;
        }
        if (!grid_sync(v.bar, st)) return;
        for (int j = warp; j < k; j += nw) {
            const double t = reduce_slot_m(v.part, j, G);
            if (lane == 0) coef[j] = t / __ldcg(&v.dvals[j]);
        }
        __syncthreads();
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            double pi = pk[i];
            for (int j = 0; j < k; j++) pi -= coef[j] * v.P[(long long)j * v.ldp + i];
            pk[i] = pi;
        }
    }
    double pr = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) pr += pk[i] * v.r[i];
    pr = block_sum(pr, red);
    publish_m(v.part, SLOT_PR, pr);
}

// alpha = p.r / p.Ap; x += alpha p; r -= alpha w; ||r||; outer loop control.
__global__ void __launch_bounds__(MB) fcg_update_kernel(MixVecs v, cudaGraphConditionalHandle h_outer) {
    __shared__ double red[MB / 32];
    State *st = v.st;
    count_launch(st);
    const int k = st->nstored;
    const double d = st->pq;
    const double pr = all_reduce_slot(v.part, SLOT_PR);
    if (!(d > 0.0) || !isfinite(pr)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->status = LS_BREAKDOWN;
            if (!isfinite(pr) || !(d == d)) set_err(st, ERRB_NAN);
            set_cond(v.st, h_outer, 0);
        }
        return;
    }
    const double alpha = pr / d;
    const double *pk = v.P + (long long)k * v.ldp;
    const double *wk = v.W + (long long)k * v.ldp;
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    double rr = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        v.x[i] += alpha * pk[i];
        const double ri = v.r[i] - alpha * wk[i];
        v.r[i] = ri;
        rr += ri * ri;
    }
    rr = block_sum(rr, red);
    publish_m(v.part, 0, rr);
    if (!grid_sync(v.bar, st)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(v.st, h_outer, 0);
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        const double r2 = reduce_slot_m(v.part, 0, gridDim.x);
        if (threadIdx.x == 0) {
            const double rn = sqrt(r2);
            v.dvals[k] = d;
            st->nstored = k + 1;
            st->outer += 1;
            st->iter += st->in_iter;
            st->rnorm = rn;
            const bool finite = isfinite(r2);
            if (!finite) set_err(st, ERRB_NAN);
            if (!finite || rn <= st->tol_abs || st->outer >= st->max_outer ||
                st->nstored >= st->m)
                set_cond(v.st, h_outer, 0);
        }
    }
}

// After the outer loop: q = b - A x and true_rnorm come from the residual GEMV.
__global__ void __launch_bounds__(MB) mx_check_kernel(MixVecs v, cudaGraphConditionalHandle h_super,
                                                      cudaGraphConditionalHandle h_outer) {
    State *st = v.st;
    count_launch(st);
    const double t = st->true_rnorm;
    int decision;   // 0 accept, 1 limit, 2 breakdown/error, 3 continue from the true residual
    if (st->err || !isfinite(t)) decision = 2;
    else if (st->status == LS_BREAKDOWN) decision = 2;
    else if (t <= st->tol_abs) decision = 0;
    else if (st->outer >= st->max_outer) decision = 1;
    else decision = 3;
    if (decision == 3) {
        long long lo, hi;
        block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) v.r[i] = v.q[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (decision == 0) st->status = LS_OK;
        if (decision == 1) st->status = LS_NOT_CONVERGED;
        if (decision == 2 && !isfinite(t)) set_err(st, ERRB_NAN);
        if (decision == 3) {
            st->rnorm = t;
            // the stored directions stay A-conjugate; only the storage can run out
            if (st->nstored >= st->m) st->nstored = 0;
        }
        st->cycles += 1;
        set_cond(v.st, h_super, decision == 3);
        set_cond(v.st, h_outer, decision == 3);
    }
}

// Classic refinement: the residual GEMV wrote r = b - A x and ||r||.
__global__ void __launch_bounds__(MB) ir_start_kernel(MixVecs v, cudaGraphConditionalHandle h_outer,
                                                      cudaGraphConditionalHandle h_inner) {
    __shared__ double red[MB / 32];
    State *st = v.st;
    count_launch(st);
    const double t = st->true_rnorm;
    int go;
    if (st->err || !isfinite(t)) go = -1;
    else if (t <= st->tol_abs) go = 0;
    else if (st->outer >= st->max_outer) go = -2;
    else go = 1;
    if (go != 1) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (go == -1) set_err(st, ERRB_NAN);
            if (go == 0) st->status = LS_OK;
            if (go == -2) st->status = LS_NOT_CONVERGED;
            st->rnorm = t;
            st->in_stop = 3;      // no step this time: ir_update must not apply z again
            set_cond(v.st, h_outer, 0);
            set_cond(v.st, h_inner, 0);
        }
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) st->rnorm = t;
    inner_setup(v, t, red, h_inner);
}

__global__ void __launch_bounds__(MB) ir_update_kernel(MixVecs v) {
    State *st = v.st;
    count_launch(st);
    if (st->err || st->in_stop == 3) return;
    const double rn = st->rnorm;
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) v.x[i] += rn * (double)v.zf[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->outer += 1;
        st->iter += st->in_iter;
    }
}

MixedKernels mixed_kernels() {
    MixedKernels K{};
    K.mx_init = reinterpret_cast<void *>(&mx_init_kernel);
    K.in_init = reinterpret_cast<void *>(&in_init_kernel);
    K.in_update = reinterpret_cast<void *>(&in_update_kernel);
    K.fcg_project = reinterpret_cast<void *>(&fcg_project_kernel);
    K.fcg_update = reinterpret_cast<void *>(&fcg_update_kernel);
    K.mx_check = reinterpret_cast<void *>(&mx_check_kernel);
    K.ir_start = reinterpret_cast<void *>(&ir_start_kernel);
    K.ir_update = reinterpret_cast<void *>(&ir_update_kernel);
    return K;
}

}  // namespace lsi
