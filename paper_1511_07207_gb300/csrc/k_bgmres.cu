// k_bgmres.cu -- restarted block GMRES(m) for s right-hand sides.
//
// Block GMRES (the GMRES pseudocode and restart paragraph of the paper, with
// a block Arnoldi process over the s right-hand sides at once).  A cycle:
//   the block product writes A X into V's first block;
//   bgm_start  R = B - A X there and ||R_c||^2; stop if every column passes;
//              else V_1 S = R by CholQR2 (two
//              passes of Gram matrix, Cholesky, triangular solve per row),
//              G = [S; 0]; when R is rank-deficient (a Cholesky pivot at
//              most 1e-12 of its diagonal entry) and deflation is on, its
//              dependent columns (found in column order) are replaced by
//              fixed pseudo-random vectors, V_1 is the CholQR2 of that block
//              and S = V_1^T R (deflate_start);
//   per block step j (graph while-node): P split + block product W = A V_j
//              (k_bgemv.cu, A read once for all s columns), then bgm_orth:
//              two passes of block classical Gram-Schmidt against V_1..V_j
//              (partial Gram matrices per CTA, reduced in CTA order, spread
//              over the CTAs), V_{j+1} H_{j+1,j} = W by CholQR2 (a block that
//              loses rank ends the cycle with a zero block), then one warp
//              applies the cycle's earlier Givens rotations to the s new
//              columns of the band Hessenberg matrix (a lane a column), makes
//              s rotations per column from the bottom up, rotates G (a lane a
//              right-hand side) and tests ||G[k:k+s, c]|| <= rtol ||B_c||;
//   bgm_finish back substitution R Y = G (a warp a right-hand side, column
//              oriented) and X += V Y.
// All of it FP64; every grid barrier is bounded; every decision is taken
// from values all CTAs read after a barrier, so they agree.
#include <cuda_runtime.h>

#include "ls_device.cuh"
#include "ls_internal.h"

namespace lsi {

namespace {

constexpr int GT = 256;   // threads per CTA

__device__ __forceinline__ int ldh(const BgmVecs &v) { return (v.m + 1) * v.s; }

// This CTA's partial U^T M (U: ku columns, M: s columns, rows [lo, hi)).
// When there are fewer entries than threads, T = GT / (ku s) threads share
// an entry, thread q summing rows lo + q, lo + q + T, ..., their sums added
// in q order (all threads of the CTA call it; a warp's FP64 instruction
// takes about 64 cycles of its scheduler's FP64 unit on this GPU, so the
// work is spread over all warps).
__device__ void gram_part(const BgmVecs &v, const double *U, int ku, const double *M, long long lo, long long hi) {
    __shared__ double red[GT];
    const int s = v.s, E = ku * s;
    if (E >= GT) {
        for (int e = threadIdx.x; e < E; e += blockDim.x) {
            const int a = e % ku, b = e / ku;
            const double *u = U + (long long)a * v.ld, *w = M + (long long)b * v.ld;
            double t0 = 0.0, t1 = 0.0;
            long long i = lo;
            for (; i + 1 < hi; i += 2) {
                t0 += u[i] * w[i];
                t1 += u[i + 1] * w[i + 1];
            }
            if (i < hi) t0 += u[i] * w[i];
            v.part[(size_t)blockIdx.x * v.part_stride + e] = t0 + t1;
        }
        return;
    }
    const int T = GT / E;
    const int e = threadIdx.x / T, q = threadIdx.x - e * T;
    double acc = 0.0;
    if (e < E) {
        const int a = e % ku, b = e / ku;
        const double *u = U + (long long)a * v.ld, *w = M + (long long)b * v.ld;
        for (long long i = lo + q; i < hi; i += T) acc += u[i] * w[i];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    if (e < E && q == 0) {
        double sum = 0.0;
        for (int t = 0; t < T; t++) sum += red[threadIdx.x + t];
        v.part[(size_t)blockIdx.x * v.part_stride + e] = sum;
    }
    __syncthreads();
}

// The sum over the CTAs of entry e of the partial Gram matrices: eight
// interleaved sums (CTA c into sum c % 8) added pairwise; a fixed order.
__device__ __forceinline__ double cta_sum(const BgmVecs &v, int e) {
    double t[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const int nc = (int)gridDim.x;
    for (int c = 0; c < nc; c++) t[c & 7] += __ldcg(&v.part[(size_t)c * v.part_stride + e]);
    return ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
}

// Entries of the reduced Gram matrix spread over the CTAs, into out[0 .. cnt).
__device__ void gram_reduce_spread(const BgmVecs &v, int cnt, double *out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) out[e] = cta_sum(v, e);
}

// One warp: G = L L^T in place (column-major s x s).  False when a pivot is
// at most 1e-12 of its diagonal entry: the squared norm of the column's part
// orthogonal to the earlier ones carries an absolute rounding error of about
// u G_jj, so a Gram-matrix QR cannot tell an orthogonal part below about
// 1e-6 of the column from zero -- the block is treated as rank-deficient.
__device__ bool warp_chol(int s, double *G) {
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < s; j++) {
        const double gjj = G[j + j * s];
        double d = gjj;
        for (int k = 0; k < j; k++) d -= G[j + k * s] * G[j + k * s];
        if (!(d > 1e-12 * gjj) || !isfinite(d)) return false;
        d = sqrt(d);
        __syncwarp();
        if (lane > j && lane < s) {
            double x = G[lane + j * s];
            for (int k = 0; k < j; k++) x -= G[lane + k * s] * G[j + k * s];
            G[lane + j * s] = x / d;
        }
        if (lane == 0) G[j + j * s] = d;
        __syncwarp();
    }
    return true;
}

// One CholQR pass on the n x s block M: M = Q L^T with Q over M's rows; the
// factor L goes to v.Lm.  All CTAs; returns 1 on success, 0 when the Gram
// matrix is not positive definite (every CTA agrees), -1 on a barrier
// timeout.
__device__ int cholqr_pass(const BgmVecs &v, double *M, long long lo, long long hi) {
    __shared__ double Gs[BGM_MAX_S * BGM_MAX_S];
    const int s = v.s;
    gram_part(v, M, s, M, lo, hi);
    if (!grid_sync(v.bar, v.st)) return -1;
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        for (int e = threadIdx.x; e < s * s; e += 32) Gs[e] = cta_sum(v, e);
        __syncwarp();
        const bool ok = warp_chol(s, Gs);
        for (int e = threadIdx.x; e < s * s; e += 32) v.Lm[e] = Gs[e];
        if (threadIdx.x == 0) v.flags[BGF_CHOL] = ok ? 1 : 0;
    }
    if (!grid_sync(v.bar, v.st)) return -1;
    if (!*(volatile int *)&v.flags[BGF_CHOL]) return 0;
    __shared__ double L[BGM_MAX_S * BGM_MAX_S];
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) L[e] = __ldcg(&v.Lm[e]);
    __syncthreads();
    // each row m: solve y L^T = m (y_j = (m_j - sum_{i<j} y_i L_ji) / L_jj)
    for (long long r = lo + threadIdx.x; r < hi; r += blockDim.x) {
        double y[BGM_MAX_S];
#pragma unroll
        for (int j = 0; j < BGM_MAX_S; j++) {
            if (j >= s) break;
            double x = M[(long long)j * v.ld + r];
            for (int i = 0; i < j; i++) x -= y[i] * L[j + i * s];
            y[j] = x / L[j + j * s];
            M[(long long)j * v.ld + r] = y[j];
        }
    }
    __syncthreads();
    return 1;
}

// One warp: the dependent columns of the s x s Gram matrix G of a block, in
// column order.  The Cholesky factorisation of warp_chol, except that a
// column whose pivot is at most 1e-12 of its diagonal entry (its part
// orthogonal to the columns kept before it has at most 1e-6 of its norm) is
// marked dead[j] = 1 and its column of the factor set to zero, so that it
// takes no part in the later columns.
__device__ void warp_chol_skip(int s, double *G, int *dead) {
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < s; j++) {
        const double gjj = G[j + j * s];
        double d = gjj;
        for (int k = 0; k < j; k++) d -= G[j + k * s] * G[j + k * s];
        const bool dj = !(d > 1e-12 * gjj) || !isfinite(d);
        __syncwarp();
        if (dj) {
            if (lane < s) G[lane + j * s] = 0.0;
        } else {
            d = sqrt(d);
            if (lane > j && lane < s) {
                double x = G[lane + j * s];
                for (int k = 0; k < j; k++) x -= G[lane + k * s] * G[j + k * s];
                G[lane + j * s] = x / d;
            }
            if (lane == 0) G[j + j * s] = d;
        }
        if (lane == 0) dead[j] = dj ? 1 : 0;
        __syncwarp();
    }
}

// Output k (counted from 0) of SplitMix64 seeded with 0 (Steele, Lea and
// Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
// the state after k + 1 steps of its Weyl sequence, then its mixing function.
__device__ __forceinline__ unsigned long long splitmix64_out(unsigned long long k) {
    unsigned long long x = (k + 1ull) * 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Entry i of the vector that replaces dependent column c of a starting
// block: 2 u - 1, u = the top 53 bits of output c 2^32 + i over 2^53.
__device__ __forceinline__ double replacement_entry(int c, long long i) {
    const unsigned long long k = ((unsigned long long)c << 32) | (unsigned long long)i;
    const double u = (double)(splitmix64_out(k) >> 11) * 0x1.0p-53;
    return __dsub_rn(__dmul_rn(2.0, u), 1.0);
}

// T = R2 R1 for upper-triangular R = L^T factors (block 0, one warp):
// R1 (from the first pass) is kept in R; R2 is v.Lm^T.  Column-major s x s.
__device__ void combine_r(const BgmVecs &v, double *R) {
    const int s = v.s;
    __shared__ double T[BGM_MAX_S * BGM_MAX_S];
    for (int e = threadIdx.x & 31; e < s * s; e += 32) {
        const int i = e % s, j = e / s;   // T_ij = sum_k R2_ik R1_kj, R2_ik = Lm_ki
        double acc = 0.0;
        for (int k = i; k <= j; k++) acc += v.Lm[k + i * s] * R[k + j * s];
        T[e] = acc;
    }
    __syncwarp();
    for (int e = threadIdx.x & 31; e < s * s; e += 32) R[e] = T[e];
    __syncwarp();
}

__device__ __forceinline__ void stop_both(State *st, cudaGraphConditionalHandle ho, cudaGraphConditionalHandle hi) {
    set_cond(st, ho, 0u);
    set_cond(st, hi, 0u);
}

// V_1 S = R for a rank-deficient R (V's first block), called by every CTA
// right after a CholQR pass over R found a pivot at most 1e-12 of its
// diagonal entry (R's partial Gram matrices are still in v.part):
//   the dependent columns, in column order (warp_chol_skip);
//   R kept in W, each dependent column of V's first block replaced by its
//   replacement vector (replacement_entry);
//   V_1 by CholQR2 of that block;
//   S = V_1^T R into G's first s rows, G's other rows zero.
// R = V_1 S then holds for every column up to the dependent columns'
// remainders (at most 1e-6 of their norms); the block Krylov space grows
// from the kept directions and the replacements.  Returns 1 on success, 0
// when the block with the replacements is still rank-deficient (every CTA
// agrees), -1 on a barrier timeout.
__device__ int deflate_start(const BgmVecs &v, long long lo, long long hi) {
    __shared__ double Gs[BGM_MAX_S * BGM_MAX_S];
    __shared__ int dd[BGM_MAX_S];
    const int s = v.s;
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        for (int e = threadIdx.x; e < s * s; e += 32) Gs[e] = cta_sum(v, e);
        __syncwarp();
        warp_chol_skip(s, Gs, dd);
        __syncwarp();
        if (threadIdx.x < s) v.dead[threadIdx.x] = dd[threadIdx.x];
    }
    if (!grid_sync(v.bar, v.st)) return -1;
    if (threadIdx.x < s) dd[threadIdx.x] = __ldcg(&v.dead[threadIdx.x]);
    __syncthreads();
    for (int c = 0; c < s; c++)
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const long long o = (long long)c * v.ld + i;
            v.W[o] = v.V[o];
            if (dd[c]) v.V[o] = replacement_entry(c, i);
        }
    __syncthreads();
    int ok = cholqr_pass(v, v.V, lo, hi);
    if (ok <= 0) return ok;
    ok = cholqr_pass(v, v.V, lo, hi);
    if (ok <= 0) return ok;
    gram_part(v, v.V, s, v.W, lo, hi);              // entry q + c s: V_q . R_c
    if (!grid_sync(v.bar, v.st)) return -1;
    if (blockIdx.x == 0) {
        const int L = ldh(v);
        for (int e = threadIdx.x; e < L * s; e += blockDim.x) {
            const int q = e % L, c = e / L;
            v.G[e] = q < s ? cta_sum(v, q + c * s) : 0.0;
        }
    }
    return 1;
}

}  // namespace

// ---- init: X = 0 (or X0), ||B_c|| -------------------------------------------------------
__global__ void __launch_bounds__(GT) bgm_init_kernel(BgmVecs v, int x0_given, cudaGraphConditionalHandle h_outer,
                                                      cudaGraphConditionalHandle h_inner) {
    State *st = v.st;
    count_launch(st);
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    const int s = v.s;
    if (!x0_given)
        for (int c = 0; c < s; c++)
            for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) v.X[(long long)c * v.ld + i] = 0.0;
    for (int c = threadIdx.x; c < s; c += blockDim.x) {
        const double *b = v.B + (long long)c * v.ld;
        double acc = 0.0;
        for (long long i = lo; i < hi; i++) acc += b[i] * b[i];
        v.part[(size_t)blockIdx.x * v.part_stride + c] = acc;
    }
    if (!grid_sync(v.bar, st)) return;
    if (blockIdx.x == 0 && threadIdx.x < s) {
        const double acc = cta_sum(v, threadIdx.x);
        v.bn[threadIdx.x] = sqrt(acc);
        if (!isfinite(acc)) set_err(st, ERRB_NAN);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        set_cond(st, h_outer, 1u);
        set_cond(st, h_inner, 0u);
    }
}

// ---- start of a cycle (after the residual GEMVs) -------------------------------------------------
__global__ void __launch_bounds__(GT) bgm_start_kernel(BgmVecs v, cudaGraphConditionalHandle h_outer,
                                                       cudaGraphConditionalHandle h_inner) {
    __shared__ int decide_s;
    __shared__ double R[BGM_MAX_S * BGM_MAX_S];
    State *st = v.st;
    count_launch(st);
    const int s = v.s;
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    // R = B - A X in V's first block (A X from the block product), ||R_c||^2
    for (int c = 0; c < s; c++)
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const long long o = (long long)c * v.ld + i;
            v.V[o] = v.B[o] - v.V[o];
        }
    __syncthreads();
    for (int c = threadIdx.x; c < s; c += blockDim.x) {
        const double *r = v.V + (long long)c * v.ld;
        double acc = 0.0;
        for (long long i = lo; i < hi; i++) acc += r[i] * r[i];
        v.part[(size_t)blockIdx.x * v.part_stride + c] = acc;
    }
    if (!grid_sync(v.bar, st)) return;
    if (threadIdx.x == 0) {
        bool pass = true, nan = false;
        for (int c = 0; c < s; c++) {
            double r2 = 0.0;
            for (int b = 0; b < (int)gridDim.x; b++) r2 += __ldcg(&v.part[(size_t)b * v.part_stride + c]);
            if (blockIdx.x == 0) v.r2[c] = r2;
            nan = nan || !isfinite(r2);
            pass = pass && sqrt(r2) <= v.rtol * v.bn[c];
        }
        int d = 0;   // 0 run a cycle, 1 stop
        if (*(volatile int *)&st->err || nan) {
            if (nan) set_err(st, ERRB_NAN);
            d = 1;
        } else if (*(volatile int *)&st->status == LS_BREAKDOWN) {
            d = 1;
        } else if (pass) {
            if (blockIdx.x == 0) st->status = LS_OK;
            d = 1;
        } else if (*(volatile int *)&st->iter >= st->max_iter) {
            if (blockIdx.x == 0) st->status = LS_NOT_CONVERGED;
            d = 1;
        }
        decide_s = d;
    }
    __syncthreads();
    if (decide_s) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->k = 0;   // bgm_finish has nothing to add
            stop_both(st, h_outer, h_inner);
        }
        return;
    }
    // V_1 S = R (CholQR2); a rank-deficient block is deflated (deflate_start)
    // or, without deflation, a breakdown
    int ok = cholqr_pass(v, v.V, lo, hi);
    if (ok < 0) return;
    const bool deflated = !ok && v.deflate;
    if (deflated) {
        ok = deflate_start(v, lo, hi);
        if (ok < 0) return;
    } else {
        if (ok && blockIdx.x == 0 && threadIdx.x < 32) {
            for (int e = threadIdx.x; e < s * s; e += 32) {
                const int i = e % s, j = e / s;
                R[e] = i <= j ? v.Lm[j + i * s] : 0.0;   // R1 = L^T
            }
            __syncwarp();
        }
        if (ok) ok = cholqr_pass(v, v.V, lo, hi);
        if (ok < 0) return;
    }
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        if (ok && !deflated) {
            combine_r(v, R);
            const int L = ldh(v);
            for (int e = threadIdx.x; e < L * s; e += 32) v.G[e] = 0.0;
            __syncwarp();
            for (int e = threadIdx.x; e < s * s; e += 32) v.G[(e / s) * L + (e % s)] = R[e];
        }
        if (threadIdx.x == 0) {
            if (!ok) {
                st->status = LS_BREAKDOWN;
                st->k = 0;
                stop_both(st, h_outer, h_inner);
            } else {
                st->cycles++;
                st->k = 0;
                v.flags[BGF_NROT] = 0;
                v.flags[BGF_LUCKY] = 0;
                set_cond(st, h_inner, 1u);
                set_cond(st, h_outer, 1u);
            }
        }
    }
}

// ---- one block step after W = A V_j ----------------------------------------------------------------
__global__ void __launch_bounds__(GT) bgm_orth_kernel(BgmVecs v, cudaGraphConditionalHandle h_inner) {
    extern __shared__ __align__(16) double dsm[];
    __shared__ double R[BGM_MAX_S * BGM_MAX_S];
    State *st = v.st;
    count_launch(st);
    const int s = v.s, L = ldh(v);
    const int j = *(volatile int *)&st->k, kc = (j + 1) * s;
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    double *Hs = dsm;   // kc x s reduced coefficients (each CTA's copy)
    // two passes of block classical Gram-Schmidt against V[:, 0:kc]
    for (int pass = 0; pass < 2; pass++) {
        gram_part(v, v.V, kc, v.W, lo, hi);
        if (!grid_sync(v.bar, st)) return;
        gram_reduce_spread(v, kc * s, v.Hc);
        if (!grid_sync(v.bar, st)) return;
        for (int e = threadIdx.x; e < kc * s; e += blockDim.x) Hs[e] = __ldcg(&v.Hc[e]);
        __syncthreads();
        if (blockIdx.x == 0)
            for (int e = threadIdx.x; e < kc * s; e += blockDim.x) {
                const int q = e % kc, c = e / kc;
                double *h = &v.H[(long long)(j * s + c) * L + q];
                *h = (pass == 0 ? 0.0 : *h) + Hs[e];
            }
        for (long long r = lo + threadIdx.x; r < hi; r += blockDim.x) {
            double w[BGM_MAX_S];
#pragma unroll
            for (int c = 0; c < BGM_MAX_S; c++) w[c] = c < s ? v.W[(long long)c * v.ld + r] : 0.0;
            for (int q = 0; q < kc; q++) {
                const double vq = v.V[(long long)q * v.ld + r];
#pragma unroll
                for (int c = 0; c < BGM_MAX_S; c++)
                    if (c < s) w[c] -= vq * Hs[q + c * kc];
            }
#pragma unroll
            for (int c = 0; c < BGM_MAX_S; c++)
                if (c < s) v.W[(long long)c * v.ld + r] = w[c];
        }
        __syncthreads();
    }
    // V_{j+1} H_{j+1,j} = W (CholQR2); a block that lost rank ends the cycle
    int ok = cholqr_pass(v, v.W, lo, hi);
    if (ok < 0) return;
    if (ok && blockIdx.x == 0 && threadIdx.x < 32) {
        for (int e = threadIdx.x; e < s * s; e += 32) {
            const int i = e % s, jj = e / s;
            R[e] = i <= jj ? v.Lm[jj + i * s] : 0.0;
        }
        __syncwarp();
    }
    if (ok) ok = cholqr_pass(v, v.W, lo, hi);
    if (ok < 0) return;
    for (int c = 0; c < s; c++)
        for (long long r = lo + threadIdx.x; r < hi; r += blockDim.x)
            v.V[(long long)(kc + c) * v.ld + r] = ok ? v.W[(long long)c * v.ld + r] : 0.0;
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;

    // ---- block 0, warp 0: the Hessenberg block column and the rotations ----
    const int lane = threadIdx.x;
    if (ok) combine_r(v, R);
    double *Hb = dsm;                   // (kc + s) x s, column-major, leading dimension kc + s
    double *Gs = Hb + (kc + s) * s;     // L x s, leading dimension L
    const int lb = kc + s;
    for (int e = lane; e < lb * s; e += 32) {
        const int q = e % lb, c = e / lb;
        double x;
        if (q < kc) x = v.H[(long long)(j * s + c) * L + q];
        else x = (ok && q - kc <= c) ? R[(q - kc) + c * s] : 0.0;
        Hb[e] = x;
    }
    for (int e = lane; e < L * s; e += 32) Gs[e] = v.G[e];
    __syncwarp();
    int nrot = v.flags[BGF_NROT];
    // earlier rotations on each new column (a lane a column)
    if (lane < s) {
        double *h = Hb + (long long)lane * lb;
        for (int t = 0; t < nrot; t++) {
            const int r = v.rrow[t];
            const double cc = v.cs[t], ss = v.sn[t];
            const double a = h[r], b = h[r + 1];
            h[r] = cc * a + ss * b;
            h[r + 1] = -ss * a + cc * b;
        }
    }
    __syncwarp();
    bool broke = false;
    for (int c = 0; c < s; c++) {
        const int col = j * s + c;
        for (int r = col + s - 1; r >= col; r--) {       // zero row r + 1 of column c
            const double a = Hb[r + c * lb], b = Hb[r + 1 + c * lb];
            const double den = hypot(a, b);
            const double cc = den > 0.0 ? a / den : 1.0, ss = den > 0.0 ? b / den : 0.0;
            __syncwarp();
            if (lane >= c && lane < s) {                   // columns c .. s-1 of the block
                double *h = Hb + (long long)lane * lb;
                const double x = h[r], y = h[r + 1];
                h[r] = cc * x + ss * y;
                h[r + 1] = -ss * x + cc * y;
            }
            if (lane < s) {                                 // G, a lane a right-hand side
                double *g = Gs + (long long)lane * L;
                const double x = g[r], y = g[r + 1];
                g[r] = cc * x + ss * y;
                g[r + 1] = -ss * x + cc * y;
            }
            if (lane == 0) {
                v.rrow[nrot] = r;
                v.cs[nrot] = cc;
                v.sn[nrot] = ss;
            }
            nrot++;
            __syncwarp();
        }
        broke = broke || Hb[col + c * lb] == 0.0;
    }
    for (int e = lane; e < lb * s; e += 32) v.H[(long long)(j * s + e / lb) * L + (e % lb)] = Hb[e];
    for (int e = lane; e < L * s; e += 32) v.G[e] = Gs[e];
    // residual estimates ||G[kc+s-? ...]||: rows kc .. kc + s - 1 after this step hold the residual
    bool pass = true;
    if (lane < s) {
        double e2 = 0.0;
        for (int r = kc; r < kc + s; r++) e2 += Gs[r + lane * L] * Gs[r + lane * L];
        pass = sqrt(e2) <= v.rtol * v.bn[lane];
    }
    const bool conv = __all_sync(0xffffffffu, pass);
    if (lane == 0) {
        v.flags[BGF_NROT] = nrot;
        st->iter++;
        st->k = j + 1;
        int go = !conv && ok && (j + 1) < v.m && st->iter < st->max_iter;
        if (broke) {
            st->status = LS_BREAKDOWN;
            go = 0;
        }
        set_cond(st, h_inner, go ? 1u : 0u);
    }
}

// ---- end of a cycle: R Y = G, X += V Y ------------------------------------------------------------
__global__ void __launch_bounds__(GT) bgm_finish_kernel(BgmVecs v) {
    extern __shared__ __align__(16) double dsm[];
    State *st = v.st;
    count_launch(st);
    const int s = v.s, L = ldh(v);
    const int K = *(volatile int *)&st->k * s;
    if (K == 0 || *(volatile int *)&st->status == LS_BREAKDOWN || *(volatile int *)&st->err) return;
    if (blockIdx.x == 0) {
        // one warp a right-hand side: column-oriented back substitution
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        double *g = dsm + (long long)warp * L;
        for (int q = warp; q < s; q += blockDim.x >> 5) {
            for (int r = lane; r < K; r += 32) g[r] = v.G[(long long)q * L + r];
            __syncwarp();
            for (int i = K - 1; i >= 0; i--) {
                const double yi = g[i] / v.H[(long long)i * L + i];
                __syncwarp();
                for (int r = lane; r < i; r += 32) g[r] -= v.H[(long long)i * L + r] * yi;
                if (lane == 0) g[i] = yi;
                __syncwarp();
            }
            for (int r = lane; r < K; r += 32) v.Y[(long long)q * K + r] = g[r];
            __syncwarp();
        }
    }
    if (!grid_sync(v.bar, st)) return;
    double *Ys = dsm;   // K x s
    for (int e = threadIdx.x; e < K * s; e += blockDim.x) Ys[e] = __ldcg(&v.Y[e]);
    __syncthreads();
    long long lo, hi;
    block_range(v.n, blockIdx.x, gridDim.x, lo, hi);
    for (long long r = lo + threadIdx.x; r < hi; r += blockDim.x) {
        double x[BGM_MAX_S];
#pragma unroll
        for (int c = 0; c < BGM_MAX_S; c++) x[c] = 0.0;
        for (int q = 0; q < K; q++) {
            const double vq = v.V[(long long)q * v.ld + r];
#pragma unroll
            for (int c = 0; c < BGM_MAX_S; c++)
                if (c < s) x[c] += vq * Ys[q + c * K];
        }
#pragma unroll
        for (int c = 0; c < BGM_MAX_S; c++)
            if (c < s) v.X[(long long)c * v.ld + r] += x[c];
    }
}

BgmKernels bgm_kernels() {
    BgmKernels K{};
    K.init = reinterpret_cast<void *>(&bgm_init_kernel);
    K.start = reinterpret_cast<void *>(&bgm_start_kernel);
    K.orth = reinterpret_cast<void *>(&bgm_orth_kernel);
    K.finish = reinterpret_cast<void *>(&bgm_finish_kernel);
    K.block = GT;
    return K;
}

size_t bgm_orth_smem(int m, int s) {
    const size_t L = (size_t)(m + 1) * s;
    const size_t coef = (size_t)(m + 1) * s * s;                 // kc x s at most
    const size_t givens = (size_t)(m * s + s) * s + L * s;       // the block column and G
    return sizeof(double) * (coef > givens ? coef : givens);
}

size_t bgm_finish_smem(int m, int s) {
    const size_t L = (size_t)(m + 1) * s;
    const size_t back = (size_t)(GT / 32) * L;                   // a column of G per warp
    const size_t ys = (size_t)m * s * s;                         // Y
    return sizeof(double) * (back > ys ? back : ys);
}

}  // namespace lsi
