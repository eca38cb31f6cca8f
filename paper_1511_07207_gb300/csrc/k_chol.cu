// k_chol.cu -- the paper's Cholesky factorization A = L L^T (FP64) and the
// solve L y = b, L^T x = y.
//
// The paper writes the blocked Cholesky (the direct-methods section, Fig. 3
// and the three block relations after it) as the factorization of a leading
// block, a triangular solve for the block below it and the update of the
// trailing block.  Element by element that is the column-by-column
// factorization: at step k, l_kk = sqrt(w_kk), l_ik = w_ik / l_kk for i > k,
// and w_ij = w_ij - l_ik l_jk for k < j <= i.  b rides along as an extra row
// n of the working matrix W (only its lower triangle is used), so row n
// becomes y = L^-1 b during the factorization: y_k = w_nk / l_kk is the
// forward substitution's division and w_nj -= y_k l_jk its updates, in the
// same order.
//
// Per panel of CH_NB = 32 columns:
// chol_panel_kernel (cooperative, over the panel's steps, its columns only):
//   l_kk from the current w_kk; each row i > k (row n included) belongs to
//   one warp: l_ik = w_ik / l_kk (IEEE division) into the panel buffer Lp,
//   and lane c updates the row's panel column j = k + 1 + c (j <= i) with
//   l_jk = w_jk / l_kk formed by the lane itself from the unchanged column k:
//   w_ij = w_ij - l_ik l_jk as a separate multiply and subtract.  One bounded
//   grid barrier per step; every read of W goes to L2 (ld.global.cg).  After
//   the last step the panel's l's are written into W's panel columns.
// chol_trail_kernel: the trailing lower triangle (rows k1 .. n, columns
//   k1 .. min(i, n - 1)) in 64 x 64 tiles: each element takes the panel's 32
//   updates in order from the panel's l's staged in shared memory (two FP64
//   instructions an element and step: bound by the FP64 pipe).
// chol_backsolve_kernel (cooperative): L^T x = y by blocks of 64 rows from
//   the bottom: CTA 0 solves the diagonal block (one warp), then every CTA
//   subtracts the block's contribution l_ji x_j from the rows above it (a
//   thread a row, reading the block's rows of L, which are contiguous).
// So L and y are bit for bit those of the plain column factorization and
// forward substitution; x differs from a scalar back substitution by the
// order of its sums.
//
// Work: n^3 / 6 updates of two FP64 instructions (half of the LU's).
#include <cuda_runtime.h>

#include "ls_device.cuh"
#include "ls_internal.h"

namespace lsi {

namespace {
constexpr int CT = 512;            // threads per CTA of the cooperative kernels (16 warps)
constexpr int CW = CT / 32;
constexpr int CH_NB = 32;          // panel width
constexpr int CH_ROWS = 4;         // rows a warp loads before it computes
constexpr int CTT = 64;            // trailing-update tile
constexpr int CB = 64;             // rows per back-substitution block
}  // namespace

__global__ void __launch_bounds__(CT, 1) chol_panel_kernel(CholArgs a, int k0, int k1) {
    State *st = a.st;
    count_launch(st);
    const int n = a.n;
    const long long ld = a.ld;
    double *W = a.W, *Lp = a.Lp;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * CW + warp, nw = gridDim.x * CW;
    if (*(volatile int *)&st->status == LS_BREAKDOWN) return;
    for (int k = k0; k < k1; k++) {
        if (!grid_sync(a.bar, st)) return;
        const double piv = __ldcg(&W[(long long)k * ld + k]);
        if (!(piv > 0.0)) {                      // not positive definite (or NaN)
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                st->status = LS_BREAKDOWN;
                st->iter = k;
            }
            return;
        }
        const double lkk = sqrt(piv);
        if (blockIdx.x == 0 && threadIdx.x == 0) Lp[(long long)k * CH_NB + (k - k0)] = lkk;
        // lane c: panel column j = k + 1 + c, its l_jk from the unchanged column k
        const int j = k + 1 + lane;
        const bool on = j < k1;
        const double ljk = on ? __ldcg(&W[(long long)j * ld + k]) / lkk : 0.0;
        for (int i0 = k + 1 + gw; i0 <= n; i0 += CH_ROWS * nw) {
            double wik[CH_ROWS], wij[CH_ROWS];
#pragma unroll
            for (int u = 0; u < CH_ROWS; u++) {
                const int i = i0 + u * nw;
                wik[u] = i <= n ? __ldcg(&W[(long long)i * ld + k]) : 0.0;
                wij[u] = (i <= n && on && j <= i) ? __ldcg(&W[(long long)i * ld + j]) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < CH_ROWS; u++) {
                const int i = i0 + u * nw;
                if (i <= n) {
                    const double lik = wik[u] / lkk;
                    if (on && j <= i) W[(long long)i * ld + j] = __dsub_rn(wij[u], __dmul_rn(lik, ljk));
                    if (lane == 0) Lp[(long long)i * CH_NB + (k - k0)] = lik;
                }
            }
        }
    }
    if (!grid_sync(a.bar, st)) return;
    // the panel's columns of L (and the panel's y entries in row n) into W
    const long long cnt = (long long)(n + 1 - k0) * CH_NB;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < cnt;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = k0 + (int)(e / CH_NB), t = (int)(e % CH_NB);
        const int jj = k0 + t;
        if (jj < k1 && jj <= i && jj < n) W[(long long)i * ld + jj] = __ldcg(&Lp[(long long)i * CH_NB + t]);
    }
}

// Rows k1 .. n, columns k1 .. min(i, n - 1): w_ij -= l_it l_jt for the
// panel's steps t in order.
__global__ void __launch_bounds__(256) chol_trail_kernel(CholArgs a, int k0, int nb) {
    __shared__ double Ls[CTT][CH_NB + 1], Ms[CH_NB][CTT];
    State *st = a.st;
    count_launch(st);
    if (*(volatile int *)&st->status == LS_BREAKDOWN) return;
    const int n = a.n;
    const long long ld = a.ld;
    double *W = a.W;
    const double *Lp = a.Lp;
    const int k1 = k0 + nb;
    const int r0 = k1 + blockIdx.y * CTT, c0 = k1 + blockIdx.x * CTT;
    if (c0 > r0 + CTT - 1) return;               // the tile lies above the diagonal
    for (int e = threadIdx.x; e < CTT * CH_NB; e += blockDim.x) {
        const int r = e / CH_NB, t = e % CH_NB;
        Ls[r][t] = (r0 + r <= n && t < nb) ? __ldcg(&Lp[(long long)(r0 + r) * CH_NB + t]) : 0.0;
        const int tt = e / CTT, c = e % CTT;
        Ms[tt][c] = (c0 + c < n && tt < nb) ? __ldcg(&Lp[(long long)(c0 + c) * CH_NB + tt]) : 0.0;
    }
    __syncthreads();
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    double acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int r = r0 + ty + 16 * p, c = c0 + tx + 16 * q;
            acc[p][q] = (r <= n && c < n && c <= r) ? W[(long long)r * ld + c] : 0.0;
        }
    for (int t = 0; t < nb; t++) {
        double l[4], m[4];
#pragma unroll
        for (int p = 0; p < 4; p++) l[p] = Ls[ty + 16 * p][t];
#pragma unroll
        for (int q = 0; q < 4; q++) m[q] = Ms[t][tx + 16 * q];
#pragma unroll
        for (int p = 0; p < 4; p++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[p][q] = __dsub_rn(acc[p][q], __dmul_rn(l[p], m[q]));
    }
#pragma unroll
    for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int r = r0 + ty + 16 * p, c = c0 + tx + 16 * q;
            if (r <= n && c < n && c <= r) W[(long long)r * ld + c] = acc[p][q];
        }
}

__global__ void __launch_bounds__(CT, 1) chol_backsolve_kernel(CholArgs a) {
    __shared__ double s[CB], xs[CB];
    State *st = a.st;
    count_launch(st);
    const int n = a.n;
    const long long ld = a.ld;
    double *W = a.W;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (*(volatile int *)&st->status == LS_BREAKDOWN) return;
    double *y = a.y;                             // a copy of row n: y, then the updated right sides
    for (int r1 = n; r1 > 0; r1 -= CB) {
        const int r0 = r1 > CB ? r1 - CB : 0, nb = r1 - r0;
        if (blockIdx.x == 0 && warp == 0) {
            // the diagonal block, column oriented: x_i = s_i / l_ii, then s_r -= l_ir x_i (r < i)
            for (int r = lane; r < nb; r += 32) s[r] = __ldcg(&y[r0 + r]);
            __syncwarp();
            for (int i = nb - 1; i >= 0; i--) {
                const double xi = s[i] / W[(long long)(r0 + i) * ld + r0 + i];
                __syncwarp();
                for (int r = lane; r < i; r += 32) s[r] -= W[(long long)(r0 + i) * ld + r0 + r] * xi;
                if (lane == 0) xs[i] = xi;
                __syncwarp();
            }
            for (int r = lane; r < nb; r += 32) a.x[r0 + r] = xs[r];
        }
        if (!grid_sync(a.bar, st)) return;
        // rows above the block: y_i -= sum_{j in block} l_ji x_j, a thread a row i
        // (the block's rows of L are contiguous in i)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < r0; i += gridDim.x * blockDim.x) {
            double acc = 0.0;
            for (int jj = 0; jj < nb; jj++) acc += W[(long long)(r0 + jj) * ld + i] * __ldcg(&a.x[r0 + jj]);
            y[i] = __ldcg(&y[i]) - acc;
        }
        if (!grid_sync(a.bar, st)) return;
    }
}

// Entries above the diagonal of the n x n factor (the rest of A's copy) to zero.
__global__ void chol_zero_upper_kernel(CholArgs a) {
    const int n = a.n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)n * n;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        if (j > i) a.W[(long long)i * a.ld + j] = 0.0;
    }
}

CholKernels chol_kernels() {
    CholKernels K{};
    K.panel = reinterpret_cast<void *>(&chol_panel_kernel);
    K.trail = reinterpret_cast<void *>(&chol_trail_kernel);
    K.backsolve = reinterpret_cast<void *>(&chol_backsolve_kernel);
    K.zero_upper = reinterpret_cast<void *>(&chol_zero_upper_kernel);
    K.nb = CH_NB;
    K.tile = CTT;
    K.block = CT;
    return K;
}

}  // namespace lsi
