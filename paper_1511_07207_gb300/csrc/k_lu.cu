// k_lu.cu -- the paper's direct method: LU factorization with partial
// pivoting (right-looking Gaussian elimination), FP64, and the solve.
//
// The paper's right-looking LU: at step k take the row v >= k with the
// largest |a_vk| (the first one on ties), swap rows k and v, divide the
// sub-column by the pivot and subtract the rank-1 update from the trailing
// block.  The right-hand side rides along as column n of the working matrix
// W = [A | b], so the forward substitution L y = P b happens during the
// elimination (y in column n), and U x = y is solved afterwards.
//
// The elimination runs as the paper's block LU factorization (Figures 1-2,
// equations (1)-(4)) with panels of LU_NB = 32 columns, and stays the same
// elimination element by element: every a_ij receives a_ij - l_it u_tj for
// t = 0, 1, ... in order, as a rounded product and a rounded difference.
// Per panel:
// lu_factor_kernel (cooperative, over the panel's steps, its columns only):
//   * the pivot candidates of column k are the CTAs' partial maxima (value
//     and first row index), formed while updating the previous column and
//     reduced by every CTA (a total order, so all CTAs pick the same v);
//   * rows k and v are swapped over the panel's columns by the whole grid;
//   * each row i > k belongs to one warp: l = w_ik / w_kk (IEEE division),
//     w_ij = w_ij - l * w_kj as a separate multiply and subtract (no fused
//     multiply-add), so every element is bit for bit what the same
//     elimination gives in plain FP64 arithmetic; the warp also forms the
//     row's next pivot candidate |w_i,k+1|.
//   Two bounded grid barriers per step.  A row is updated by different warps
//   at different steps and swapped by any CTA, so every read of W here goes
//   to L2 (ld.global.cg), never to a possibly stale L1 line.
// lu_laswp_kernel: the panel's row swaps on every other column (a thread a
//   column, the swaps in step order).
// lu_u12_kernel: the panel's pivot rows right of the panel (the paper's
//   triangular solve for U01): the panel's updates t = k0 .. in order, four
//   lanes a column, each holding 8 of the 32 values in registers.
// lu_trail_kernel: the block below and right of the panel, 64 x 64 tiles:
//   each element takes the panel's 32 updates in order from the multipliers
//   and pivot rows staged in shared memory.  This is where the time goes:
//   two FP64 instructions per element and step (a product and a difference,
//   not fused), so the elimination is bound by the FP64 pipe, and A crosses
//   DRAM once per panel instead of once per step.
// lu_backsolve_kernel (cooperative): U x = y by blocks of 64 rows from the
//   bottom: CTA 0 solves the diagonal block (one warp, column oriented),
//   then every CTA subtracts the block's contribution from the rows above
//   it (a warp a row).  Two grid barriers per block.
//
// Work: n^3 / 3 updates of two FP64 instructions; traffic about 16 n^3 / (3 LU_NB) bytes.
#include <cuda_runtime.h>

#include "ls_device.cuh"
#include "ls_internal.h"

namespace lsi {

namespace {

constexpr int LT = 512;            // threads per CTA (16 warps: enough loads in flight)
constexpr int LU_ROWS = 4;         // rows a warp loads before it computes (panel steps)
constexpr int U12_T = 128;         // threads per CTA of lu_u12_kernel (32 columns)
constexpr int LU_NB = 32;          // panel width
constexpr int LW = LT / 32;        // warps per CTA
constexpr int LB = 64;             // rows per back-substitution block
constexpr int TT = 64;             // trailing-update tile (rows and columns)

struct Cand {
    double v;
    int i;
};

// The better of two pivot candidates: the larger |a|, the first row on ties.
__device__ __forceinline__ Cand better(Cand a, Cand b) {
    if (b.v > a.v || (b.v == a.v && b.i < a.i)) return b;
    return a;
}

// This CTA's candidate from its warps' candidates (fixed order) into part.
__device__ void publish_cand(const LuArgs &a, Cand mine, Cand *red) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        Cand c = red[0];
        for (int w = 1; w < LW; w++) c = better(c, red[w]);
        a.cand_v[blockIdx.x] = c.v;
        a.cand_i[blockIdx.x] = c.i;
    }
}

}  // namespace

__global__ void __launch_bounds__(LT, 1) lu_factor_kernel(LuArgs a, int k0, int k1) {
    // k0 .. k1 - 1: the steps of one panel, whose columns are k0 .. k1 - 1
    __shared__ Cand red[LW];
    __shared__ int v_s;
    State *st = a.st;
    count_launch(st);
    const int n = a.n;
    const long long ld = a.ld;
    double *W = a.W;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * LW + warp, nw = gridDim.x * LW;
    if (*(volatile int *)&st->status == LS_BREAKDOWN) return;
    {   // candidates of the panel's first column (rows k0 .. n-1)
        Cand mine = {-1.0, n};
        for (int i = k0 + gw; i < n; i += nw)
            if (lane == 0) mine = better(mine, Cand{fabs(__ldcg(&W[(long long)i * ld + k0])), i});
        publish_cand(a, mine, red);
    }
    for (int k = k0; k < k1; k++) {
        if (!grid_sync(a.bar, st)) return;
        // the pivot row, the same in every CTA: warp 0 reads the CTAs'
        // candidates in parallel and reduces them by shuffles.  No NaN enters
        // a candidate (a comparison with NaN never prefers it), so "better" is
        // a total order and the reduction order does not change the result.
        if (warp == 0) {
            Cand c = {-1.0, n};
            for (int b = lane; b < (int)gridDim.x; b += 32)
                c = better(c, Cand{__ldcg(&a.cand_v[b]), __ldcg(&a.cand_i[b])});
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                c = better(c, Cand{__shfl_xor_sync(0xffffffffu, c.v, o), __shfl_xor_sync(0xffffffffu, c.i, o)});
            if (lane == 0) {
                // no comparable candidate (all NaN): row k stays the pivot, as the
                // sequential scan that starts from it would leave it
                v_s = c.i >= k && c.i < n ? c.i : k;
                if (blockIdx.x == 0) a.ipiv[k] = v_s;
            }
        }
        __syncthreads();
        const int v = v_s;
        if (v != k)   // the panel's columns (the others: lu_laswp_kernel)
            for (long long j = k0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; j < k1;
                 j += (long long)gridDim.x * blockDim.x) {
                const double t = __ldcg(&W[(long long)k * ld + j]);
                W[(long long)k * ld + j] = __ldcg(&W[(long long)v * ld + j]);
                W[(long long)v * ld + j] = t;
            }
        if (!grid_sync(a.bar, st)) return;
        const double piv = __ldcg(&W[(long long)k * ld + k]);
        if (piv == 0.0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) st->status = LS_BREAKDOWN;
            return;
        }
        // rows i > k of the panel: l, the rank-1 update, next candidates.  The
        // panel has at most 31 columns right of k: lane c owns column k + 1 + c
        // (lane 0 the next pivot column); a warp takes LU_ROWS rows at a time
        // with all their loads issued before any arithmetic.
        Cand mine = {-1.0, n};
        const int j = k + 1 + lane;
        const bool on = j < k1;
        const double wkj = on ? __ldcg(&W[(long long)k * ld + j]) : 0.0;
        for (int i0 = k + 1 + gw; i0 < n; i0 += LU_ROWS * nw) {
            double wik[LU_ROWS], wij[LU_ROWS];
#pragma unroll
            for (int u = 0; u < LU_ROWS; u++) {
                const int i = i0 + u * nw;
                wik[u] = i < n ? __ldcg(&W[(long long)i * ld + k]) : 0.0;
                wij[u] = (i < n && on) ? __ldcg(&W[(long long)i * ld + j]) : 0.0;
            }
            __syncwarp();   // every lane has read w_ik before lane 0 overwrites it with l
#pragma unroll
            for (int u = 0; u < LU_ROWS; u++) {
                const int i = i0 + u * nw;
                if (i < n) {
                    const double l = wik[u] / piv;
                    const double w = __dsub_rn(wij[u], __dmul_rn(l, wkj));
                    if (on) W[(long long)i * ld + j] = w;
                    if (lane == 0) {
                        W[(long long)i * ld + k] = l;
                        if (on) mine = better(mine, Cand{fabs(w), i});
                    }
                }
            }
        }
        publish_cand(a, mine, red);
    }
}

// The panel's swaps (steps k0 .. k0 + nb - 1) on the columns outside it.
__global__ void __launch_bounds__(256) lu_laswp_kernel(LuArgs a, int k0, int nb) {
    State *st = a.st;
    count_launch(st);
    if (*(volatile int *)&st->status == LS_BREAKDOWN) return;
    const int n = a.n;
    const long long ld = a.ld;
    double *W = a.W;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c <= n; c += (long long)gridDim.x * blockDim.x) {
        if (c >= k0 && c < k0 + nb) continue;
        for (int t = k0; t < k0 + nb; t++) {
            const int v = a.ipiv[t];
            if (v != t) {
                const double x = W[(long long)t * ld + c];
                W[(long long)t * ld + c] = W[(long long)v * ld + c];
                W[(long long)v * ld + c] = x;
            }
        }
    }
}

// The pivot rows k0 .. k0 + nb - 1 right of the panel: u_rj -= l_rt u_tj for
// t = k0 .. r - 1 in order.  Four lanes a column (lane q of the quad holds
// rows q, q + 4, ...; the owner of row t hands u_tj to the others by a
// shuffle once it is final), so there are enough warps to keep the FP64
// pipes of every SM busy.
__global__ void __launch_bounds__(U12_T) lu_u12_kernel(LuArgs a, int k0, int nb) {
    __shared__ double Lp[LU_NB][LU_NB + 1];   // the panel's multipliers l_rt, zero past nb
    State *st = a.st;
    count_launch(st);
    if (*(volatile int *)&st->status == LS_BREAKDOWN) return;
    const int n = a.n;
    const long long ld = a.ld;
    double *W = a.W;
    for (int e = threadIdx.x; e < LU_NB * LU_NB; e += blockDim.x) {
        const int r = e / LU_NB, t = e % LU_NB;
        Lp[r][t] = (r < nb && t < r) ? W[(long long)(k0 + r) * ld + k0 + t] : 0.0;
    }
    __syncthreads();
    const int q = threadIdx.x & 3, lane = threadIdx.x & 31;
    const long long ncols = (long long)n + 1 - (k0 + nb);
    const int cpb = U12_T / 4;   // columns a CTA takes at a time
    // the loop bound is the same for the whole CTA, so every lane reaches the shuffles
    for (long long c0 = (long long)blockIdx.x * cpb; c0 < ncols; c0 += (long long)gridDim.x * cpb) {
        const long long jj = c0 + threadIdx.x / 4;
        const bool on = jj < ncols;
        const long long j = k0 + nb + jj;
        // rows past the panel's nb (a short last panel) stay zero and are not stored
        double u[LU_NB / 4];
#pragma unroll
        for (int x = 0; x < LU_NB / 4; x++) {
            const int r = q + 4 * x;
            u[x] = (on && r < nb) ? W[(long long)(k0 + r) * ld + j] : 0.0;
        }
#pragma unroll
        for (int t = 0; t < LU_NB - 1; t++) {
            const double ut = __shfl_sync(0xffffffffu, u[t / 4], (lane & ~3) | (t & 3));
#pragma unroll
            for (int x = 0; x < LU_NB / 4; x++)
                if (q + 4 * x > t) u[x] = __dsub_rn(u[x], __dmul_rn(Lp[q + 4 * x][t], ut));
        }
#pragma unroll
        for (int x = 0; x < LU_NB / 4; x++) {
            const int r = q + 4 * x;
            if (on && r < nb) W[(long long)(k0 + r) * ld + j] = u[x];
        }
    }
}

// The block below and right of the panel (rows k0 + LU_NB .. n - 1, columns
// k0 + LU_NB .. n): a_ij -= l_it u_tj for the panel's steps t in order.
__global__ void __launch_bounds__(256) lu_trail_kernel(LuArgs a, int k0) {
    __shared__ double Ls[TT][LU_NB + 1], Us[LU_NB][TT];
    State *st = a.st;
    count_launch(st);
    if (*(volatile int *)&st->status == LS_BREAKDOWN) return;
    const int n = a.n;
    const long long ld = a.ld;
    double *W = a.W;
    const int r0 = k0 + LU_NB + blockIdx.y * TT, c0 = k0 + LU_NB + blockIdx.x * TT;
    for (int e = threadIdx.x; e < TT * LU_NB; e += blockDim.x) {
        const int r = e / LU_NB, t = e % LU_NB;
        Ls[r][t] = r0 + r < n ? W[(long long)(r0 + r) * ld + k0 + t] : 0.0;
        const int tt = e / TT, c = e % TT;
        Us[tt][c] = c0 + c <= n ? W[(long long)(k0 + tt) * ld + c0 + c] : 0.0;
    }
    __syncthreads();
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    double acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int r = r0 + ty + 16 * p, c = c0 + tx + 16 * q;
            acc[p][q] = (r < n && c <= n) ? W[(long long)r * ld + c] : 0.0;
        }
#pragma unroll 4
    for (int t = 0; t < LU_NB; t++) {
        double l[4], u[4];
#pragma unroll
        for (int p = 0; p < 4; p++) l[p] = Ls[ty + 16 * p][t];
#pragma unroll
        for (int q = 0; q < 4; q++) u[q] = Us[t][tx + 16 * q];
#pragma unroll
        for (int p = 0; p < 4; p++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[p][q] = __dsub_rn(acc[p][q], __dmul_rn(l[p], u[q]));
    }
#pragma unroll
    for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int r = r0 + ty + 16 * p, c = c0 + tx + 16 * q;
            if (r < n && c <= n) W[(long long)r * ld + c] = acc[p][q];
        }
}

__global__ void __launch_bounds__(LT, 1) lu_backsolve_kernel(LuArgs a) {
    __shared__ double s[LB], xs[LB];
    State *st = a.st;
    count_launch(st);
    const int n = a.n;
    const long long ld = a.ld;
    double *W = a.W;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * LW + warp, nw = gridDim.x * LW;
    if (*(volatile int *)&st->status == LS_BREAKDOWN) return;
#define Y(i) W[(long long)(i) * ld + n]   // y = L^-1 P b, column n of the working matrix
    for (int r1 = n; r1 > 0; r1 -= LB) {
        const int r0 = r1 > LB ? r1 - LB : 0, nb = r1 - r0;
        if (blockIdx.x == 0 && warp == 0) {
            // the diagonal block, column oriented: x_i = s_i / u_ii, then s_r -= u_ri x_i
            for (int r = lane; r < nb; r += 32) s[r] = __ldcg(&Y(r0 + r));
            __syncwarp();
            for (int i = nb - 1; i >= 0; i--) {
                const double xi = s[i] / W[(long long)(r0 + i) * ld + r0 + i];
                __syncwarp();
                for (int r = lane; r < i; r += 32) s[r] -= W[(long long)(r0 + r) * ld + r0 + i] * xi;
                if (lane == 0) xs[i] = xi;
                __syncwarp();
            }
            for (int r = lane; r < nb; r += 32) a.x[r0 + r] = xs[r];
        }
        if (!grid_sync(a.bar, st)) return;
        // rows above the block: y_i -= sum_{j in block} u_ij x_j (a warp a row)
        for (int i = gw; i < r0; i += nw) {
            const double *wi = W + (long long)i * ld + r0;
            double acc = 0.0;
            for (int j = lane; j < nb; j += 32) acc += wi[j] * __ldcg(&a.x[r0 + j]);
            acc = warp_sum(acc);
            if (lane == 0) Y(i) = __ldcg(&Y(i)) - acc;
        }
        if (!grid_sync(a.bar, st)) return;
    }
#undef Y
}

LuKernels lu_kernels() {
    LuKernels K{};
    K.factor = reinterpret_cast<void *>(&lu_factor_kernel);
    K.backsolve = reinterpret_cast<void *>(&lu_backsolve_kernel);
    K.laswp = reinterpret_cast<void *>(&lu_laswp_kernel);
    K.u12 = reinterpret_cast<void *>(&lu_u12_kernel);
    K.trail = reinterpret_cast<void *>(&lu_trail_kernel);
    K.nb = LU_NB;
    K.u12_block = U12_T;
    K.tile = TT;
    K.block = LT;
    return K;
}

}  // namespace lsi
