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
// lu_factor_kernel (cooperative, persistent over a range of steps k):
//   * the pivot candidates of column k are the CTAs' partial maxima (value
//     and first row index), formed while updating the previous column and
//     reduced by every CTA in CTA order, so all CTAs pick the same v;
//   * rows k and v are swapped over all n + 1 columns by the whole grid;
//   * each row i > k belongs to one warp: l = w_ik / w_kk (IEEE division),
//     w_ij = w_ij - l * w_kj as a separate multiply and subtract (no fused
//     multiply-add), so every element is bit for bit what the same
//     elimination gives in plain FP64 arithmetic; the warp also forms the
//     row's next pivot candidate |w_i,k+1|.
//   Two bounded grid barriers per step.  A row is updated by different warps
//   at different steps and swapped by any CTA, so every read of W here goes
//   to L2 (ld.global.cg), never to a possibly stale L1 line.
// lu_backsolve_kernel (cooperative): U x = y by blocks of 64 rows from the
//   bottom: CTA 0 solves the diagonal block (one warp, column oriented),
//   then every CTA subtracts the block's contribution from the rows above
//   it (a warp a row).  Two grid barriers per block.
//
// The unblocked elimination streams the trailing block once per step
// (16 (n-k)^2 bytes at step k): HBM-bound, 16 n^3 / 3 bytes in all.
#include <cuda_runtime.h>

#include "ls_device.cuh"
#include "ls_internal.h"

namespace lsi {

namespace {

constexpr int LT = 512;            // threads per CTA (16 warps: enough loads in flight)
constexpr int LU_UNROLL = 4;       // elements of a row a lane loads before it computes
constexpr int LW = LT / 32;        // warps per CTA
constexpr int LB = 64;             // rows per back-substitution block

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
    if (k0 == 0) {   // candidates of column 0
        Cand mine = {-1.0, n};
        for (int i = gw; i < n; i += nw)
            if (lane == 0) mine = better(mine, Cand{fabs(__ldcg(&W[(long long)i * ld])), i});
        publish_cand(a, mine, red);
    }
    for (int k = k0; k < k1; k++) {
        if (!grid_sync(a.bar, st)) return;
        // the pivot row, the same in every CTA
        if (threadIdx.x == 0) {
            Cand c = {-1.0, n};
            for (int b = 0; b < (int)gridDim.x; b++)
                c = better(c, Cand{__ldcg(&a.cand_v[b]), __ldcg(&a.cand_i[b])});
            // a row k whose value is not comparable (NaN) stays the pivot, as the
            // sequential scan that starts from it would leave it
            v_s = c.i >= k && c.i < n ? c.i : k;
            if (blockIdx.x == 0) a.ipiv[k] = v_s;
        }
        __syncthreads();
        const int v = v_s;
        if (v != k)
            for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j <= n;
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
        // rows i > k: l, the rank-1 update (and y in column n), next candidates
        Cand mine = {-1.0, n};
        const double *wk = W + (long long)k * ld;
        for (int i = k + 1 + gw; i < n; i += nw) {
            double *wi = W + (long long)i * ld;
            const double l = __ldcg(&wi[k]) / piv;
            __syncwarp();
            double next = 0.0;   // w_i,k+1 after the update (lane 0 owns column k + 1)
            for (int j0 = k + 1 + lane; j0 <= n; j0 += 32 * LU_UNROLL) {
                double wv[LU_UNROLL], kv[LU_UNROLL];
#pragma unroll
                for (int u = 0; u < LU_UNROLL; u++) {
                    const int j = j0 + 32 * u;
                    wv[u] = j <= n ? __ldcg(&wi[j]) : 0.0;
                    kv[u] = j <= n ? __ldcg(&wk[j]) : 0.0;
                }
#pragma unroll
                for (int u = 0; u < LU_UNROLL; u++) {
                    const int j = j0 + 32 * u;
                    if (j <= n) {
                        const double w = __dsub_rn(wv[u], __dmul_rn(l, kv[u]));
                        wi[j] = w;
                        if (j == k + 1) next = w;
                    }
                }
            }
            __syncwarp();
            if (lane == 0) {
                wi[k] = l;
                if (k + 1 < n) mine = better(mine, Cand{fabs(next), i});
            }
        }
        publish_cand(a, mine, red);
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
    K.block = LT;
    return K;
}

}  // namespace lsi
