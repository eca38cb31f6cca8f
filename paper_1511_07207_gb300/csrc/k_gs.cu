// k_gs.cu -- the Gauss-Seidel sweep on the GPU.
//
// Gauss-Seidel (paper, introduction: the classical stationary methods, taken
// from the textbooks) recomputes x_i from the newest values of the others.
// Written as a correction, one sweep is
//     r = b - A x(k),   (D + L) d = r,   x(k+1) = x(k) + d,
// with D + L the lower triangle of A including the diagonal: the residual
// is the GEMV with the Jacobi stop test in its last CTA (k_gemv.cu), and
// this file solves the triangular system.
//
// The triangular solve is a dependency chain over row blocks of 64: block I
// needs d_j for every block j < I.  One persistent cooperative grid runs it:
//   * CTA 0 walks the chain: d_I = u_I - T_I^-1 sum_{w=1..W} A_{I,I-w} d_{I-w},
//     with T_I^-1 the inverse of the diagonal block (formed once per solve by
//     gs_tinv_kernel) and the last W blocks of d kept in shared memory;
//   * the other CTAs own row blocks (a snake order balances their lengths)
//     and stream, for each, the tiles A_{I,j} with j < I - W as soon as d_j
//     is published, then publish u_I = T_I^-1 (r_I - sum_j A_{I,j} d_j);
//   * publication is a flag per block written with release semantics after
//     the data, polled with acquire by one thread, with the sweep's number as
//     its value (flags are zeroed per solve, so stale ones never match);
//     every wait gives up after the library's time limit with ERRB_TIMEOUT.
// A is read as the FP32 pair hi + lo of the solvers' products and every tile
// product is double-single arithmetic on the FP32 pipe, so the sweep matches
// the FP64 recurrence to rounding; each helper sums its row block's tiles in
// column order, so results are deterministic.
#include <cuda_runtime.h>

#include "ls_device.cuh"
#include "ls_internal.h"

namespace lsi {

constexpr int GS_B = 64;         // rows (and columns) of a block
constexpr int GS_W = 2;          // sub-diagonal blocks the chain CTA multiplies itself
constexpr int GS_T = 256;        // threads per CTA

// ---- double-single arithmetic (Dekker's product by FMA, Knuth's two-sum) ------------------
struct F2 {
    float h, l;
};

__device__ __forceinline__ F2 f2_split(double v) {
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - (double)h)};
}

// acc += (mh + ml)(vh + vl), the product's terms below ml*vl kept
__device__ __forceinline__ void f2_mac(F2 &acc, float mh, float ml, float vh, float vl) {
    const float p = __fmul_rn(mh, vh);
    float e = __fmaf_rn(mh, vh, -p);
    e = __fmaf_rn(mh, vl, e);
    e = __fmaf_rn(ml, vh, e);
    const float s = __fadd_rn(acc.h, p);
    const float bb = __fsub_rn(s, acc.h);
    const float err = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    acc.h = s;
    acc.l = __fadd_rn(acc.l, __fadd_rn(e, err));
}

__device__ __forceinline__ double f2_value(F2 a) { return (double)a.h + (double)a.l; }

// Sum over the four lanes that share a row (lanes 4r .. 4r+3), in FP64.
__device__ __forceinline__ double row_sum(double a) {
    a += __shfl_xor_sync(0xffffffffu, a, 1);
    a += __shfl_xor_sync(0xffffffffu, a, 2);
    return a;
}

// ---- one thread's share of a 64 x 64 tile -------------------------------------------------
// Thread t owns row t / 4 and, with q = t % 4, the float4 chunks q, q + 4,
// q + 8, q + 12 of the row (so the four lanes of a row read 64 contiguous
// bytes per load).
struct TileRegs {
    float4 h[4], l[4];
};

// Loads the tile at rows r0.., columns c0.. of a pair matrix with row pitch
// ld (floats); elements outside rows < nrow, columns < ncol read as zero.
__device__ __forceinline__ void tile_load(TileRegs &T, const float *__restrict__ hi,
                                          const float *__restrict__ lo, long long ld, int r0, int c0,
                                          int nrow, int ncol) {
    const int row = threadIdx.x >> 2, q = threadIdx.x & 3;
    const int gr = r0 + row;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int c = c0 + (4 * k + q) * 4;
        float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
        if (gr < nrow && c < ncol) {
            const long long off = (long long)gr * ld + c;
            h = __ldg(reinterpret_cast<const float4 *>(hi + off));
            l = __ldg(reinterpret_cast<const float4 *>(lo + off));
            if (c + 3 >= ncol) {     // ragged last chunk: the padding columns are not A
                if (c + 1 >= ncol) h.y = l.y = 0.f;
                if (c + 2 >= ncol) h.z = l.z = 0.f;
                h.w = l.w = 0.f;
            }
        }
        T.h[k] = h;
        T.l[k] = l;
    }
}

// (this thread's 16 terms of the tile) . v in double-single, v given split in
// shared memory; the short sum keeps its low part small, and longer sums
// add these partials in FP64.
__device__ __forceinline__ double tile_dot(const TileRegs &T, const float *vh, const float *vl) {
    F2 acc = {0.f, 0.f};
    const int q = threadIdx.x & 3;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int c = (4 * k + q) * 4;
        const float4 xh = *reinterpret_cast<const float4 *>(vh + c);
        const float4 xl = *reinterpret_cast<const float4 *>(vl + c);
        f2_mac(acc, T.h[k].x, T.l[k].x, xh.x, xl.x);
        f2_mac(acc, T.h[k].y, T.l[k].y, xh.y, xl.y);
        f2_mac(acc, T.h[k].z, T.l[k].z, xh.z, xl.z);
        f2_mac(acc, T.h[k].w, T.l[k].w, xh.w, xl.w);
    }
    return f2_value(acc);
}

// ---- flags --------------------------------------------------------------------------------
// Thread 0 waits until *f == ep; false (and ERRB_TIMEOUT) after the time
// limit, or false at once when another CTA has recorded an error.
__device__ __forceinline__ bool flag_wait(const unsigned *f, unsigned ep, State *st) {
    if (ld_acquire_u32(f) == ep) return true;
    const unsigned long long t0 = gtimer();
    while (ld_acquire_u32(f) != ep) {
        if (*(volatile int *)&st->err) return false;
        if (gtimer() - t0 > WAIT_LIMIT_NS) {
            set_err(st, ERRB_TIMEOUT);
            return false;
        }
    }
    return true;
}

// All threads: wait for the flag (thread 0 polls); false on timeout/error.
__device__ __forceinline__ bool cta_wait(const unsigned *f, unsigned ep, State *st, int *ok_s) {
    if (threadIdx.x == 0) *ok_s = flag_wait(f, ep, st) ? 1 : 0;
    __syncthreads();
    return *ok_s != 0;
}

// All threads: publish after this CTA's data writes.
__device__ __forceinline__ void cta_publish(unsigned *f, unsigned ep) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        st_release_u32(f, ep);
    }
}

// ---- T_I^-1 of every diagonal block (once per solve) ----------------------------------------
// One CTA of 64 threads per block (grid-stride): thread c forward-substitutes
// column c of the identity through the block's lower triangle (FP64, from the
// FP64 A; the column in thread-local memory), and the inverse is stored as an
// FP32 pair, row-major 64 x 64 per block.  Rows past n are the identity.  A
// zero diagonal entry marks the solve a breakdown (and is replaced by 1 so
// nothing overflows).
__global__ void __launch_bounds__(GS_B) gs_tinv_kernel(int n, const double *__restrict__ A, long long lda,
                                                       float *__restrict__ Thi, float *__restrict__ Tlo,
                                                       State *st) {
    __shared__ double T[GS_B][GS_B + 1];
    double y[GS_B];
    count_launch(st);
    const int nblk = (n + GS_B - 1) / GS_B;
    const int c = threadIdx.x;
    for (int I = blockIdx.x; I < nblk; I += gridDim.x) {
        const int r0 = I * GS_B;
        for (int i = 0; i < GS_B; i++) {
            double v = 0.0;
            if (c <= i) {
                if (r0 + i < n) v = A[(long long)(r0 + i) * lda + r0 + c];
                else v = c == i ? 1.0 : 0.0;
            }
            if (c == i && v == 0.0) {
                st->status = LS_BREAKDOWN;
                v = 1.0;
            }
            T[i][c] = v;
        }
        __syncthreads();
        for (int i = 0; i < GS_B; i++) {
            double s = i == c ? 1.0 : 0.0;
            for (int j = c; j < i; j++) s -= T[i][j] * y[j];
            y[i] = i < c ? 0.0 : s / T[i][i];
        }
        float *th = Thi + (size_t)I * GS_B * GS_B, *tl = Tlo + (size_t)I * GS_B * GS_B;
        for (int i = 0; i < GS_B; i++) {
            const F2 v = f2_split(y[i]);
            th[i * GS_B + c] = v.h;
            tl[i * GS_B + c] = v.l;
        }
        __syncthreads();
    }
}

// ---- the triangular solve (cooperative) ------------------------------------------------------
struct GsShared {
    float dh[GS_W + 1][GS_B], dl[GS_W + 1][GS_B];   // chain: ring of the last d blocks, split
    float vh[GS_B], vl[GS_B];                         // the vector of the current tile product
    double rowv[GS_B];
    int ok;
};

// Row block owned by helper g (0 .. H-1) in round k, or -1: blocks are
// dealt from the last one down in a snake order, so the long rows at the
// bottom and the short ones at the top share helpers.
__device__ __forceinline__ int gs_owned(int g, int H, int k, int nblk) {
    const int p = k * H + ((k & 1) ? H - 1 - g : g);
    return nblk - 1 - p;
}

__global__ void __launch_bounds__(GS_T, 1) gs_trsv_kernel(GsArgs a, cudaGraphConditionalHandle h_loop) {
    __shared__ __align__(16) GsShared S;
    State *st = a.st;
    count_launch(st);
    const int stop = *(volatile int *)&st->skip || *(volatile int *)&st->err;
    if (stop) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(st, h_loop, 0u);
        return;
    }
    const unsigned ep = (unsigned)*(volatile int *)&st->iter;
    const int n = a.n, nblk = (n + GS_B - 1) / GS_B;
    const int row = threadIdx.x >> 2, q = threadIdx.x & 3;
    const size_t TB = (size_t)GS_B * GS_B;

    if (blockIdx.x == 0) {
        // ---------------- the chain ----------------
        for (int i = threadIdx.x; i < (GS_W + 1) * GS_B; i += GS_T) {
            (&S.dh[0][0])[i] = 0.f;
            (&S.dl[0][0])[i] = 0.f;
        }
        bool ok = true;
        for (int I = 0; I < nblk && ok; I++) {
            const int r0 = I * GS_B;
            TileRegs Ti, Aw[GS_W];
            tile_load(Ti, a.Thi + I * TB, a.Tlo + I * TB, GS_B, 0, 0, GS_B, GS_B);
#pragma unroll
            for (int w = 1; w <= GS_W; w++)
                if (I - w >= 0) tile_load(Aw[w - 1], a.Ahi, a.Alo, a.ld, r0, (I - w) * GS_B, n, n);
            // s = sum_w A_{I,I-w} d_{I-w}
            double acc = 0.0;
#pragma unroll
            for (int w = 1; w <= GS_W; w++)
                if (I - w >= 0) {
                    const int slot = (I - w) % (GS_W + 1);
                    acc += tile_dot(Aw[w - 1], S.dh[slot], S.dl[slot]);
                }
            acc = row_sum(acc);
            if (q == 0) {
                const F2 sv = f2_split(acc);
                S.vh[row] = sv.h;
                S.vl[row] = sv.l;
            }
            __syncthreads();
            // t = T_I^-1 s
            const double t = row_sum(tile_dot(Ti, S.vh, S.vl));
            // d_I = u_I - t, once u_I is published
            ok = cta_wait(&a.flagU[I], ep, st, &S.ok);
            if (!ok) break;
            const int slot = I % (GS_W + 1);
            if (q == 0) {
                const int gr = r0 + row;
                double d = 0.0;
                if (gr < n) {
                    d = __ldcg(&a.u[gr]) - t;
                    a.delta[gr] = d;
                    a.x[gr] += d;
                }
                const F2 ds = f2_split(d);
                S.dh[slot][row] = ds.h;
                S.dl[slot][row] = ds.l;
            }
            cta_publish(&a.flagD[I], ep);
        }
        if (threadIdx.x == 0) set_cond(st, h_loop, ok && !*(volatile int *)&st->err ? 1u : 0u);
        return;
    }

    // ---------------- helpers ----------------
    const int H = gridDim.x - 1, g = blockIdx.x - 1;
    // owned blocks in ascending order: the snake deals them from the bottom up
    int rounds = (nblk + H - 1) / H;
    for (int k = rounds - 1; k >= 0; k--) {
        const int I = gs_owned(g, H, k, nblk);
        if (I < 0) continue;
        const int r0 = I * GS_B;
        const int jend = I - GS_W;   // tiles j < jend are this CTA's
        double acc = 0.0;
        TileRegs cur, nxt;
        if (jend > 0) tile_load(cur, a.Ahi, a.Alo, a.ld, r0, 0, n, n);
        for (int j = 0; j < jend; j++) {
            if (j + 1 < jend) tile_load(nxt, a.Ahi, a.Alo, a.ld, r0, (j + 1) * GS_B, n, n);
            if (!cta_wait(&a.flagD[j], ep, st, &S.ok)) return;
            if (threadIdx.x < GS_B) {
                const int gc = j * GS_B + threadIdx.x;
                const F2 v = f2_split(gc < n ? __ldcg(&a.delta[gc]) : 0.0);
                S.vh[threadIdx.x] = v.h;
                S.vl[threadIdx.x] = v.l;
            }
            __syncthreads();
            acc += tile_dot(cur, S.vh, S.vl);
            __syncthreads();
            cur = nxt;
        }
        // u_I = T_I^-1 (r_I - P_I)
        acc = row_sum(acc);
        if (q == 0) {
            const int gr = r0 + row;
            const F2 s = f2_split(gr < n ? a.r[gr] - acc : 0.0);
            S.vh[row] = s.h;
            S.vl[row] = s.l;
        }
        TileRegs Ti;
        tile_load(Ti, a.Thi + I * TB, a.Tlo + I * TB, GS_B, 0, 0, GS_B, GS_B);
        __syncthreads();
        const double t = row_sum(tile_dot(Ti, S.vh, S.vl));
        if (q == 0 && r0 + row < n) a.u[r0 + row] = t;
        cta_publish(&a.flagU[I], ep);
        __syncthreads();
    }
}

GsKernels gs_kernels() {
    GsKernels K{};
    K.tinv = reinterpret_cast<void *>(&gs_tinv_kernel);
    K.trsv = reinterpret_cast<void *>(&gs_trsv_kernel);
    K.tinv_block = GS_B;
    K.trsv_block = GS_T;
    K.blk = GS_B;
    return K;
}

}  // namespace lsi
