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
//   * CTA 0 walks the chain: d_I = u_I - sum_{w=1..W} M_{I,w} d_{I-w} with
//     M_{I,w} = T_I^-1 A_{I,I-w}, T_I^-1 the inverse of the diagonal block
//     (both formed once per solve: gs_tinv_kernel, gs_panel_kernel) and the
//     last W blocks of d kept in shared memory;
//   * the other CTAs own row blocks (a snake order balances their lengths)
//     and walk the columns j = 0, 1, ...: once d_j is published, the tile
//     A_{I,j} of every owned block with j < I - W; when a block's last tile
//     is in, they publish u_I = T_I^-1 (r_I - sum_j A_{I,j} d_j);
//   * in every CTA one producer lane streams the CTA's fixed sequence of
//     64 x 64 tiles (hi and lo) into a ring of shared-memory slots (mbarrier
//     full/empty), so the tiles arrive ahead of the flags that gate their
//     use; sixteen consumer warps compute.  Helpers load with 2-D TMA
//     (128-byte swizzle, zero fill past n); the chain's M_{I,w} sit in a
//     contiguous panel in its threads' read order, one 32 KB bulk copy per
//     tile;
//   * publication is a flag per block written with release semantics after
//     the data, polled with acquire, with the sweep's number as its value
//     (flags are zeroed per solve, so stale ones never match); the chain's
//     flags are written by a second lane of the producer warp, signalled by
//     an mbarrier, so the chain never waits for its own stores;
//   * every wait is bounded (the library's time limit, ERRB_TIMEOUT) and
//     every decision that several warps act on is combined with a
//     barrier-reduction, so no thread is left waiting on one that gave up;
//   * x += d is applied by the whole grid after one grid barrier.
#include <cuda_runtime.h>

#include "ls_device.cuh"
#include "ls_internal.h"

namespace lsi {

constexpr int GS_B = 64;         // rows (and columns) of a block
constexpr int GS_W = 3;          // sub-diagonal blocks the chain CTA multiplies itself
constexpr int GS_C = 512;        // consumer threads (16 warps)
constexpr int GS_LPR = GS_C / 64;// consumer lanes per tile row (8)
constexpr int GS_T = GS_C + 64;  // plus the producer warp and the chain's u-fetcher warp
constexpr int GS_SLOTS = 6;      // tile slots in the ring
constexpr int GS_SLOT_B = 32768; // one tile: hi and lo, two 32-column boxes each
constexpr int GS_BOX_B = 8192;   // 32 columns x 64 rows of FP32
constexpr int GS_PUB = 8;        // chain publication mbarriers (steps in flight, > W + 1)
constexpr int GS_UB = 4;         // chain: u blocks staged ahead in shared memory
constexpr int GS_KMAX = 8;       // row blocks a helper owns at most
constexpr int GS_BAR_C = 1;      // named barrier of the consumer warps

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

// a + b, renormalised (Knuth's two-sum on the high parts, then a fast two-sum)
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    const float s = __fadd_rn(a.h, b.h);
    const float bb = __fsub_rn(s, a.h);
    const float err = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
    const float l = __fadd_rn(__fadd_rn(a.l, b.l), err);
    const float h = __fadd_rn(s, l);
    return {h, __fsub_rn(l, __fsub_rn(h, s))};
}

// Sum over the eight lanes that share a row, FP32 pairs (no FP64 pipe
// work: on this GPU a warp-wide FP64 instruction costs 16 FP32 ones).
__device__ __forceinline__ F2 f2_row_sum(F2 a) {
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        F2 b;
        b.h = __shfl_xor_sync(0xffffffffu, a.h, o);
        b.l = __shfl_xor_sync(0xffffffffu, a.l, o);
        a = f2_add(a, b);
    }
    return a;
}

// Sum over the eight lanes that share a row, in FP64.
__device__ __forceinline__ double row_sum(double a) {
    a += __shfl_xor_sync(0xffffffffu, a, 1);
    a += __shfl_xor_sync(0xffffffffu, a, 2);
    a += __shfl_xor_sync(0xffffffffu, a, 4);
    return a;
}

// ---- one thread's share of a 64 x 64 tile in a ring slot ---------------------------------------
// A slot holds the tile as four TMA boxes (hi cols 0-31, hi 32-63, lo 0-31,
// lo 32-63), each 64 rows of 128 bytes with the 128-byte swizzle: 16-byte
// chunk c of row r sits at chunk c ^ (r & 7).  Consumer thread t owns row
// t / 8 and, with q = t % 8, chunk q of both halves (columns 4q .. 4q + 3
// and 32 + 4q ..); the eight lanes of a shared-memory phase are one row and
// touch eight distinct chunks.
__device__ __forceinline__ F2 tile_dot(const unsigned char *slot, const float *vh, const float *vl) {
    F2 acc[2] = {{0.f, 0.f}, {0.f, 0.f}};   // one a half: two short chains
    const int row = threadIdx.x / GS_LPR, q = threadIdx.x % GS_LPR;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int off = h * GS_BOX_B + row * 128 + ((q ^ (row & 7)) << 4);
        const float4 mh = *reinterpret_cast<const float4 *>(slot + off);
        const float4 ml = *reinterpret_cast<const float4 *>(slot + 2 * GS_BOX_B + off);
        const int col = h * 32 + q * 4;
        const float4 xh = *reinterpret_cast<const float4 *>(vh + col);
        const float4 xl = *reinterpret_cast<const float4 *>(vl + col);
        f2_mac(acc[h], mh.x, ml.x, xh.x, xl.x);
        f2_mac(acc[h], mh.y, ml.y, xh.y, xl.y);
        f2_mac(acc[h], mh.z, ml.z, xh.z, xl.z);
        f2_mac(acc[h], mh.w, ml.w, xh.w, xl.w);
    }
    return f2_add(acc[0], acc[1]);   // renormalised
}

// The chain's panel tile: for h = 0, 1 and part (hi, lo), GS_C float4, the
// one of consumer thread t at index t: columns 32h + 4q .. +3 of row t / 8,
// q = t % 8 (the same columns as tile_dot).
constexpr int GS_PANEL_TILE = 8192;   // floats
__device__ __forceinline__ F2 tile_dot_panel(const unsigned char *slot, const float *vh, const float *vl) {
    F2 acc[2] = {{0.f, 0.f}, {0.f, 0.f}};
    const float4 *P = reinterpret_cast<const float4 *>(slot);
    const int q = threadIdx.x % GS_LPR;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const float4 mh = P[(2 * h) * GS_C + threadIdx.x];
        const float4 ml = P[(2 * h + 1) * GS_C + threadIdx.x];
        const int col = h * 32 + q * 4;
        const float4 xh = *reinterpret_cast<const float4 *>(vh + col);
        const float4 xl = *reinterpret_cast<const float4 *>(vl + col);
        f2_mac(acc[h], mh.x, ml.x, xh.x, xl.x);
        f2_mac(acc[h], mh.y, ml.y, xh.y, xl.y);
        f2_mac(acc[h], mh.z, ml.z, xh.z, xl.z);
        f2_mac(acc[h], mh.w, ml.w, xh.w, xl.w);
    }
    return f2_add(acc[0], acc[1]);
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

// Consumer threads: thread 0 polls the flag; all agree on the outcome.
__device__ __forceinline__ bool consumers_wait_flag(const unsigned *f, unsigned ep, State *st) {
    bool bad = false;
    if (threadIdx.x == 0) bad = !flag_wait(f, ep, st);
    return !named_bar_or(GS_BAR_C, GS_C, bad);
}

// Consumer threads: every thread waits for the slot's TMA data; all agree.
__device__ __forceinline__ bool consumers_wait_full(uint64_t *full, int seq, State *st) {
    bool bad = !mbar_wait(full, (seq / GS_SLOTS) & 1);
    if (bad) set_err(st, ERRB_TIMEOUT);
    return !named_bar_or(GS_BAR_C, GS_C, bad);
}

// Consumer threads: hand the slot back to the producer (one arrive a warp).
__device__ __forceinline__ void consumers_release(uint64_t *empty) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(empty);
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

// ---- the chain's panel (once per solve, after T_I^-1) ---------------------------------------------
// Tile (I, w), w = 1..W: M_{I,w} = T_I^-1 A_{I,I-w} in double-single
// arithmetic from the FP32 pairs of T_I^-1 and A, laid out as tile_dot_panel
// reads it (zero where I - w < 0 and past n).  T_I^-1 is lower triangular,
// so row i sums k = 0..i; each warp runs k up to its last row (the entries
// above the diagonal are stored zeros).
constexpr size_t GS_PANEL_SMEM = (size_t)2 * GS_B * (GS_B + 1) * 4 + (size_t)2 * GS_B * GS_B * 4;
__global__ void __launch_bounds__(GS_C) gs_panel_kernel(int n, const float *__restrict__ Ahi,
                                                        const float *__restrict__ Alo, long long ld,
                                                        const float *__restrict__ Thi,
                                                        const float *__restrict__ Tlo, float *__restrict__ panel,
                                                        State *st) {
    extern __shared__ __align__(16) float pm[];
    float *Th = pm, *Tl = Th + GS_B * (GS_B + 1);           // [64][65]: rows padded against conflicts
    float *Ah = Tl + GS_B * (GS_B + 1), *Al = Ah + GS_B * GS_B;   // [64][64]
    count_launch(st);
    const int nblk = (n + GS_B - 1) / GS_B;
    const int row = threadIdx.x / GS_LPR, q = threadIdx.x % GS_LPR;
    const int kmax = (threadIdx.x / 32) * (32 / GS_LPR) + (32 / GS_LPR) - 1;   // the warp's last row
    for (int b = blockIdx.x; b < nblk * GS_W; b += gridDim.x) {
        const int I = b / GS_W, w = b % GS_W + 1;
        float4 *out = reinterpret_cast<float4 *>(panel + (size_t)b * GS_PANEL_TILE);
        __syncthreads();
        for (int e = threadIdx.x; e < GS_B * GS_B; e += blockDim.x) {
            const int r = e / GS_B, c = e % GS_B;
            Th[r * (GS_B + 1) + c] = Thi[(size_t)I * GS_B * GS_B + e];
            Tl[r * (GS_B + 1) + c] = Tlo[(size_t)I * GS_B * GS_B + e];
            const int gr = I * GS_B + r, gc = (I - w) * GS_B + c;
            const bool in = I - w >= 0 && gr < n && gc < n;
            Ah[e] = in ? Ahi[(long long)gr * ld + gc] : 0.f;
            Al[e] = in ? Alo[(long long)gr * ld + gc] : 0.f;
        }
        __syncthreads();
        F2 acc[2][4] = {};
        for (int k = 0; k <= kmax; k++) {
            const float th = Th[row * (GS_B + 1) + k], tl = Tl[row * (GS_B + 1) + k];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int col = h * 32 + q * 4;
                const float4 ah = *reinterpret_cast<const float4 *>(Ah + k * GS_B + col);
                const float4 al = *reinterpret_cast<const float4 *>(Al + k * GS_B + col);
                f2_mac(acc[h][0], th, tl, ah.x, al.x);
                f2_mac(acc[h][1], th, tl, ah.y, al.y);
                f2_mac(acc[h][2], th, tl, ah.z, al.z);
                f2_mac(acc[h][3], th, tl, ah.w, al.w);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            F2 v[4];
            for (int e = 0; e < 4; e++) v[e] = f2_add(acc[h][e], F2{0.f, 0.f});
            out[(2 * h) * GS_C + threadIdx.x] = make_float4(v[0].h, v[1].h, v[2].h, v[3].h);
            out[(2 * h + 1) * GS_C + threadIdx.x] = make_float4(v[0].l, v[1].l, v[2].l, v[3].l);
        }
    }
}

// ---- the triangular solve (cooperative) ------------------------------------------------------
// 16-byte aligned: tile_dot reads the vectors as float4
struct alignas(16) GsShared {
    float dh[GS_W + 1][GS_B], dl[GS_W + 1][GS_B];   // chain: the last d blocks, split
    float vh[2][GS_B], vl[2][GS_B];                   // vectors of the tile products
    float2 ub[GS_UB][GS_B];                           // chain: u_I staged by the fetcher warp
    float sh[GS_B], sl[GS_B];                         // helper: r_I - P_I of the block being finished
    uint64_t full[GS_SLOTS], empty[GS_SLOTS], pub[GS_PUB], uready[GS_UB], ufree[GS_UB];
};

// Row block owned by helper g (0 .. H-1) in round k, or -1: blocks are
// dealt from the last one down in a snake order, so the long rows at the
// bottom and the short ones at the top share helpers.
__device__ __forceinline__ int gs_owned(int g, int H, int k, int nblk) {
    const int p = k * H + ((k & 1) ? H - 1 - g : g);
    return nblk - 1 - p;
}

enum : int { GM_AHI = 0, GM_ALO = 1, GM_THI = 2, GM_TLO = 3 };

// The row blocks helper g owns, ascending; returns how many (<= GS_KMAX).
__device__ __forceinline__ int gs_owned_list(int g, int H, int nblk, int *I) {
    int K = 0;
    for (int k = (nblk + H - 1) / H - 1; k >= 0 && K < GS_KMAX; k--) {
        const int b = gs_owned(g, H, k, nblk);
        if (b >= 0) I[K++] = b;
    }
    return K;
}

// Producer lane: the CTA's tiles in the order its consumers take them
// (chain: A_{I,I-1}, A_{I,I-2}, T_I for I = 0, 1, ...; helper: for each owned
// block A_{I,0} .. A_{I,I-W-1}, T_I).  Before returning it waits for the
// copies of the last ring's worth of tiles, so none is in flight at exit.
__device__ void gs_produce(const GsArgs &a, int nblk, GsShared *S, unsigned char *ring, bool chain) {
    State *st = a.st;
    const CUtensorMap *M = a.tmaps;
    for (int m = 0; m < 4; m++) tmap_acquire(M + m);
    int seq = 0;
    auto put = [&](int mh, int x, int y) -> bool {
        const int sl = seq % GS_SLOTS;
        if (seq >= GS_SLOTS && !mbar_wait(&S->empty[sl], ((seq / GS_SLOTS) - 1) & 1)) {
            set_err(st, ERRB_TIMEOUT);
            return false;
        }
        if (*(volatile int *)&st->err) return false;
        unsigned char *dst = ring + (size_t)sl * GS_SLOT_B;
        mbar_arrive_expect_tx(&S->full[sl], GS_SLOT_B);
        tma_load_2d(dst, M + mh, x, y, &S->full[sl]);
        tma_load_2d(dst + GS_BOX_B, M + mh, x + 32, y, &S->full[sl]);
        tma_load_2d(dst + 2 * GS_BOX_B, M + mh + 1, x, y, &S->full[sl]);
        tma_load_2d(dst + 3 * GS_BOX_B, M + mh + 1, x + 32, y, &S->full[sl]);
        seq++;
        return true;
    };
    auto put_panel = [&](int b) -> bool {
        const int sl = seq % GS_SLOTS;
        if (seq >= GS_SLOTS && !mbar_wait(&S->empty[sl], ((seq / GS_SLOTS) - 1) & 1)) {
            set_err(st, ERRB_TIMEOUT);
            return false;
        }
        if (*(volatile int *)&st->err) return false;
        mbar_arrive_expect_tx(&S->full[sl], GS_SLOT_B);
        bulk_load_1d(ring + (size_t)sl * GS_SLOT_B, a.panel + (size_t)b * GS_PANEL_TILE, GS_SLOT_B, &S->full[sl]);
        seq++;
        return true;
    };
    bool go = true;
    if (chain) {
        for (int I = 0; I < nblk && go; I++)
            for (int w = 1; w <= GS_W && go; w++)
                if (I - w >= 0) go = put_panel(I * GS_W + w - 1);
    } else {
        // the order gs_helper takes them: blocks without tiles first, then
        // for each column j the tiles of the blocks that still have one, then
        // T_I of the block whose last tile that was
        int Iown[GS_KMAX];
        const int K = gs_owned_list(blockIdx.x - 1, gridDim.x - 1, nblk, Iown);
        int jmax = 0;
        for (int m = 0; m < K && go; m++) {
            if (Iown[m] - GS_W <= 0) go = put(GM_THI, 0, Iown[m] * GS_B);
            jmax = max(jmax, Iown[m] - GS_W);
        }
        for (int j = 0; j < jmax && go; j++) {
            for (int m = 0; m < K && go; m++)
                if (j < Iown[m] - GS_W) go = put(GM_AHI, j * GS_B, Iown[m] * GS_B);
            for (int m = 0; m < K && go; m++)
                if (j == Iown[m] - GS_W - 1) go = put(GM_THI, 0, Iown[m] * GS_B);
        }
    }
    for (int k = seq > GS_SLOTS ? seq - GS_SLOTS : 0; k < seq; k++)
        if (!mbar_wait(&S->full[k % GS_SLOTS], (k / GS_SLOTS) & 1)) set_err(st, ERRB_TIMEOUT);
}

// Publisher lane of the chain CTA: flagD[I] once the consumer warps have
// stored d_I (they arrive on pub[I % GS_PUB]).
__device__ void gs_publish(const GsArgs &a, unsigned ep, int nblk, GsShared *S) {
    for (int I = 0; I < nblk; I++) {
        if (!mbar_wait(&S->pub[I % GS_PUB], (I / GS_PUB) & 1)) {
            set_err(a.st, ERRB_TIMEOUT);
            return;
        }
        st_release_u32(&a.flagD[I], ep);
    }
}

// Consumer thread 0 of a helper: wait until d_j is published.  The chain
// publishes in order, so one acquire of flagD[J] covers every j <= J; the
// furthest published flag among the next few is remembered in *known.
__device__ __forceinline__ bool helper_wait_d(const GsArgs &a, unsigned ep, int j, int nblk, int *known) {
    if (j < *known) return true;
    if (!flag_wait(&a.flagD[j], ep, a.st)) return false;
    int k = j + 1;
#pragma unroll
    for (int t = 0; t < 7; t++) {
        if (k >= nblk) break;
        unsigned v;
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(&a.flagD[k]) : "memory");
        if (v != ep) break;
        k++;
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    *known = k;
    return true;
}

// u-fetcher warp of the chain CTA: for I = 0, 1, ... wait until u_I is
// published, copy it into ub[I % GS_UB] and signal uready; a buffer is
// reused once the consumers have signalled ufree.
__device__ void gs_fetch_u(const GsArgs &a, unsigned ep, int nblk, GsShared *S) {
    const int lane = threadIdx.x & 31;
    for (int I = 0; I < nblk; I++) {
        const int b = I % GS_UB;
        bool ok = I < GS_UB || mbar_wait(&S->ufree[b], ((I / GS_UB) - 1) & 1);
        if (lane == 0 && ok) ok = flag_wait(&a.flagU[I], ep, a.st);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (!ok) {
            set_err(a.st, ERRB_TIMEOUT);
            return;
        }
        __syncwarp();
        for (int r = lane; r < GS_B; r += 32) {
            const int gr = I * GS_B + r;
            S->ub[b][r] = gr < a.n ? __ldcg(&a.u[gr]) : make_float2(0.f, 0.f);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&S->uready[b]);
    }
}

// Chain consumers (CTA 0): d_I = u_I - sum_w M_{I,w} d_{I-w}.
__device__ void gs_chain(const GsArgs &a, unsigned ep, int nblk, GsShared *S, const unsigned char *ring) {
    State *st = a.st;
    const int n = a.n, row = threadIdx.x / GS_LPR, q = threadIdx.x % GS_LPR;
    for (int i = threadIdx.x; i < (GS_W + 1) * GS_B; i += GS_C) {
        (&S->dh[0][0])[i] = 0.f;
        (&S->dl[0][0])[i] = 0.f;
    }
    named_bar(GS_BAR_C, GS_C);
    int seq = 0;
    for (int I = 0; I < nblk; I++) {
        const int gr = I * GS_B + row;
        F2 acc = {0.f, 0.f};
        for (int w = 1; w <= GS_W; w++) {
            if (I - w < 0) continue;
            const int sl = seq % GS_SLOTS;
            if (!consumers_wait_full(&S->full[sl], seq, st)) return;
            const int dslot = (I - w) % (GS_W + 1);
            acc = f2_add(acc, tile_dot_panel(ring + (size_t)sl * GS_SLOT_B, S->dh[dslot], S->dl[dslot]));
            consumers_release(&S->empty[sl]);
            seq++;
        }
        const F2 t = f2_row_sum(acc);
        // u_I, staged by the fetcher warp
        const int ubi = I % GS_UB;
        const bool bad = !mbar_wait(&S->uready[ubi], (I / GS_UB) & 1);
        if (bad) set_err(st, ERRB_TIMEOUT);
        if (named_bar_or(GS_BAR_C, GS_C, bad)) return;
        if (q == 0) {
            F2 d = {0.f, 0.f};
            if (gr < n) {
                const float2 u = S->ub[ubi][row];
                d = f2_add(F2{u.x, u.y}, F2{-t.h, -t.l});
                a.delta[gr] = make_float2(d.h, d.l);
            }
            S->dh[I % (GS_W + 1)][row] = d.h;
            S->dl[I % (GS_W + 1)][row] = d.l;
        }
        __syncwarp();
        if ((threadIdx.x & 31) == 0) {
            mbar_arrive(&S->pub[I % GS_PUB]);
            mbar_arrive(&S->ufree[ubi]);
        }
        named_bar(GS_BAR_C, GS_C);   // d_I in shared memory before the next step
    }
}

// Helper consumers: for each owned row block I, P_I = sum over j < I - W of
// A_Ij d_j in column order, all owned blocks together as each d_j is
// published; then u_I = T_I^-1 (r_I - P_I).
__device__ bool gs_helper_finish(const GsArgs &a, unsigned ep, int I, double acc, GsShared *S,
                                 const unsigned char *ring, int *seq) {
    State *st = a.st;
    const int n = a.n, row = threadIdx.x / GS_LPR, q = threadIdx.x % GS_LPR;
    const int r0 = I * GS_B;
    acc = row_sum(acc);
    if (q == 0) {
        const int gr = r0 + row;
        const F2 sv = f2_split(gr < n ? a.r[gr] - acc : 0.0);
        S->sh[row] = sv.h;
        S->sl[row] = sv.l;
    }
    const int sl = *seq % GS_SLOTS;
    if (!consumers_wait_full(&S->full[sl], *seq, st)) return false;   // also orders the s stores
    const F2 t = f2_row_sum(tile_dot(ring + (size_t)sl * GS_SLOT_B, S->sh, S->sl));
    consumers_release(&S->empty[sl]);
    (*seq)++;
    if (q == 0 && r0 + row < n) a.u[r0 + row] = make_float2(t.h, t.l);
    named_bar(GS_BAR_C, GS_C);
    if (threadIdx.x == 0) st_release_u32(&a.flagU[I], ep);
    return true;
}

__device__ void gs_helper(const GsArgs &a, unsigned ep, int nblk, GsShared *S, const unsigned char *ring) {
    State *st = a.st;
    const int n = a.n;
    int Iown[GS_KMAX];
    const int K = gs_owned_list(blockIdx.x - 1, gridDim.x - 1, nblk, Iown);
    double acc[GS_KMAX];
    int jmax = 0;
#pragma unroll
    for (int m = 0; m < GS_KMAX; m++) {
        acc[m] = 0.0;
        if (m < K) jmax = max(jmax, Iown[m] - GS_W);
    }
    int seq = 0, known = 0;
#pragma unroll
    for (int m = 0; m < GS_KMAX; m++)
        if (m < K && Iown[m] - GS_W <= 0 && !gs_helper_finish(a, ep, Iown[m], 0.0, S, ring, &seq)) return;
    for (int j = 0; j < jmax; j++) {
        bool bad = false;
        if (threadIdx.x == 0) bad = !helper_wait_d(a, ep, j, nblk, &known);
        if (named_bar_or(GS_BAR_C, GS_C, bad)) return;
        const int buf = j & 1;
        if (threadIdx.x < GS_B) {
            const int gc = j * GS_B + threadIdx.x;
            const float2 v = gc < n ? __ldcg(&a.delta[gc]) : make_float2(0.f, 0.f);
            S->vh[buf][threadIdx.x] = v.x;
            S->vl[buf][threadIdx.x] = v.y;
        }
#pragma unroll
        for (int m = 0; m < GS_KMAX; m++) {
            if (m >= K || j >= Iown[m] - GS_W) continue;
            const int sl = seq % GS_SLOTS;
            if (!consumers_wait_full(&S->full[sl], seq, st)) return;   // also orders the d_j stores
            acc[m] += f2_value(tile_dot(ring + (size_t)sl * GS_SLOT_B, S->vh[buf], S->vl[buf]));
            consumers_release(&S->empty[sl]);
            seq++;
        }
#pragma unroll
        for (int m = 0; m < GS_KMAX; m++)
            if (m < K && j == Iown[m] - GS_W - 1 && !gs_helper_finish(a, ep, Iown[m], acc[m], S, ring, &seq))
                return;
    }
}

__global__ void __launch_bounds__(GS_T, 1) gs_trsv_kernel(const GsArgs a, cudaGraphConditionalHandle h_loop) {
    extern __shared__ __align__(1024) unsigned char gs_dyn[];
    __shared__ __align__(16) GsShared S;
    unsigned char *ring =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(gs_dyn) + 1023) & ~(uintptr_t)1023);
    State *st = a.st;
    count_launch(st);
    const int stop = *(volatile int *)&st->skip || *(volatile int *)&st->err;
    if (stop) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(st, h_loop, 0u);
        return;
    }
    const unsigned ep = (unsigned)*(volatile int *)&st->iter;
    const int n = a.n, nblk = (n + GS_B - 1) / GS_B;
    const bool chain = blockIdx.x == 0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < GS_SLOTS; i++) {
            mbar_init(&S.full[i], 1);
            mbar_init(&S.empty[i], GS_C / 32);
        }
        for (int i = 0; i < GS_PUB; i++) mbar_init(&S.pub[i], GS_C / 32);
        for (int i = 0; i < GS_UB; i++) {
            mbar_init(&S.uready[i], 1);
            mbar_init(&S.ufree[i], GS_C / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x >= GS_C + 32) {
        if (chain) gs_fetch_u(a, ep, nblk, &S);
    } else if (threadIdx.x >= GS_C) {
        const int lane = threadIdx.x & 31;
        if (lane == 0) gs_produce(a, nblk, &S, ring, chain);
        else if (lane == 1 && chain) gs_publish(a, ep, nblk, &S);
    } else if (chain) {
        gs_chain(a, ep, nblk, &S, ring);
    } else {
        gs_helper(a, ep, nblk, &S, ring);
    }
    // x += d once the chain has published every block (a CTA that gave up
    // on a wait still meets the others here)
    if (!grid_sync(a.bar, st)) return;
    if (*(volatile int *)&st->err) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(st, h_loop, 0u);
        return;
    }
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
    {
        const float2 d = __ldcg(&a.delta[i]);
        a.x[i] += (double)d.x + (double)d.y;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(st, h_loop, 1u);
}

GsKernels gs_kernels() {
    GsKernels K{};
    K.tinv = reinterpret_cast<void *>(&gs_tinv_kernel);
    K.trsv = reinterpret_cast<void *>(&gs_trsv_kernel);
    K.panel = reinterpret_cast<void *>(&gs_panel_kernel);
    K.panel_block = GS_C;
    K.panel_tiles_per_block = GS_W;
    K.panel_tile_floats = GS_PANEL_TILE;
    K.panel_smem = GS_PANEL_SMEM;
    K.max_owned = GS_KMAX;
    K.tinv_block = GS_B;
    K.trsv_block = GS_T;
    K.trsv_smem = (size_t)GS_SLOTS * GS_SLOT_B + 1024;
    K.blk = GS_B;
    set_smem_limit(K.trsv, K.trsv_smem);
    set_smem_limit(K.panel, K.panel_smem);
    return K;
}

bool gs_encode_maps(void *maps, const float *Ahi, const float *Alo, int n, long long ld, const float *Thi,
                    const float *Tlo, int nblk) {
    unsigned char *m = static_cast<unsigned char *>(maps);
    const size_t sz = sizeof(CUtensorMap);
    return encode_f32_tile_map_sw128(m + GM_AHI * sz, Ahi, n, n, ld, 32, GS_B) &&
           encode_f32_tile_map_sw128(m + GM_ALO * sz, Alo, n, n, ld, 32, GS_B) &&
           encode_f32_tile_map_sw128(m + GM_THI * sz, Thi, nblk * GS_B, GS_B, GS_B, 32, GS_B) &&
           encode_f32_tile_map_sw128(m + GM_TLO * sz, Tlo, nblk * GS_B, GS_B, GS_B, 32, GS_B);
}

}  // namespace lsi
