// k_bgemv.cu -- Q = A P for an n x s block P (the block product of block CG),
// A read once as its FP32 pair hi + lo, double-single arithmetic.
//
// One CTA per SM: a producer lane streams, for each of the CTA's 16-row
// blocks and each 256-column tile, the A tile (hi and lo, the solvers' 2-D
// TMA map) and the matching 256-row chunk of P (pre-split into FP32 pairs,
// column panels padded with zeros to a multiple of 256, one 1-D bulk copy
// per column and part) through a ring of shared-memory stages (mbarrier
// full/empty).  Consumer warps: for S <= 8 sixteen warps, warp w owning row
// w of the 16-row block (enough warps to hide the latency of the
// double-single chains); for S = 16 eight warps of two rows each (w and
// w + 8: registers); lane g takes the 4-column chunks g and g + 32 of each
// tile.  A thread accumulates all S columns of P for its rows in
// double-single (two-sum of the high parts, the low parts and rounding
// errors summed apart, as the GEMV does), and the 32 lanes of a row add
// their sums by shuffles at the end of the row block.  Every row block
// belongs to one CTA and is summed in column order, so results are
// deterministic.  Work per element of A is 12 FP32 operations per column of
// P: compute-bound for S >= 4 (HBM-bound below).
#include <cuda_runtime.h>

#include "ls_device.cuh"
#include "ls_internal.h"
#include "split_pair.h"

namespace lsi {

namespace {

constexpr int BG_TR = 16, BG_TC = 256;
constexpr int BG_A_B = BG_TR * BG_TC * 4;   // one part of an A tile (16 KB)

struct F2 {
    float h, l;
};

// acc += (mh + ml)(vh + vl), terms below ml*vl kept, low part unnormalised
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

// a + b with Knuth's two-sum on the high parts, renormalised
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    const float s = __fadd_rn(a.h, b.h);
    const float bb = __fsub_rn(s, a.h);
    const float err = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
    const float l = __fadd_rn(__fadd_rn(a.l, b.l), err);
    const float h = __fadd_rn(s, l);
    return {h, __fsub_rn(l, __fsub_rn(h, s))};
}

// Rows of a 16-row block per consumer warp: one for S <= 8 (sixteen warps,
// to hide the latency of the double-single chains), two for S = 16 (eight
// warps: registers).  Plus the producer warp.
template <int S>
__host__ __device__ constexpr int bg_rows_per_warp() {
    return S <= 8 ? 1 : 2;
}
template <int S>
__host__ __device__ constexpr int bg_consumers() {
    return 32 * 16 / bg_rows_per_warp<S>();
}
template <int S>
__host__ __device__ constexpr int bg_threads() {
    return bg_consumers<S>() + 32;
}

template <int S>
__host__ __device__ constexpr int stages() {
    return S >= 16 ? 3 : 4;
}
template <int S>
__host__ __device__ constexpr size_t stage_bytes() {
    return (size_t)2 * BG_A_B + (size_t)2 * S * BG_TC * 4;
}

}  // namespace

// P (column-major n x s, FP64) -> Ph, Pl (column panels of ldp floats, S of
// them; zero past n and for columns >= s).  With kptr set, P starts at
// P + (*kptr) * kstride (a graph node walking the blocks of a basis).
__global__ void bgemv_split_kernel(int n, int s, int S, const double *__restrict__ P, long long ld,
                                   float *__restrict__ Ph, float *__restrict__ Pl, long long ldp, State *st,
                                   const int *kptr, long long kstride) {
    count_launch(st);
    if (kptr) P += (long long)(*kptr) * kstride;
    const long long total = (long long)S * ldp;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e / ldp);
        const long long c = e % ldp;
        const double v = (j < s && c < n) ? P[(long long)j * ld + c] : 0.0;
        split_pair(v, Ph[e], Pl[e]);
    }
}

template <int S>
__global__ void __launch_bounds__(bg_threads<S>(), 1) bgemv_kernel(const MatDesc *__restrict__ dA, BgemvArgs a) {
    constexpr int BG_C = bg_consumers<S>();
    constexpr int RPW = bg_rows_per_warp<S>(), WS = 16 / RPW;   // rows per warp, their stride
    constexpr int NST = stages<S>();
    constexpr size_t SB = stage_bytes<S>();
    extern __shared__ __align__(1024) unsigned char bg_dyn[];
    unsigned char *ring =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(bg_dyn) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full[NST], empty[NST];
    State *st = a.st;
    count_launch(st);
    const int n = a.n;
    const int RB = (n + BG_TR - 1) / BG_TR, CT = (n + BG_TC - 1) / BG_TC;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NST; i++) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], BG_C / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (threadIdx.x >= BG_C) {
        // ---- producer lane ----
        if ((threadIdx.x & 31) != 0) return;
        const MatDesc &M = *dA;
        tmap_acquire(&M.tmap);
        tmap_acquire(&M.tmap_lo);
        int seq = 0;
        bool go = true;
        for (int rb = blockIdx.x; rb < RB && go; rb += gridDim.x)
            for (int t = 0; t < CT && go; t++) {
                const int sl = seq % NST;
                if (seq >= NST && !mbar_wait(&empty[sl], ((seq / NST) - 1) & 1)) {
                    set_err(st, ERRB_TIMEOUT);
                    go = false;
                    break;
                }
                unsigned char *dst = ring + (size_t)sl * SB;
                mbar_arrive_expect_tx(&full[sl], (unsigned)SB);
                tma_load_2d(dst, &M.tmap, t * BG_TC, rb * BG_TR, &full[sl]);
                tma_load_2d(dst + BG_A_B, &M.tmap_lo, t * BG_TC, rb * BG_TR, &full[sl]);
                for (int j = 0; j < S; j++) {
                    const long long off = (long long)j * a.ldp + (long long)t * BG_TC;
                    bulk_load_1d(dst + 2 * BG_A_B + (size_t)j * BG_TC * 4, a.Ph + off, BG_TC * 4, &full[sl]);
                    bulk_load_1d(dst + 2 * BG_A_B + (size_t)(S + j) * BG_TC * 4, a.Pl + off, BG_TC * 4, &full[sl]);
                }
                seq++;
            }
        // no copy may be in flight when the CTA exits
        for (int k = seq > NST ? seq - NST : 0; k < seq; k++)
            if (!mbar_wait(&full[k % NST], (k / NST) & 1)) set_err(st, ERRB_TIMEOUT);
        return;
    }

    // ---- consumers ----
    // warp w: rows w, w + WS, ... of the block (RPW of them); lane g: the
    // 4-column chunks g and g + 32 of each tile
    const int w = threadIdx.x >> 5, g = threadIdx.x & 31;
    int seq = 0;
    // one row per warp (S <= 8): the two column chunks accumulate apart (two
    // independent chains per column of P), added at the end of the row block
    constexpr int NA = RPW == 1 ? 2 : 1;
    for (int rb = blockIdx.x; rb < RB; rb += gridDim.x) {
        F2 acc[RPW * NA][S];
#pragma unroll
        for (int q = 0; q < RPW * NA; q++)
#pragma unroll
            for (int j = 0; j < S; j++) acc[q][j] = {0.f, 0.f};
        for (int t = 0; t < CT; t++) {
            const int sl = seq % NST;
            const bool ok = mbar_wait(&full[sl], (seq / NST) & 1);
            if (!__all_sync(0xffffffffu, ok)) {   // the warp leaves together
                set_err(st, ERRB_TIMEOUT);
                return;
            }
            const unsigned char *base = ring + (size_t)sl * SB;
            const float *Ah = reinterpret_cast<const float *>(base);
            const float *Al = reinterpret_cast<const float *>(base + BG_A_B);
            const float *Xh = reinterpret_cast<const float *>(base + 2 * BG_A_B);
            const float *Xl = Xh + S * BG_TC;
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const int c0 = (k * 32 + g) * 4;
                float4 ah[RPW], al[RPW];
#pragma unroll
                for (int q = 0; q < RPW; q++) {
                    ah[q] = *reinterpret_cast<const float4 *>(Ah + (w + WS * q) * BG_TC + c0);
                    al[q] = *reinterpret_cast<const float4 *>(Al + (w + WS * q) * BG_TC + c0);
                }
#pragma unroll
                for (int j = 0; j < S; j++) {
                    const float4 xh = *reinterpret_cast<const float4 *>(Xh + j * BG_TC + c0);
                    const float4 xl = *reinterpret_cast<const float4 *>(Xl + j * BG_TC + c0);
#pragma unroll
                    for (int q = 0; q < RPW; q++) {
                        F2 &a2 = acc[NA == 2 ? k : q][j];
                        f2_mac(a2, ah[q].x, al[q].x, xh.x, xl.x);
                        f2_mac(a2, ah[q].y, al[q].y, xh.y, xl.y);
                        f2_mac(a2, ah[q].z, al[q].z, xh.z, xl.z);
                        f2_mac(a2, ah[q].w, al[q].w, xh.w, xl.w);
                    }
                }
            }
            __syncwarp();
            if (g == 0) mbar_arrive(&empty[sl]);
            seq++;
        }
        if constexpr (NA == 2)
#pragma unroll
            for (int j = 0; j < S; j++) acc[0][j] = f2_add(acc[0][j], acc[1][j]);
        // the 32 lanes of a row
#pragma unroll
        for (int q = 0; q < RPW; q++)
#pragma unroll
            for (int j = 0; j < S; j++) {
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    F2 b;
                    b.h = __shfl_xor_sync(0xffffffffu, acc[q][j].h, o);
                    b.l = __shfl_xor_sync(0xffffffffu, acc[q][j].l, o);
                    acc[q][j] = f2_add(acc[q][j], b);
                }
            }
        if (g == 0)
#pragma unroll
            for (int q = 0; q < RPW; q++) {
                const int row = rb * BG_TR + w + WS * q;
                if (row < n)
#pragma unroll
                    for (int j = 0; j < S; j++)
                        if (j < a.s) a.Q[(long long)j * a.ldq + row] = (double)acc[q][j].h + (double)acc[q][j].l;
            }
    }
}

namespace {
template <int S>
void *bg_func() {
    return reinterpret_cast<void *>(&bgemv_kernel<S>);
}
}  // namespace

BgemvLaunch bgemv_plan(int s, int num_sms) {
    BgemvLaunch L{};
    L.split = reinterpret_cast<void *>(&bgemv_split_kernel);
    L.grid = num_sms;
    L.S = s <= 1 ? 1 : s <= 2 ? 2 : s <= 4 ? 4 : s <= 8 ? 8 : 16;
    L.block = L.S <= 8 ? bg_threads<8>() : bg_threads<16>();
    switch (L.S) {
        case 1: L.func = bg_func<1>(); L.smem = stages<1>() * stage_bytes<1>() + 1024; break;
        case 2: L.func = bg_func<2>(); L.smem = stages<2>() * stage_bytes<2>() + 1024; break;
        case 4: L.func = bg_func<4>(); L.smem = stages<4>() * stage_bytes<4>() + 1024; break;
        case 8: L.func = bg_func<8>(); L.smem = stages<8>() * stage_bytes<8>() + 1024; break;
        default: L.func = bg_func<16>(); L.smem = stages<16>() * stage_bytes<16>() + 1024; break;
    }
    set_smem_limit(L.func, L.smem);
    return L;
}

}  // namespace lsi
