// k_gemv.cu -- the dense matrix-vector product y = A x (K1 FP64, K2 BF16 /
// FP8 / FP32 storage) and the quantisation of A (stage A).
//
// The matrix-vector product is the Theta(n^2) operation that every Krylov
// step needs once (paper, section "Serial iterative and direct methods",
// Krylov paragraph: "inner products, saxpy and matrix-vector products");
// it moves all of A, so it is bound by HBM bandwidth (or, for FP64 on
// GB300, by the FP64 FMA pipe: one FMA per 8 bytes of A).
//
// Design (GB300):
//  * persistent grid of 2 CTAs per SM; the (row-tile, column-tile) sequence
//    of A is cut into equal contiguous pieces, one per CTA, so every SM gets
//    the same number of bytes whatever n is;
//  * one producer warp streams TR x TC tiles of A with 2-D TMA bulk copies
//    (cp.async.bulk.tensor) into a 6-deep (3 for FP32 pairs) shared-memory ring with
//    mbarrier completion; four consumer warps read the tiles with 128-bit
//    (64-bit for FP8) shared loads, keep RW row accumulators per lane and
//    the x chunk in registers, and reduce with warp shuffles;
//  * a row tile cut between CTAs leaves partial sums in scratch; the last
//    CTA to finish (atomic ticket) adds them in CTA order, applies the
//    epilogue to those rows and reduces the fused dot product in a fixed
//    order, so results are deterministic for a given n;
//  * fused epilogues: y = s, y = s with z.y, y = b - s with y.y, y = s with
//    y.y, and the Jacobi step y = x + D^-1 (b - s) with (b - s).(b - s);
//    the last CTA runs the solver's scalar update (alpha = rho / p.q,
//    residual norm and stop test, ...) so no extra launch is needed.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "ls_device.cuh"
#include "ls_ds.cuh"
#include "ls_internal.h"
#include "split_pair.h"

namespace lsi {

template <int DT>
struct Cfg;
// T: stored element; V: accumulator; X: vector element read; Y: result stored
template <>
struct Cfg<DT_F64> {
    using T = double;
    using V = double;
    using X = double;
    using Y = double;
    static constexpr int VEC = 2, WC = 4, WR = 1, RW = 8, PARTS = 1;
};
// 16 rows per warp: each lane's split x values (FP64-pipe conversions) serve
// twice as many products as with 8
template <>
struct Cfg<DT_DS> {
    using T = float;    // hi and lo tiles of the same shape, one after the other
    using V = DSV;
    using X = double;
    using Y = double;
    static constexpr int VEC = 2, WC = 4, WR = 1, RW = 16, PARTS = 2;
};
template <>
struct Cfg<DT_BF16> {
    using T = uint16_t;
    using V = float;
    using X = float;
    using Y = float;
    static constexpr int VEC = 8, WC = 1, WR = 4, RW = 8, PARTS = 1;
};
template <>
struct Cfg<DT_FP8> {
    using T = uint8_t;
    using V = float;
    using X = float;
    using Y = float;
    static constexpr int VEC = 8, WC = 1, WR = 4, RW = 16, PARTS = 1;
};
template <>
struct Cfg<DT_F32> {
    using T = float;
    using V = float;
    using X = float;
    using Y = float;
    static constexpr int VEC = 4, WC = 2, WR = 2, RW = 8, PARTS = 1;
};

template <int DT>
struct Geo {
    using C = Cfg<DT>;
    static constexpr int TC = C::WC * 32 * C::VEC;
    static constexpr int TR = C::WR * C::RW;
    static constexpr int TILE_ELEMS = TC * TR;
    static constexpr int TILE_BYTES = TILE_ELEMS * (int)sizeof(typename C::T);
    static_assert(TC <= 256 && TR <= 256, "TMA box dimension");
    static_assert(TR <= GEMV_MAX_TR, "scratch");
    static_assert(C::WC * C::WR == GEMV_CONSUMER_WARPS, "warp grid");
};

// Ring depth: the FP32-pair tiles are twice as large, so fewer stages keep
// two CTAs per SM.
template <int DT>
__host__ __device__ constexpr int stages() { return Cfg<DT>::PARTS > 1 ? 3 : GEMV_STAGES; }

int gemv_tile_rows(int dtype) {
    switch (dtype) {
        case DT_F64: return Geo<DT_F64>::TR;
        case DT_DS: return Geo<DT_DS>::TR;
        case DT_BF16: return Geo<DT_BF16>::TR;
        case DT_FP8: return Geo<DT_FP8>::TR;
        default: return Geo<DT_F32>::TR;
    }
}

// ---- x chunk loads --------------------------------------------------------------
template <int DT>
__device__ __forceinline__ void load_x(const typename Cfg<DT>::X *x, int c0, int cols,
                                       typename Cfg<DT>::V (&p)[Cfg<DT>::VEC]) {
    constexpr int VEC = Cfg<DT>::VEC;
    if constexpr (DT == DT_DS) {        // FP64 x split into (hi, lo) floats
        double v[VEC];
        if (c0 + VEC <= cols && ((reinterpret_cast<uintptr_t>(x) & 15) == 0)) {
            const double2 w = __ldg(reinterpret_cast<const double2 *>(x + c0));
            v[0] = w.x;
            v[1] = w.y;
        } else {
#pragma unroll
            for (int k = 0; k < VEC; k++) v[k] = (c0 + k < cols) ? x[c0 + k] : 0.0;
        }
#pragma unroll
        for (int k = 0; k < VEC; k++) {
            const float h = __double2float_rn(v[k]);
            p[k] = DSV{h, __double2float_rn(v[k] - (double)h)};
        }
    } else if (c0 + VEC <= cols && ((reinterpret_cast<uintptr_t>(x) & 15) == 0)) {
        if constexpr (DT == DT_F64) {
            double2 v = __ldg(reinterpret_cast<const double2 *>(x + c0));
            p[0] = v.x;
            p[1] = v.y;
        } else {
#pragma unroll
            for (int k = 0; k < VEC; k += 4) {
                float4 v = __ldg(reinterpret_cast<const float4 *>(x + c0 + k));
                p[k] = v.x;
                p[k + 1] = v.y;
                p[k + 2] = v.z;
                p[k + 3] = v.w;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < VEC; k++) p[k] = (c0 + k < cols) ? x[c0 + k] : 0;
    }
}

// acc0 + acc1 += a[0:VEC] . p[0:VEC] (two independent FMA chains); `a` points
// at VEC consecutive stored elements in shared memory, aligned to the vector.
template <int DT>
__device__ __forceinline__ void dot_tile(const typename Cfg<DT>::T *a,
                                         const typename Cfg<DT>::V (&p)[Cfg<DT>::VEC],
                                         typename Cfg<DT>::V &acc0, typename Cfg<DT>::V &acc1) {
    if constexpr (DT == DT_F64) {
        double2 v = *reinterpret_cast<const double2 *>(a);
        acc0 = fma(v.x, p[0], acc0);
        acc1 = fma(v.y, p[1], acc1);
    } else if constexpr (DT == DT_DS) {    // the lo tile follows the hi tile
        const float2 h = *reinterpret_cast<const float2 *>(a);
        const float2 l = *reinterpret_cast<const float2 *>(a + Geo<DT>::TILE_ELEMS);
        ds_fma(h.x, l.x, p[0], acc0);
        ds_fma(h.y, l.y, p[1], acc1);
    } else if constexpr (DT == DT_BF16) {
        uint4 v = *reinterpret_cast<const uint4 *>(a);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            acc0 = fmaf(__uint_as_float(w[k] << 16), p[2 * k], acc0);
            acc1 = fmaf(__uint_as_float(w[k] & 0xffff0000u), p[2 * k + 1], acc1);
        }
    } else if constexpr (DT == DT_FP8) {
        uint2 v = *reinterpret_cast<const uint2 *>(a);
        const uint32_t w[2] = {v.x, v.y};
#pragma unroll
        for (int k = 0; k < 2; k++) {
            __half2_raw h0 = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[k] & 0xffffu),
                                                        __NV_E4M3);
            __half2_raw h1 = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[k] >> 16),
                                                        __NV_E4M3);
            float2 f0 = __half22float2(*reinterpret_cast<__half2 *>(&h0));
            float2 f1 = __half22float2(*reinterpret_cast<__half2 *>(&h1));
            acc0 = fmaf(f0.x, p[4 * k + 0], acc0);
            acc1 = fmaf(f0.y, p[4 * k + 1], acc1);
            acc0 = fmaf(f1.x, p[4 * k + 2], acc0);
            acc1 = fmaf(f1.y, p[4 * k + 3], acc1);
        }
    } else {
        float4 v = *reinterpret_cast<const float4 *>(a);
        acc0 = fmaf(v.x, p[0], acc0);
        acc1 = fmaf(v.y, p[1], acc1);
        acc0 = fmaf(v.z, p[2], acc0);
        acc1 = fmaf(v.w, p[3], acc1);
    }
}

// Butterfly transpose-reduction of RW per-lane row accumulators over the warp:
// each round a lane keeps half of its rows and adds the partner's copy of
// them, so RW - 1 + (5 - log2 RW) additions replace RW full reductions.
// Afterwards lane l holds the warp total of row (l >> (5 - log2 RW)).
template <int N, int OFF, class V, int RW>
__device__ __forceinline__ void butterfly(V (&acc)[RW], int lane) {
    if constexpr (OFF >= 1) {
        if constexpr (N > 1) {
            constexpr int H = N / 2;
            const bool upper = (lane & OFF) != 0;
#pragma unroll
            for (int i = 0; i < H; i++) {
                const V send = upper ? acc[i] : acc[i + H];
                const V keep = upper ? acc[i + H] : acc[i];
                acc[i] = keep + shfl_xor_v(send, OFF);
            }
            butterfly<H, OFF / 2>(acc, lane);
        } else {
            acc[0] += shfl_xor_v(acc[0], OFF);
            butterfly<1, OFF / 2>(acc, lane);
        }
    }
}

template <int RW>
__host__ __device__ constexpr int log2i() { return RW <= 1 ? 0 : 1 + log2i<RW / 2>(); }

// plain global loads (fallback when A cannot be described by a TMA map)
template <int DT>
__device__ __forceinline__ void dot_global(const typename Cfg<DT>::T *A, const typename Cfg<DT>::T *Alo,
                                           long long lda, int row, int c0, int cols,
                                           const typename Cfg<DT>::V (&p)[Cfg<DT>::VEC],
                                           typename Cfg<DT>::V &acc, typename Cfg<DT>::V &acc1) {
    using T = typename Cfg<DT>::T;
    const T *a = A + (long long)row * lda;
    if constexpr (DT == DT_DS) {
        const T *al = Alo + (long long)row * lda;
#pragma unroll
        for (int k = 0; k < Cfg<DT>::VEC; k++)
            if (c0 + k < cols) ds_fma(a[c0 + k], al[c0 + k], p[k], (k & 1) ? acc1 : acc);
        return;
    }
#pragma unroll
    for (int k = 0; k < Cfg<DT>::VEC; k++) {
        int c = c0 + k;
        if (c < cols) {
            T e = a[c];
            if constexpr (DT == DT_F64) {
                if (k & 1) acc1 = fma(e, p[k], acc1);
                else acc = fma(e, p[k], acc);
            } else if constexpr (DT == DT_BF16) {
                acc = fmaf(__uint_as_float((uint32_t)e << 16), p[k], acc);
            } else if constexpr (DT == DT_FP8) {
                __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)e, __NV_E4M3);
                acc = fmaf(__half2float(*reinterpret_cast<__half *>(&h)), p[k], acc);
            } else if constexpr (DT == DT_F32) {
                acc = fmaf(e, p[k], acc);
            }
        }
    }
}

// ---- epilogue for one finished row ---------------------------------------------------
template <int DT>
__device__ __forceinline__ double epilogue(const GemvArgs &a, const MatDesc &M, int row,
                                           typename Cfg<DT>::Y s) {
    using V = typename Cfg<DT>::Y;
    if constexpr (DT == DT_FP8) s *= M.scale[row];
    V *y = static_cast<V *>(a.y);
    switch (a.epi) {
        case EPI_STORE:
            y[row] = s;
            return 0.0;
        case EPI_DOT:
            y[row] = s;
            return (double)(static_cast<const V *>(a.z)[row] * s);
        case EPI_RESID: {
            V r = (V)(a.b[row] - (double)s);
            y[row] = r;
            return (double)r * (double)r;
        }
        case EPI_JACOBI: {   // y is the next iterate; x and z are read at this row
            const double r = a.b[row] - (double)s;
            y[row] = (V)((double)static_cast<const V *>(a.x)[row] + static_cast<const double *>(a.z)[row] * r);
            return r * r;
        }
        default:  // EPI_NRM
            y[row] = s;
            return (double)s * (double)s;
    }
}

__device__ __forceinline__ void run_finaliser(const GemvArgs &a, double dot) {
    State *st = a.st;
    if (a.dot_out) *a.dot_out = dot;
    switch (a.fin) {
        case FIN_CG_ALPHA:
            st->pq = dot;
            if (!(dot > 0.0)) {
                st->status = LS_BREAKDOWN;
                st->alpha = 0.0;
            } else {
                st->alpha = st->rho / dot;
            }
            break;
        case FIN_TRUE_RES:
            st->true_rnorm = sqrt(dot);
            break;
        case FIN_WNORM0:
            st->wnorm0 = dot;
            break;
        case FIN_INNER_ALPHA:
            st->in_pq = dot;
            if (!(dot > 0.0)) {
                st->in_stop = 2;    // breakdown of the inner solve: keep the iterate
                st->in_alpha = 0.0;
            } else {
                st->in_alpha = st->in_rho / dot;
            }
            break;
        case FIN_FCG_D:
            st->pq = dot;
            break;
        case FIN_BS_ALPHA:
            st->pq = dot;
            if (dot == 0.0 || !isfinite(dot)) {
                st->status = LS_BREAKDOWN;
                st->alpha = 0.0;
            } else {
                st->alpha = st->rho / dot;
            }
            break;
        case FIN_JACOBI: {
            // the residual of the iterate that was just multiplied; the next
            // iterate is already in y, taken (or not) by the next kernel
            const double rn = sqrt(dot);
            st->rnorm = rn;
            st->true_rnorm = rn;
            int stop = 1;
            if (st->status == LS_BREAKDOWN) {
                // zero diagonal entry: this product only measured x
            } else {
                st->iter++;
                if (!isfinite(dot)) set_err(st, ERRB_NAN);
                else if (rn <= st->tol_abs) st->status = LS_OK;
                else if (st->iter >= st->max_iter) st->status = LS_NOT_CONVERGED;
                else stop = 0;
            }
            st->skip = stop;
            break;
        }
        default:
            st->dot = dot;
            break;
    }
}

// Consumer-warp-only named barrier (ids 1..; 0 is __syncthreads).
__device__ __forceinline__ void consumers_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(GEMV_CONSUMER_WARPS * 32) : "memory");
}

// ---- the kernel ----------------------------------------------------------------------------
// Tile t of the (row tile, column tile) sequence belongs to CTA c with
// start(c) <= t < start(c + 1), start(c) = floor(T c / G).
__device__ __forceinline__ long long tile_start(long long T, int c, int G) { return T * c / G; }
__device__ __forceinline__ int tile_owner(long long t, long long T, int G) {
    return (int)(((long long)G * (t + 1) + T - 1) / T) - 1;
}

template <int DT, bool TMA>
__global__ void __launch_bounds__(GEMV_THREADS, 2)
    gemv_kernel(const MatDesc *__restrict__ dA, GemvArgs args) {
    using C = Cfg<DT>;
    using G = Geo<DT>;
    using T = typename C::T;
    using V = typename C::V;
    using X = typename C::X;
    using Y = typename C::Y;
    constexpr int TC = G::TC, TR = G::TR, VEC = C::VEC, RW = C::RW, WC = C::WC;
    constexpr int STAGE_ELEMS = G::TILE_ELEMS * C::PARTS;
    constexpr int NST = stages<DT>();
    constexpr int LGR = log2i<RW>();
    static_assert((1 << LGR) == RW && RW <= 32, "RW must be a power of two");

    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *ring = reinterpret_cast<T *>(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + (size_t)NST * G::TILE_BYTES * C::PARTS);
    uint64_t *empty = full + NST;
    __shared__ V red[WC][TR];
    __shared__ double dred[GEMV_THREADS / 32];
    __shared__ int abort_s, last_s, fin_s, ca_s, cb_s;
    __shared__ double tdot[TR];

    const MatDesc &M = *dA;
    const int rows = M.rows, cols = M.cols;
    if (args.kptr) {   // walk a stored basis: x = column k, y = column k + kyoff
        const long long k = *args.kptr;
        args.x = static_cast<const X *>(args.x) + k * args.kstride;
        args.y = static_cast<Y *>(args.y) + (k + args.kyoff) * args.kstride;
    }
    if (args.z_is_x) args.z = args.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int RT = (rows + TR - 1) / TR, CT = (cols + TC - 1) / TC;
    const long long T_all = (long long)RT * CT;
    const int G_ = gridDim.x, cta = blockIdx.x;
    const long long t0 = tile_start(T_all, cta, G_), t1 = tile_start(T_all, cta + 1, G_);
    const int ntiles = (int)(t1 - t0);
    count_launch(args.st);

    if (threadIdx.x == 0) {
        abort_s = 0;
        // The dot contribution of a row tile shared between CTAs goes to the
        // slot of the CTA holding its first tile, so that the final sum does
        // not depend on which CTA finished the tile.  A CTA that is not the
        // first holder of a shared tile clears its own slot.
        bool holds_shared_first = false;
        if (ntiles > 0) {
            const long long rl = (t1 - 1) / CT;                 // last row tile of this CTA
            holds_shared_first = (t0 <= rl * CT) && (t1 < (rl + 1) * CT);
        }
        if (!holds_shared_first) args.scr->fixdot[cta] = 0.0;
        if (TMA) {
            for (int s = 0; s < NST; s++) {
                mbar_init(&full[s], 1);
                mbar_init(&empty[s], GEMV_CONSUMER_WARPS);
            }
            fence_mbar_init();
        }
    }
    __syncthreads();

    double mydot = 0.0;
    if (warp == GEMV_CONSUMER_WARPS) {
        // ---------------- producer warp ----------------
        if (TMA && lane == 0 && ntiles > 0) {
            tmap_acquire(&M.tmap);
            if (C::PARTS > 1) tmap_acquire(&M.tmap_lo);
            int issued = 0;
            int rt = (int)(t0 / CT), ct = (int)(t0 % CT);
            for (int i = 0; i < ntiles; i++) {
                const int s = i % NST;
                if (i >= NST) {
                    if (!mbar_wait(&empty[s], ((i / NST) - 1) & 1)) {
                        set_err(args.st, ERRB_TIMEOUT);
                        abort_s = 1;
                        break;
                    }
                }
                if (*(volatile int *)&abort_s) break;
                mbar_arrive_expect_tx(&full[s], G::TILE_BYTES * C::PARTS);
                tma_load_2d(ring + (size_t)s * STAGE_ELEMS, &M.tmap, ct * TC, rt * TR, &full[s]);
                if (C::PARTS > 1)
                    tma_load_2d(ring + (size_t)s * STAGE_ELEMS + G::TILE_ELEMS, &M.tmap_lo, ct * TC, rt * TR,
                                &full[s]);
                issued = i + 1;
                if (++ct == CT) { ct = 0; ++rt; }
            }
            // never leave with copies in flight: wait for the last stages
            for (int i = issued > NST ? issued - NST : 0; i < issued; i++) {
                if (!mbar_wait(&full[i % NST], (i / NST) & 1)) {
                    set_err(args.st, ERRB_TIMEOUT);
                }
            }
        }
    } else {
        // ---------------- consumer warps ----------------
        const int wr = warp / WC, wc = warp % WC;
        const int lane_col = wc * 32 * VEC + lane * VEC;   // column offset inside a tile
        V acc[RW], acc1[RW];
#pragma unroll
        for (int r = 0; r < RW; r++) acc[r] = acc1[r] = V{};
        const T *Ag = static_cast<const T *>(M.ptr);
        const T *Agl = static_cast<const T *>(M.ptr_lo);
        const X *x = static_cast<const X *>(args.x);
        int rt = ntiles > 0 ? (int)(t0 / CT) : 0, ct = ntiles > 0 ? (int)(t0 % CT) : 0;
        const int first_rt = rt;

        for (int i = 0; i < ntiles; i++) {
            V p[VEC];
            load_x<DT>(x, ct * TC + lane_col, cols, p);
            if (TMA) {
                // On a timeout the warp stops waiting and computing but keeps
                // walking the tile sequence, so it still meets the other
                // consumer warps at every named barrier below.
                const int s = i % NST;
                if (!*(volatile int *)&abort_s && !mbar_wait(&full[s], (i / NST) & 1)) {
                    set_err(args.st, ERRB_TIMEOUT);
                    abort_s = 1;
                }
                if (!*(volatile int *)&abort_s) {
                    const T *tile = ring + (size_t)s * STAGE_ELEMS;
#pragma unroll
                    for (int r = 0; r < RW; r++)
                        dot_tile<DT>(tile + (wr * RW + r) * TC + lane_col, p, acc[r], acc1[r]);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
            } else {
#pragma unroll
                for (int r = 0; r < RW; r++) {
                    const int row = rt * TR + wr * RW + r;
                    if (row < rows)
                        dot_global<DT>(Ag, Agl, M.lda, row, ct * TC + lane_col, cols, p, acc[r], acc1[r]);
                }
            }
            if (ct == CT - 1 || i == ntiles - 1) {
                // this CTA's share of row tile rt is done: reduce it over the warp
#pragma unroll
                for (int r = 0; r < RW; r++) {
                    acc[r] += acc1[r];
                    acc1[r] = V{};
                }
                butterfly<RW, 16>(acc, lane);
                if ((lane & ((32 >> LGR) - 1)) == 0) red[wc][wr * RW + (lane >> (5 - LGR))] = acc[0];
#pragma unroll
                for (int r = 0; r < RW; r++) acc[r] = V{};
                consumers_sync();
                const long long rfirst = (long long)rt * CT;
                const bool complete = (t0 <= rfirst) && (rfirst + CT <= t1);
                if (complete) {
                    for (int tr = threadIdx.x; tr < TR; tr += GEMV_CONSUMER_WARPS * 32) {
                        V s{};
#pragma unroll
                        for (int c = 0; c < WC; c++) s += red[c][tr];
                        const int row = rt * TR + tr;
                        if (row < rows) mydot += epilogue<DT>(args, M, row, (Y)to_double(s));
                    }
                } else {
                    // A row tile shared with neighbouring CTAs: publish the
                    // partial sums; the last of the sharing CTAs to arrive adds
                    // them in CTA order and finishes those rows.
                    const int slot = (rt == first_rt) ? 0 : 1;
                    for (int tr = threadIdx.x; tr < TR; tr += GEMV_CONSUMER_WARPS * 32) {
                        V s{};
#pragma unroll
                        for (int c = 0; c < WC; c++) s += red[c][tr];
                        args.scr->fix[((size_t)cta * 2 + slot) * TR + tr] = (double)to_double(s);
                        __threadfence();
                    }
                    consumers_sync();
                    if (threadIdx.x == 0) {
                        const int ca = tile_owner(rfirst, T_all, G_);
                        const int cb = tile_owner(rfirst + CT - 1, T_all, G_);
                        int ncov = 0;
                        for (int c = ca; c <= cb; c++)
                            ncov += tile_start(T_all, c, G_) < tile_start(T_all, c + 1, G_);
                        const unsigned prev = atomicAdd(&args.scr->bticket[ca], 1u);
                        fin_s = (prev == (unsigned)ncov - 1);
                        if (fin_s) atomicExch(&args.scr->bticket[ca], 0u);
                        ca_s = ca;
                        cb_s = cb;
                    }
                    consumers_sync();
                    if (fin_s) {
                        __threadfence();
                        for (int tr = threadIdx.x; tr < TR; tr += GEMV_CONSUMER_WARPS * 32) {
                            double s = 0.0;
                            for (int c = ca_s; c <= cb_s; c++) {
                                const long long a0 = tile_start(T_all, c, G_);
                                if (tile_start(T_all, c + 1, G_) <= a0) continue;   // empty CTA
                                const int sl = (rt == (int)(a0 / CT)) ? 0 : 1;
                                s += __ldcg(&args.scr->fix[((size_t)c * 2 + sl) * TR + tr]);
                            }
                            const int row = rt * TR + tr;
                            tdot[tr] = row < rows ? epilogue<DT>(args, M, row, (Y)s) : 0.0;
                        }
                        consumers_sync();
                        if (threadIdx.x == 0) {
                            double d = 0.0;
                            for (int tr = 0; tr < TR; tr++) d += tdot[tr];
                            args.scr->fixdot[ca_s] = d;
                        }
                    }
                }
                consumers_sync();
            }
            if (++ct == CT) { ct = 0; ++rt; }
        }
    }

    // ---- per-CTA dot; the last CTA reduces them (all threads, fixed order) ----
    double cd = block_sum(mydot, dred);
    if (threadIdx.x == 0) {
        args.scr->cta_dot[cta] = cd;
        __threadfence();
        unsigned tk = atomicAdd(&args.scr->ticket, 1u);
        last_s = (tk == (unsigned)G_ - 1);
    }
    __syncthreads();
    if (!last_s) return;
    __threadfence();
    double part = 0.0;
    for (int c = threadIdx.x; c < G_; c += GEMV_THREADS)
        part += __ldcg(&args.scr->cta_dot[c]) + __ldcg(&args.scr->fixdot[c]);
    const double tot = block_sum(part, dred);
    if (threadIdx.x == 0) {
        run_finaliser(args, tot);
        atomicExch(&args.scr->ticket, 0u);
    }
}

// ---- host side -------------------------------------------------------------------------
template <int DT>
static size_t gemv_smem() {
    return (size_t)stages<DT>() * Geo<DT>::TILE_BYTES * Cfg<DT>::PARTS + 2 * stages<DT>() * sizeof(uint64_t);
}

template <int DT, bool TMA>
static void *gemv_func() {
    return reinterpret_cast<void *>(&gemv_kernel<DT, TMA>);
}

GemvLaunch gemv_plan(int dtype, bool use_tma, int epi, int num_sms) {
    (void)epi;
    GemvLaunch L{};
    L.block = GEMV_THREADS;
    L.grid = 2 * num_sms;
    switch (dtype) {
        case DT_F64:
            L.func = use_tma ? gemv_func<DT_F64, true>() : gemv_func<DT_F64, false>();
            L.smem = gemv_smem<DT_F64>();
            break;
        case DT_DS:
            L.func = use_tma ? gemv_func<DT_DS, true>() : gemv_func<DT_DS, false>();
            L.smem = gemv_smem<DT_DS>();
            break;
        case DT_BF16:
            L.func = use_tma ? gemv_func<DT_BF16, true>() : gemv_func<DT_BF16, false>();
            L.smem = gemv_smem<DT_BF16>();
            break;
        case DT_FP8:
            L.func = use_tma ? gemv_func<DT_FP8, true>() : gemv_func<DT_FP8, false>();
            L.smem = gemv_smem<DT_FP8>();
            break;
        default:
            L.func = use_tma ? gemv_func<DT_F32, true>() : gemv_func<DT_F32, false>();
            L.smem = gemv_smem<DT_F32>();
            break;
    }
    if (!use_tma) L.smem = 2 * GEMV_STAGES * sizeof(uint64_t);   // barriers only (no ring)
    set_smem_limit(L.func, L.smem);
    if (L.grid > MAX_GRID) L.grid = MAX_GRID;
    return L;
}

cudaError_t gemv_launch(const GemvLaunch &L, const MatDesc *dA, const GemvArgs &a,
                        cudaStream_t s) {
    GemvArgs aa = a;
    void *params[] = {(void *)&dA, (void *)&aa};
    return cudaLaunchKernel(L.func, dim3(L.grid), dim3(L.block), params, L.smem, s);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    // initialised once, thread-safe (function-local static)
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<EncodeTiledFn>(p);
        return nullptr;
    }();
    return fn;
}

bool make_tensor_map(MatDesc *h, int dtype, const void *ptr, int rows, int cols, long long lda) {
    h->ptr = ptr;
    h->lda = lda;
    h->rows = rows;
    h->cols = cols;
    h->dtype = dtype;
    h->use_tma = 0;
    const int esz = dtype == DT_F64 ? 8 : dtype == DT_BF16 ? 2 : dtype == DT_FP8 ? 1 : 4;
    const int tc = dtype == DT_F64 ? Geo<DT_F64>::TC : dtype == DT_BF16 ? Geo<DT_BF16>::TC
                   : dtype == DT_FP8 ? Geo<DT_FP8>::TC : Geo<DT_F32>::TC;
    const int tr = gemv_tile_rows(dtype);
    EncodeTiledFn fn = encode_fn();
    if (!fn || rows <= 0 || cols <= 0) return false;
    if (((uintptr_t)ptr & 15) != 0 || ((lda * esz) & 15) != 0) return false;
    if ((unsigned long long)lda * esz >= (1ull << 40)) return false;
    CUtensorMapDataType dt = dtype == DT_F64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                             : dtype == DT_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                             : dtype == DT_FP8  ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                                : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t gstride[1] = {(cuuint64_t)lda * esz};
    cuuint32_t box[2] = {(cuuint32_t)tc, (cuuint32_t)tr};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(&h->tmap, dt, 2, const_cast<void *>(ptr), gdim, gstride, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    h->use_tma = 1;
    return true;
}

bool make_tensor_map_ds(MatDesc *h, const float *hi, const float *lo, int rows, int cols, long long ld) {
    h->ptr = hi;
    h->ptr_lo = lo;
    h->lda = ld;
    h->rows = rows;
    h->cols = cols;
    h->dtype = DT_DS;
    h->use_tma = 0;
    EncodeTiledFn fn = encode_fn();
    if (!fn || rows <= 0 || cols <= 0) return false;
    if (((uintptr_t)hi & 15) != 0 || ((uintptr_t)lo & 15) != 0 || ((ld * 4) & 15) != 0) return false;
    cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t gstride[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {(cuuint32_t)Geo<DT_DS>::TC, (cuuint32_t)Geo<DT_DS>::TR};
    cuuint32_t estr[2] = {1, 1};
    for (int part = 0; part < 2; part++) {
        CUresult r = fn(part ? &h->tmap_lo : &h->tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                        const_cast<float *>(part ? lo : hi), gdim, gstride, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    }
    h->use_tma = 1;
    return true;
}

// hi = fp32(A), lo = fp32(A - hi): one pass over A, done once per solve
// (split_pair: integer operations on the bit pattern, off the FP64 pipe).
// Any alignment: a CTA a row, a thread an element.
__global__ void split_f64_kernel(int rows, int cols, const double *__restrict__ A, long long lda,
                                 float *__restrict__ hi, float *__restrict__ lo, long long ld) {
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const double *a = A + (long long)row * lda;
        float *h = hi + (long long)row * ld, *l = lo + (long long)row * ld;
        for (int j = threadIdx.x; j < cols; j += blockDim.x) split_pair(__ldcs(&a[j]), h[j], l[j]);
    }
}

// The same with 16-byte accesses: A rows 16-byte aligned (lda even), hi and lo
// rows 16-byte aligned (ld a multiple of 4).  A thread takes SPLIT_U groups of
// four elements at a time (two 16-byte loads each, all issued before the
// arithmetic); the last cols % 4 elements of a row go one a thread.  A is read
// once and streamed past the caches.
constexpr int SPLIT_U = 2;
__global__ void __launch_bounds__(256) split_f64_vec_kernel(int rows, int cols, const double *__restrict__ A,
                                                            long long lda, float *__restrict__ hi,
                                                            float *__restrict__ lo, long long ld) {
    const int q4 = cols >> 2;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const double2 *a = reinterpret_cast<const double2 *>(A + (long long)row * lda);
        float4 *h = reinterpret_cast<float4 *>(hi + (long long)row * ld);
        float4 *l = reinterpret_cast<float4 *>(lo + (long long)row * ld);
        for (int q0 = threadIdx.x; q0 < q4; q0 += SPLIT_U * blockDim.x) {
            double2 v[SPLIT_U][2];
#pragma unroll
            for (int u = 0; u < SPLIT_U; u++) {
                const int q = q0 + u * blockDim.x;
                if (q < q4) {
                    v[u][0] = __ldcs(&a[2 * q]);
                    v[u][1] = __ldcs(&a[2 * q + 1]);
                }
            }
#pragma unroll
            for (int u = 0; u < SPLIT_U; u++) {
                const int q = q0 + u * blockDim.x;
                if (q < q4) {
                    float4 hv, lv;
                    split_pair(v[u][0].x, hv.x, lv.x);
                    split_pair(v[u][0].y, hv.y, lv.y);
                    split_pair(v[u][1].x, hv.z, lv.z);
                    split_pair(v[u][1].y, hv.w, lv.w);
                    h[q] = hv;
                    l[q] = lv;
                }
            }
        }
        for (int j = 4 * q4 + threadIdx.x; j < cols; j += blockDim.x)
            split_pair(__ldcs(&A[(long long)row * lda + j]), hi[(long long)row * ld + j], lo[(long long)row * ld + j]);
    }
}

cudaError_t split_f64_launch(int rows, int cols, const double *A, long long lda, float *hi, float *lo,
                             long long ld, int num_sms, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const int grid = rows < 8 * num_sms ? rows : 8 * num_sms;
    const bool vec = ((uintptr_t)A & 15) == 0 && (lda & 1) == 0 && ((uintptr_t)hi & 15) == 0 &&
                     ((uintptr_t)lo & 15) == 0 && (ld & 3) == 0;
    if (vec) split_f64_vec_kernel<<<grid, 256, 0, s>>>(rows, cols, A, lda, hi, lo, ld);
    else split_f64_kernel<<<grid, 256, 0, s>>>(rows, cols, A, lda, hi, lo, ld);
    return cudaGetLastError();
}

bool encode_f32_tile_map_sw128(void *map, const float *ptr, int rows, int cols, long long ld,
                               int box_cols, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn || rows <= 0 || cols <= 0 || box_cols * 4 > 128) return false;
    if (((uintptr_t)ptr & 15) != 0 || ((ld * 4) & 15) != 0 || ((uintptr_t)map & 63) != 0) return false;
    cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t gstride[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(static_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                    const_cast<float *>(ptr), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// ---- quantisation of A (stage A, done once per solve) ------------------------------------
// BF16: round-to-nearest-even directly from FP64.  FP32: the same to FP32.
// FP8-e4m3: s_i = fp32(max_j |a_ij| / 448) (1 when that is 0), then
// q_ij = e4m3 round-to-nearest-even, saturating, of a_ij / s_i (FP64 division).
__global__ void quantize_kernel(int dtype, int rows, int cols, const double *__restrict__ A,
                                long long lda, void *Q, long long ldq, float *scale) {
    __shared__ double red[32];
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const double *a = A + (long long)row * lda;
        if (dtype == DT_FP8) {
            double mx = 0.0;
            for (int j = threadIdx.x; j < cols; j += blockDim.x) mx = fmax(mx, fabs(a[j]));
            // block max (fixed order)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            __syncthreads();
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
            __syncthreads();
            mx = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) mx = fmax(mx, red[w]);
            float s = __double2float_rn(mx / 448.0);
            if (!(s > 0.0f)) s = 1.0f;
            if (threadIdx.x == 0) scale[row] = s;
            const double sd = (double)s;
            uint8_t *q = static_cast<uint8_t *>(Q) + (long long)row * ldq;
            for (int j = threadIdx.x; j < cols; j += blockDim.x)
                q[j] = (uint8_t)__nv_cvt_double_to_fp8(a[j] / sd, __NV_SATFINITE, __NV_E4M3);
        } else if (dtype == DT_BF16) {
            __nv_bfloat16 *q = static_cast<__nv_bfloat16 *>(Q) + (long long)row * ldq;
            for (int j = threadIdx.x; j < cols; j += blockDim.x) q[j] = __double2bfloat16(a[j]);
        } else {
            float *q = static_cast<float *>(Q) + (long long)row * ldq;
            for (int j = threadIdx.x; j < cols; j += blockDim.x) q[j] = __double2float_rn(a[j]);
        }
    }
}

cudaError_t quantize_launch(int dtype, int rows, int cols, const double *A, long long lda,
                            void *Q, long long ldq, float *scale, int num_sms, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    int grid = rows < 8 * num_sms ? rows : 8 * num_sms;
    quantize_kernel<<<grid, 256, 0, s>>>(dtype, rows, cols, A, lda, Q, ldq, scale);
    return cudaGetLastError();
}

}  // namespace lsi
