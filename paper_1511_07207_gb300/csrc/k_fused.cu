// k_fused.cu -- CG and GMRES(m) for small dense systems, each solve one
// persistent kernel.
//
// The iterations are those of k_krylov.cu (paper, CG paragraph; GMRES
// pseudocode and restart paragraph): the same recurrences, stop tests,
// true-residual confirmation and restart rules, the same FP32-pair products
// (hi = fp32(a), lo = fp32(a - hi), double-single accumulation) and FP64
// vector arithmetic.  What changes is where the work lives.  For small n a
// step is a few microseconds of arithmetic, but the general path spends tens
// of microseconds per step on kernel launches inside the graph's loop and on
// grid-wide barriers over every SM.  Here one launch of G CTAs runs the whole
// solve:
//  * CTA c owns rows [c R, c R + R) of A; it splits them into the FP32 pair
//    once, at the start, and keeps them in shared memory for the whole solve,
//    so A is read from HBM once per solve, not once per step;
//  * every CTA holds the full vector that multiplies A (the CG direction p,
//    the Arnoldi vector v_j, or x for a residual) as its (hi, lo) split in
//    shared memory, and its own rows of the other vectors (x, r, b, the rows
//    of the Krylov basis V);
//  * a product is warp per row, lanes along the row, double-single
//    accumulation and a butterfly reduction;
//  * the vector a step produces row by row (r, w, x) is exchanged: each CTA
//    publishes its rows, meets the others, and reads the whole vector;
//  * a scalar reduction: each CTA publishes its partial sum into a slot,
//    meets the others, and every CTA adds the G partials of the slot in the
//    same fixed order, so all CTAs hold the same bits and take the same
//    decisions without further communication.
// Two forms of that communication (FComm):
//  * cluster (n up to about 650): the grid is one thread-block cluster of at
//    most 16 CTAs; partial sums and published rows stay in each CTA's shared
//    memory and the others read them through distributed shared memory; the
//    meeting is the hardware cluster barrier (about 0.4 us);
//  * global (larger n, up to one CTA per SM): partial sums and rows go
//    through global memory (L2), and the meeting is a counting grid barrier
//    with a bounded wait (about 1.7 us on this GPU).
// A CG step meets twice (p.Ap; r.r with the exchange of r); an Arnoldi step
// twice (V^T w with ||w||^2; ||w - V h||^2 with the exchange of w and the
// speculative second-pass dots), three times when the second Gram-Schmidt
// pass runs.
//
// Partial-sum slots and exchanged rows are reused step after step.  Each is
// written before a meeting and read after it; its next write comes after a
// later meeting, which no CTA reaches before it has finished reading, so no
// double buffering is needed (the argument for each buffer is at its use).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "ls_device.cuh"
#include "ls_ds.cuh"
#include "ls_internal.h"
#include "split_pair.h"

namespace cg = cooperative_groups;

namespace lsi {

namespace {
constexpr int FT = FUSED_THREADS;   // threads per CTA
constexpr int FW = FT / 32;         // warps per CTA

// CG partial-sum slots
enum : int { CS_PQ = 0, CS_RR = 1, CS_TT = 2, CS_BB = 3, CS_R0 = 4 };
// GMRES partial-sum slots: S1 (first-pass dots and ||A v_j||^2) at 0 .. m + 1,
// S2 (second-pass dots and ||w||^2 after the first pass) at m + 2 .. 2m + 3
__device__ __forceinline__ int gs1(int t) { return t; }
__device__ __forceinline__ int gs2(int m, int t) { return m + 2 + t; }
__device__ __forceinline__ int gs3(int m) { return 2 * m + 4; }   // ||w||^2 after the second pass
__device__ __forceinline__ int gsr(int m) { return 2 * m + 5; }   // ||b - A x||^2
__device__ __forceinline__ int gsb(int m) { return 2 * m + 6; }   // ||b||^2
// the two exchanged vectors
enum : int { EX_V = 0, EX_X = 1 };
}  // namespace

// ---- grid barrier (global form) -----------------------------------------------------
__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// All CTAs meet here.  Barrier e (the CTA's own count, the same in every CTA)
// counts arrivals on c[e % 3] and completes when it reaches G.  The last CTA
// to arrive clears c[(e + 2) % 3]: that counter's last use was barrier e - 1,
// which every CTA has left (they have all arrived at e), and its next use is
// barrier e + 2, which no CTA reaches before this CTA's arrival at e + 1 has
// published the clear.  So no counter is cleared while a CTA still waits on
// it; the three counters must be zero at launch.  Returns false (and sets
// ERRB_TIMEOUT) if the others did not arrive within WAIT_LIMIT_NS.
__device__ __forceinline__ bool fbar_sync(unsigned *c, unsigned &e, State *st) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned i = e % 3u;
        int ok = 1;
        __threadfence();
        const unsigned old = atom_add_acq_rel_u32(&c[i], 1u);
        if (old == gridDim.x - 1) {
            *(volatile unsigned *)&c[(i + 2u) % 3u] = 0u;
        } else {
            unsigned long long t0 = 0;
            for (unsigned spin = 0; ld_acquire_u32(&c[i]) < gridDim.x; spin++) {
                if ((spin & 255u) == 255u) {
                    const unsigned long long t = gtimer();
                    if (t0 == 0) t0 = t;
                    else if (t - t0 > WAIT_LIMIT_NS) {
                        set_err(st, ERRB_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        ok_s = ok;
    }
    e++;
    __syncthreads();
    return ok_s != 0;
}

// ---- communication between the CTAs ---------------------------------------------------
template <bool CL>
struct FComm;

// Global form: any number of co-resident CTAs (cooperative launch).
template <>
struct FComm<false> {
    double *part;        // [slot][G]
    double *ex[2];       // the exchanged vectors, n doubles each
    unsigned *bar;
    unsigned e;
    State *st;
    int G, R;
    __device__ void put(int slot, double v) { part[(size_t)slot * G + blockIdx.x] = v; }
    __device__ double get(int slot, int b) const { return __ldcg(&part[(size_t)slot * G + b]); }
    __device__ void put_row(int w, int i, double v) { ex[w][blockIdx.x * R + i] = v; }
    __device__ double get_elem(int w, int j) const { return __ldcg(&ex[w][j]); }
    __device__ bool meet() { return fbar_sync(bar, e, st); }
    __device__ void leave() {}
};

// Cluster form: the grid is one thread-block cluster.  Each CTA's partial
// sums and published rows stay in its own shared memory; the others read
// them through distributed shared memory after the cluster barrier (whose
// arrive has release and whose wait has acquire semantics).
template <>
struct FComm<true> {
    double *psm;         // this CTA's partial-sum slots
    double *exs[2];      // this CTA's published rows of the two exchanged vectors
    int G, R;
    __device__ void put(int slot, double v) { psm[slot] = v; }
    __device__ double get(int slot, int b) const { return *cg::this_cluster().map_shared_rank(psm + slot, b); }
    __device__ void put_row(int w, int i, double v) { exs[w][i] = v; }
    __device__ double get_elem(int w, int j) const {
        const int b = j / R;
        return *cg::this_cluster().map_shared_rank(exs[w] + (j - b * R), b);
    }
    __device__ bool meet() {
        cg::this_cluster().sync();
        return true;
    }
    // a CTA leaves only when no other still reads its shared memory
    __device__ void leave() { cg::this_cluster().sync(); }
};

// Butterfly sum over the first `width` lanes of the warp (the others hold
// 0), then lane 0's total broadcast, so every lane returns the same bits
// (the callers branch on it, and a branch that splits the warp around a
// full-warp shuffle would never finish).  Only as many levels as the data
// needs: on this GPU a warp's FP64 addition takes about 64 cycles.  Every
// lane of the warp must call it.
__device__ __forceinline__ double lane_sum(double s, int width) {
    int o = 1;
    while (o < width && o < 32) o <<= 1;
    for (o >>= 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return __shfl_sync(0xffffffffu, s, 0);
}

// Sum of slot `slot` over the G CTAs' partials, by the calling warp (every
// lane returns the total).  Every CTA adds the same values in the same
// order, so all CTAs get the same bits.
template <bool CL>
__device__ __forceinline__ double fsum(const FComm<CL> &C, int slot) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < C.G; b += 32) s += C.get(slot, b);
    return lane_sum(s, C.G);
}

// out[t] = sum over the CTAs of slot base + t, t < count: warps take four
// slots at a time (their loads in flight together); the per-slot order is
// fsum's.
template <bool CL>
__device__ __forceinline__ void fsum_slots(const FComm<CL> &C, int base, int count, double *out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int s0 = 4 * warp; s0 < count; s0 += 4 * FW) {
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        for (int b = lane; b < C.G; b += 32) {
            double g[4];
#pragma unroll
            for (int q = 0; q < 4; q++) g[q] = s0 + q < count ? C.get(base + s0 + q, b) : 0.0;
#pragma unroll
            for (int q = 0; q < 4; q++) v[q] += g[q];
        }
        int o = 1;
        while (o < C.G && o < 32) o <<= 1;
        for (o >>= 1; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 4; q++) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < 4; q++)
                if (s0 + q < count) out[s0 + q] = v[q];
    }
}

// ---- shared-memory pieces --------------------------------------------------------------
// The first 16-byte boundary at or after p (the float4 region after the FP64 arrays).
__device__ __forceinline__ float *align16(void *p) {
    return reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15);
}

// The split (hi, lo) of an FP64 value, from its bit pattern (integer
// operations, no FP64 instructions on the common path).
__device__ __forceinline__ DSV split_bits(double v) {
    DSV d;
    split_pair(v, d.h, d.l);
    return d;
}

// This CTA's rows of A as the FP32 pair, row-major with row length nc (n
// padded with zeros to a multiple of 4).
__device__ void load_rows(const double *__restrict__ A, long long lda, int r0, int rows, int n, int nc,
                          float *Ah, float *Al) {
    constexpr int B = 8;   // loads in flight per thread
    const int total = rows * nc;
    for (int e0 = threadIdx.x; e0 < total; e0 += B * FT) {
        double v[B];
#pragma unroll
        for (int u = 0; u < B; u++) {
            const int e = e0 + u * FT;
            const int i = e / nc, j = e - i * nc;
            v[u] = (e < total && j < n) ? A[(long long)(r0 + i) * lda + j] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < B; u++) {
            const int e = e0 + u * FT;
            if (e < total) {
                float h, l;
                split_pair(v[u], h, l);
                Ah[e] = h;
                Al[e] = l;
            }
        }
    }
}

// (vh, vl) = split of v_j = get(j) / scale (scale_it) or get(j), zero
// padding up to nc; the FP64 values optionally kept in keep[].
template <class Get>
__device__ __forceinline__ void load_vec(Get get, int n, int nc, bool scale_it, double scale, float *vh, float *vl,
                                         double *keep) {
    for (int j = threadIdx.x; j < nc; j += FT) {
        double v = 0.0;
        if (j < n) {
            v = get(j);
            if (scale_it) v = v / scale;
        }
        const DSV d = split_bits(v);
        vh[j] = d.h;
        vl[j] = d.l;
        if (keep) keep[j] = v;
    }
}

// q_i = sum_j (hi_ij + lo_ij) v_j for the CTA's rows i < rows, left as the
// double-single pair (qh_i, ql_i); q_i = qh_i + ql_i in FP64 is formed by the
// caller, one lane per row.  Warp w takes rows w, w + 8, ..., four at a time
// (independent chains; the vector chunk is loaded once for the four); lane l
// covers columns 4 l + 128 t (16-byte shared loads, no bank conflicts), two
// double-single chains per row, joined by a butterfly.
__device__ __forceinline__ void product_ds(const float *Ah, const float *Al, const float *vh, const float *vl,
                                           int rows, int nc, float *qh, float *ql) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n4 = nc >> 2;
    const float4 *xh = reinterpret_cast<const float4 *>(vh);
    const float4 *xl = reinterpret_cast<const float4 *>(vl);
    for (int i0 = warp; i0 < rows; i0 += 4 * FW) {
        DSV acc[4][2];
#pragma unroll
        for (int u = 0; u < 4; u++) acc[u][0] = acc[u][1] = DSV{0.f, 0.f};
        for (int c = lane; c < n4; c += 32) {
            const float4 ph = xh[c], pl = xl[c];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int i = i0 + u * FW;
                if (i < rows) {
                    const float4 h = reinterpret_cast<const float4 *>(Ah + (size_t)i * nc)[c];
                    const float4 l = reinterpret_cast<const float4 *>(Al + (size_t)i * nc)[c];
                    ds_fma(h.x, l.x, DSV{ph.x, pl.x}, acc[u][0]);
                    ds_fma(h.y, l.y, DSV{ph.y, pl.y}, acc[u][1]);
                    ds_fma(h.z, l.z, DSV{ph.z, pl.z}, acc[u][0]);
                    ds_fma(h.w, l.w, DSV{ph.w, pl.w}, acc[u][1]);
                }
            }
        }
        DSV t[4];
#pragma unroll
        for (int u = 0; u < 4; u++) t[u] = acc[u][0] + acc[u][1];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int u = 0; u < 4; u++) t[u] += shfl_xor_v(t[u], o);
        if (lane == 0)
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int i = i0 + u * FW;
                if (i < rows) {
                    qh[i] = t[u].h;
                    ql[i] = t[u].l;
                }
            }
    }
}

// ---- per-form setup --------------------------------------------------------------------
template <bool CL>
__device__ FComm<CL> make_comm(const FusedArgs &a, double *psm, double *ex0, double *ex1);
template <>
__device__ FComm<false> make_comm<false>(const FusedArgs &a, double *, double *, double *) {
    FComm<false> C;
    C.part = a.part;
    C.ex[0] = a.xch;
    C.ex[1] = a.xch2;
    C.bar = a.bar;
    C.e = 0;
    C.st = a.st;
    C.G = gridDim.x;
    C.R = a.R;
    return C;
}
template <>
__device__ FComm<true> make_comm<true>(const FusedArgs &a, double *psm, double *ex0, double *ex1) {
    FComm<true> C;
    C.psm = psm;
    C.exs[0] = ex0;
    C.exs[1] = ex1;
    C.G = gridDim.x;
    C.R = a.R;
    return C;
}

// rv[k] = element threadIdx.x + k FT of exchanged vector w (0 past n): the
// loads are issued together, before the caller waits on anything else.
template <bool CL>
__device__ __forceinline__ void prefetch_vec(const FComm<CL> &C, int w, int n, double (&rv)[FUSED_VEC_REGS]) {
#pragma unroll
    for (int k = 0; k < FUSED_VEC_REGS; k++) {
        const int j = threadIdx.x + k * FT;
        rv[k] = j < n ? C.get_elem(w, j) : 0.0;
    }
}

// ============================================================================
// CG (paper, CG paragraph; Hestenes-Stiefel form)
// ============================================================================
// The scalar recurrence (alpha, beta, the stop test, the counters) runs in one
// thread and reaches the others through shared memory (ctl): FP64
// instructions issue at a small fraction of the FP32 rate here, so a value
// that every thread computed would cost the FP64 pipe eight warps over.
struct CgCtl {
    double rho, tol, tol2, inv_rho, rnorm, true_rn, alpha, beta, pq, bn;
    int iter, cycles, status, nan, conv, go;
    int upd, stop;     // this step: update p; leave the CG steps
};

// Shared memory (dynamic): p[nc] (FP64 direction), xr, rr, br, qr (this CTA's
// rows of x, r, b and of the product), ex0, ex1 (cluster form: the rows it
// publishes) [Rp each], psm [FUSED_CG_SLOTS] (cluster form: its partial
// sums), then the FP32 pair of the rows Ah, Al [R nc each], the split vector
// vh, vl [nc each] and the product's double-single rows qh, ql [Rp each].
template <bool CL>
__global__ void __launch_bounds__(FT, 1) cg_fused_kernel(FusedArgs a) {
    extern __shared__ __align__(16) unsigned char fsm[];
    __shared__ CgCtl ctl;
    State *st = a.st;
    count_launch(st);
    const int n = a.n, R = a.R, nc = a.nc, Rp = (a.R + 1) & ~1;
    const int r0 = blockIdx.x * R, rows = min(R, n - r0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *p = reinterpret_cast<double *>(fsm);
    double *xr = p + nc, *rr = xr + Rp, *br = rr + Rp, *qr = br + Rp, *ex0 = qr + Rp, *ex1 = ex0 + Rp;
    double *psm = ex1 + Rp;
    float *Ah = align16(psm + FUSED_CG_SLOTS), *Al = Ah + (size_t)R * nc, *vh = Al + (size_t)R * nc,
          *vl = vh + nc, *qh = vl + nc, *ql = qh + Rp;
    FComm<CL> C = make_comm<CL>(a, psm, ex0, ex1);
    auto ex_v = [&](int j) { return C.get_elem(EX_V, j); };
    auto ex_x = [&](int j) { return C.get_elem(EX_X, j); };
    // q = A v (v in vh, vl) into qr, by warp 0 one lane per row after the product
    auto product = [&]() {
        product_ds(Ah, Al, vh, vl, rows, nc, qh, ql);
        __syncthreads();
    };

    load_rows(a.A, a.lda, r0, rows, n, nc, Ah, Al);
    for (int i = threadIdx.x; i < rows; i += FT) {
        br[i] = a.b[r0 + i];
        xr[i] = a.x0_given ? a.x[r0 + i] : 0.0;
    }
    if (a.x0_given) load_vec([&](int j) { return a.x[j]; }, n, nc, false, 1.0, vh, vl, nullptr);
    __syncthreads();
    // r = b - A x0 (or b); ||b||^2 and ||r||^2
    if (a.x0_given) product();
    if (warp == 0) {
        double bb = 0.0, r2 = 0.0;
        for (int i = lane; i < rows; i += 32) {
            const double ri = a.x0_given ? br[i] - ((double)qh[i] + (double)ql[i]) : br[i];
            rr[i] = ri;
            C.put_row(EX_V, i, ri);
            bb += br[i] * br[i];
            r2 += ri * ri;
        }
        bb = lane_sum(bb, R);
        r2 = lane_sum(r2, R);
        if (lane == 0) {
            C.put(CS_BB, bb);
            C.put(CS_R0, r2);
        }
    }
    if (!C.meet()) return;
    if (warp == 0) {
        const double b2 = fsum(C, CS_BB), r2 = fsum(C, CS_R0);
        if (lane == 0) {
            CgCtl &c = ctl;
            c.bn = sqrt(b2);
            c.tol = a.rtol * c.bn;
            c.tol2 = c.tol * c.tol;
            c.rho = r2;
            c.rnorm = c.true_rn = sqrt(r2);
            c.alpha = c.beta = c.pq = 0.0;
            c.iter = c.cycles = c.status = c.nan = c.conv = 0;
            c.go = 1;
            if (!isfinite(b2) || !isfinite(r2)) {
                c.nan = 1;
                c.go = 0;
            } else if (c.bn == 0.0 || c.rnorm <= c.tol) {
                c.status = LS_OK;   // b = 0 (x = 0), or the start already solves
                c.go = 0;
            } else if (a.max_iter <= 0) {
                c.status = LS_NOT_CONVERGED;
                c.go = 0;
            }
        }
    }
    __syncthreads();
    if (ctl.bn == 0.0 && a.x0_given)   // b = 0: x = 0 solves exactly, whatever x0 was
        for (int i = threadIdx.x; i < rows; i += FT) xr[i] = 0.0;
    // p = r: the published rows hold r (x0 given); b equals r otherwise
    if (ctl.go) {
        if (a.x0_given) load_vec(ex_v, n, nc, false, 1.0, vh, vl, p);
        else load_vec([&](int j) { return a.b[j]; }, n, nc, false, 1.0, vh, vl, p);
    }
    __syncthreads();

    while (ctl.go) {         // residual replacements
        for (;;) {           // CG steps
            // 1 / rho for this step's beta, off the critical path (its
            // latency hides behind the product)
            if (threadIdx.x == FT - 32) ctl.inv_rho = 1.0 / ctl.rho;
            // q = A p, and this CTA's part of p.q (warp 0, a lane per row)
            product();
            if (warp == 0) {
                double s = 0.0;
                for (int i = lane; i < rows; i += 32) {
                    const double q = (double)qh[i] + (double)ql[i];
                    qr[i] = q;
                    s += p[r0 + i] * q;
                }
                s = lane_sum(s, R);
                if (lane == 0) C.put(CS_PQ, s);
            }
            // CS_PQ: its readers finish before they arrive at the r.r meeting
            if (!C.meet()) return;
            // alpha, then x += alpha p, r -= alpha q on this CTA's rows and r
            // published (every reader of its previous rows has passed the
            // p.q meeting): all in warp 0
            if (warp == 0) {
                const double pq = fsum(C, CS_PQ);
                double alpha = 0.0;
                if (lane == 0) {
                    ctl.pq = pq;
                    if (!(pq > 0.0)) {   // non-positive curvature: A is not SPD (or NaN)
                        ctl.status = LS_BREAKDOWN;
                    } else {
                        alpha = ctl.rho / pq;
                    }
                    ctl.alpha = alpha;
                }
                alpha = __shfl_sync(0xffffffffu, alpha, 0);
                if (pq > 0.0) {
                    double s = 0.0;
                    for (int i = lane; i < rows; i += 32) {
                        xr[i] += alpha * p[r0 + i];
                        const double ri = rr[i] - alpha * qr[i];
                        rr[i] = ri;
                        C.put_row(EX_V, i, ri);
                        s += ri * ri;
                    }
                    s = lane_sum(s, R);
                    if (lane == 0) C.put(CS_RR, s);
                }
            }
            __syncthreads();
            if (ctl.status == LS_BREAKDOWN) break;
            if (!C.meet()) return;
            // the whole r in flight while warp 0 adds the partial sums and
            // one thread takes the scalar step
            double rv[FUSED_VEC_REGS];
            prefetch_vec(C, EX_V, n, rv);
            if (warp == 0) {
                const double rho_new = fsum(C, CS_RR);
                if (lane == 0) {
                    CgCtl &c = ctl;
                    const bool finite = isfinite(rho_new);
                    // the stop test ||r|| <= tol as ||r||^2 <= tol^2 and beta
                    // = rho' / rho through the reciprocal formed during the
                    // product: no square root or division on the critical path
                    c.beta = rho_new * c.inv_rho;
                    c.conv = finite && rho_new <= c.tol2;
                    c.upd = finite && !c.conv;
                    c.rho = rho_new;
                    c.iter += 1;
                    if (!finite) c.nan = 1;
                    c.stop = !finite || c.conv || c.iter >= a.max_iter;
                }
            }
            __syncthreads();
            if (ctl.upd) {   // p = r + beta p, the whole vector in every CTA
                const double beta = ctl.beta;
#pragma unroll
                for (int k = 0; k < FUSED_VEC_REGS; k++) {
                    const int j = threadIdx.x + k * FT;
                    if (j < n) {
                        const double pj = rv[k] + beta * p[j];
                        p[j] = pj;
                        const DSV d = split_bits(pj);
                        vh[j] = d.h;
                        vl[j] = d.l;
                    }
                }
            }
            __syncthreads();
            if (ctl.stop) break;
        }
        // the true residual b - A x: x published
        for (int i = threadIdx.x; i < rows; i += FT) C.put_row(EX_X, i, xr[i]);
        if (!C.meet()) return;
        load_vec(ex_x, n, nc, false, 1.0, vh, vl, nullptr);
        __syncthreads();
        product();
        // t = b - A x published: the last readers of r (the p update) have
        // passed the meeting above
        if (warp == 0) {
            double s = 0.0;
            for (int i = lane; i < rows; i += 32) {
                const double ti = br[i] - ((double)qh[i] + (double)ql[i]);
                qr[i] = ti;
                C.put_row(EX_V, i, ti);
                s += ti * ti;
            }
            s = lane_sum(s, R);
            if (lane == 0) C.put(CS_TT, s);
        }
        if (!C.meet()) return;
        if (warp == 0) {
            const double t2 = fsum(C, CS_TT);
            if (lane == 0) {
                CgCtl &c = ctl;
                const double t = sqrt(t2);
                c.true_rn = t;
                c.cycles += 1;
                c.go = 0;
                if (c.nan || !isfinite(t)) c.nan = 1;
                else if (c.status == LS_BREAKDOWN) {
                } else if (t <= c.tol) c.status = LS_OK;
                else if (c.iter >= a.max_iter) c.status = LS_NOT_CONVERGED;
                else {   // restart from the true residual
                    c.go = 1;
                    c.rho = t * t;
                    c.conv = 0;
                }
            }
        }
        __syncthreads();
        if (!ctl.go) break;
        // r = p = b - A x
        for (int i = threadIdx.x; i < rows; i += FT) rr[i] = qr[i];
        load_vec(ex_v, n, nc, false, 1.0, vh, vl, p);
        __syncthreads();
    }
    for (int i = threadIdx.x; i < rows; i += FT) a.x[r0 + i] = xr[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const CgCtl &c = ctl;
        st->bnorm = c.bn;
        st->tol_abs = c.tol;
        st->rho = c.rho;
        st->rnorm = sqrt(c.rho);
        st->true_rnorm = c.true_rn;
        st->alpha = c.alpha;
        st->beta = c.beta;
        st->pq = c.pq;
        st->iter = c.iter;
        st->cycles = c.cycles;
        st->conv = c.conv;
        st->status = c.status;
        if (c.nan) set_err(st, ERRB_NAN);
    }
    C.leave();
}

// ============================================================================
// GMRES(m) (paper, GMRES pseudocode and restart paragraph; least squares by
// Givens rotations)
// ============================================================================
// As for CG, the scalar work runs in one thread (ctl).  Sums over this CTA's
// rows and over the basis run as four interleaved partial sums (FP64
// latency, not throughput, bounds them here); the normalisations multiply by
// a reciprocal formed once; the back substitution is column oriented with the
// reciprocals of R's diagonal formed by the rotations.
struct GmCtl {
    double bn, tol, true_rn, est, wn, inv;
    int total, cycles, status, nan, k, go, pass2, lucky, stop;
};

// Sum over i < cnt of u[i] w[i] (strides su, sw) as four interleaved partial
// sums, added in a fixed order.
__device__ __forceinline__ double dot4(const double *u, int su, const double *w, int sw, int cnt) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = 0;
    for (; i + 4 <= cnt; i += 4) {
        s0 += u[(size_t)i * su] * w[(size_t)i * sw];
        s1 += u[(size_t)(i + 1) * su] * w[(size_t)(i + 1) * sw];
        s2 += u[(size_t)(i + 2) * su] * w[(size_t)(i + 2) * sw];
        s3 += u[(size_t)(i + 3) * su] * w[(size_t)(i + 3) * sw];
    }
    if (i < cnt) s0 += u[(size_t)i * su] * w[(size_t)i * sw];
    if (i + 1 < cnt) s1 += u[(size_t)(i + 1) * su] * w[(size_t)(i + 1) * sw];
    if (i + 2 < cnt) s2 += u[(size_t)(i + 2) * su] * w[(size_t)(i + 2) * sw];
    return (s0 + s1) + (s2 + s3);
}

// Shared memory (dynamic): Vr [(m + 1) Rp] (this CTA's rows of the basis,
// column j at Vr + j Rp), xr, br, wr, ex0, ex1 [Rp each], h1, h2, hs, g, hc
// [m + 2 each], cs, sn, ys, rinv [m + 1 each], q4 [4 max(m + 2, Rp)],
// psm [FUSED_PART_SLOTS], then
// (when h_smem) the rotated Hessenberg matrix Hs [(m + 1) m], then Ah, Al
// [R nc each], vh, vl [nc each] and qh, ql [Rp each].  Every CTA keeps its
// own copy of the rotated Hessenberg matrix (in shared memory, or at
// a.H + blockIdx.x (m + 1) m, column-major); all copies are equal because
// every CTA applies the same rotations to the same numbers.
template <bool CL>
__global__ void __launch_bounds__(FT, 1) gm_fused_kernel(FusedArgs a) {
    extern __shared__ __align__(16) unsigned char fsm[];
    __shared__ GmCtl ctl;
    State *st = a.st;
    count_launch(st);
    const int n = a.n, R = a.R, nc = a.nc, m = a.m, Rp = (a.R + 1) & ~1;
    const int r0 = blockIdx.x * R, rows = min(R, n - r0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *Vr = reinterpret_cast<double *>(fsm);
    double *xr = Vr + (size_t)(m + 1) * Rp, *br = xr + Rp, *wr = br + Rp, *ex0 = wr + Rp, *ex1 = ex0 + Rp;
    double *h1 = ex1 + Rp, *h2 = h1 + (m + 2), *hs = h2 + (m + 2), *g = hs + (m + 2), *hc = g + (m + 2);
    double *cs = hc + (m + 2), *sn = cs + (m + 1), *ys = sn + (m + 1), *rinv = ys + (m + 1);
    const int QS = max(m + 2, Rp);
    double *q4 = rinv + (m + 1);   // [4][QS] quarter sums
    double *psm = q4 + 4 * QS;
    double *Hs = psm + FUSED_PART_SLOTS;
    double *H = a.h_smem ? Hs : a.H + (size_t)blockIdx.x * (m + 1) * m;
    float *Ah = align16(a.h_smem ? Hs + (size_t)(m + 1) * m : Hs);
    float *Al = Ah + (size_t)R * nc, *vh = Al + (size_t)R * nc, *vl = vh + nc, *qh = vl + nc, *ql = qh + Rp;
    const int m1 = m + 1;
    FComm<CL> C = make_comm<CL>(a, psm, ex0, ex1);
    auto ex_x = [&](int j) { return C.get_elem(EX_X, j); };
    // w = A v (v in vh, vl) into wr
    auto product = [&]() {
        product_ds(Ah, Al, vh, vl, rows, nc, qh, ql);
        __syncthreads();
        for (int i = threadIdx.x; i < rows; i += FT) wr[i] = (double)qh[i] + (double)ql[i];
        __syncthreads();
    };
    // A warp's FP64 instruction occupies its scheduler's FP64 unit for about
    // 64 cycles here, dependent or not, so the sums over the rows and over
    // the basis run on four warps (warp w on scheduler w % 4), a quarter
    // each, the quarters added in order.
    // Slot base + t = (column t of V, or w itself for t = ne - 1) . w over this CTA's rows.
    auto dots_put = [&](int ne, int base) {
        for (int e = threadIdx.x; e < 128 * ((ne + 31) / 32); e += FT) {
            const int q = (e >> 5) & 3, t = ((e >> 7) << 5) + (e & 31);
            if (t < ne) {
                const double *u = t < ne - 1 ? Vr + (size_t)t * Rp : wr;
                double s0 = 0.0, s1 = 0.0;
                int i = q;
                for (; i + 4 < rows; i += 8) {
                    s0 += u[i] * wr[i];
                    s1 += u[i + 4] * wr[i + 4];
                }
                if (i < rows) s0 += u[i] * wr[i];
                q4[q * QS + t] = s0 + s1;
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < ne; t += FT)
            C.put(base + t, (q4[t] + q4[QS + t]) + (q4[2 * QS + t] + q4[3 * QS + t]));
    };
    // w_i -= sum_{t < nt} h_t V_ti over this CTA's rows, published: the terms
    // t = q mod 4 on warp q, the four sums added in order.
    auto w_update = [&](const double *h, int nt) {
        for (int e = threadIdx.x; e < 128 * ((rows + 31) / 32); e += FT) {
            const int q = (e >> 5) & 3, i = ((e >> 7) << 5) + (e & 31);
            if (i < rows) {
                double sum = 0.0;
                for (int t = q; t < nt; t += 4) sum += h[t] * Vr[(size_t)t * Rp + i];
                q4[q * QS + i] = sum;
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < rows; i += FT) {
            const double wi = wr[i] - ((q4[i] + q4[QS + i]) + (q4[2 * QS + i] + q4[3 * QS + i]));
            wr[i] = wi;
            C.put_row(EX_V, i, wi);
        }
    };
    // (vh, vl) = split of rv * inv (the whole vector); the CTA's rows of it into V column col
    auto scaled_basis = [&](const double (&rv)[FUSED_VEC_REGS], double inv, int col) {
#pragma unroll
        for (int q = 0; q < FUSED_VEC_REGS; q++) {
            const int jj = threadIdx.x + q * FT;
            if (jj < nc) {
                const DSV d = split_bits(jj < n ? rv[q] * inv : 0.0);
                vh[jj] = d.h;
                vl[jj] = d.l;
            }
        }
        for (int i = threadIdx.x; i < rows; i += FT) Vr[(size_t)col * Rp + i] = wr[i] * inv;
    };

    load_rows(a.A, a.lda, r0, rows, n, nc, Ah, Al);
    for (int i = threadIdx.x; i < rows; i += FT) {
        br[i] = a.b[r0 + i];
        xr[i] = a.x0_given ? a.x[r0 + i] : 0.0;
    }
    if (a.x0_given) load_vec([&](int j) { return a.x[j]; }, n, nc, false, 1.0, vh, vl, nullptr);
    else
        for (int j = threadIdx.x; j < nc; j += FT) vh[j] = vl[j] = 0.f;
    if (threadIdx.x == 0) {
        ctl.total = ctl.cycles = ctl.status = ctl.nan = ctl.k = 0;
        ctl.bn = ctl.tol = ctl.true_rn = ctl.est = 0.0;
    }
    __syncthreads();

    bool first = true;
    double rv[FUSED_VEC_REGS];
    for (;;) {   // cycles: each starts from the true residual
        // r = b - A x (x is in vh, vl), published: the last readers of the
        // previous contents (v_{k+1} of the previous cycle) have passed the
        // meeting that published x
        product();
        if (warp == 0) {
            double s = 0.0, bb = 0.0;
            for (int i = lane; i < rows; i += 32) {
                const double ri = br[i] - wr[i];
                wr[i] = ri;
                C.put_row(EX_V, i, ri);
                s += ri * ri;
                if (first) bb += br[i] * br[i];
            }
            s = lane_sum(s, R);
            if (first) bb = lane_sum(bb, R);
            if (lane == 0) {
                C.put(gsr(m), s);
                if (first) C.put(gsb(m), bb);
            }
        }
        if (!C.meet()) return;
        prefetch_vec(C, EX_V, n, rv);
        if (warp == 0) {
            const double t = fsum(C, gsr(m));
            const double b2 = first ? fsum(C, gsb(m)) : 0.0;
            if (lane == 0) {   // the cycle's start (or the end of the solve)
                GmCtl &c = ctl;
                c.go = 0;
                if (first) {
                    c.bn = sqrt(b2);
                    c.tol = a.rtol * c.bn;
                }
                const double beta = sqrt(t);
                if (first && !isfinite(b2)) c.nan = 1;
                else if (first && c.bn == 0.0) {   // b = 0: x = 0 solves exactly
                    c.status = LS_OK;
                    c.true_rn = 0.0;
                    c.go = -1;
                } else {
                    c.true_rn = beta;
                    if (c.nan || !isfinite(beta)) c.nan = 1;
                    else if (c.status == LS_BREAKDOWN) {
                    } else if (beta <= c.tol) c.status = LS_OK;
                    else if (c.total >= a.max_iter) c.status = LS_NOT_CONVERGED;
                    else {
                        c.go = 1;
                        c.cycles += 1;
                        c.inv = 1.0 / beta;
                        c.est = beta;
                        c.k = 0;
                        g[0] = beta;
                    }
                }
            }
        }
        __syncthreads();
        first = false;
        if (ctl.go < 0)   // b = 0
            for (int i = threadIdx.x; i < rows; i += FT) xr[i] = 0.0;
        if (ctl.go <= 0) break;
        scaled_basis(rv, ctl.inv, 0);   // v_0 = r / beta
        __syncthreads();

        for (int j = 0;; j++) {   // Arnoldi steps; v_j is in vh, vl
            product();
            // first pass: V_j^T w and ||w||^2 over this CTA's rows
            dots_put(j + 2, gs1(0));
            if (!C.meet()) return;
            fsum_slots(C, gs1(0), j + 2, h1);
            __syncthreads();
            // w -= V_j h, published (its readers of the last step have passed
            // the meeting above); the second-pass dots and ||w||^2 published
            // with it
            w_update(h1, j + 1);
            __syncthreads();
            dots_put(j + 2, gs2(m, 0));
            if (!C.meet()) return;
            // w in flight while the sums are formed.  When the second pass
            // runs, a CTA that has taken its decision may overwrite its rows
            // while another still loads them; those loads are discarded and
            // the vector is loaded again after the next meeting.
            prefetch_vec(C, EX_V, n, rv);
            fsum_slots(C, gs2(m, 0), j + 2, h2);
            for (int t = threadIdx.x; t <= j; t += FT) hs[t] = h1[t];
            __syncthreads();
            // a second pass only when cancellation lost accuracy (or always if asked)
            if (threadIdx.x == 0) ctl.pass2 = a.reorth || h2[j + 1] < 0.49 * h1[j + 1];
            __syncthreads();
            if (ctl.pass2) {
                w_update(h2, j + 1);
                __syncthreads();
                if (warp == 0) {
                    double s = 0.0;
                    for (int i = lane; i < rows; i += 32) s += wr[i] * wr[i];
                    s = lane_sum(s, R);
                    if (lane == 0) C.put(gs3(m), s);
                }
                for (int t = threadIdx.x; t <= j; t += FT) hs[t] += h2[t];
                if (!C.meet()) return;
                prefetch_vec(C, EX_V, n, rv);
                if (warp == 0) {
                    const double v = fsum(C, gs3(m));
                    if (lane == 0) h2[j + 1] = v;   // ||w||^2 after the second pass
                }
                __syncthreads();
            }
            if (threadIdx.x == 0) {
                GmCtl &c = ctl;
                c.wn = sqrt(h2[j + 1]);
                c.lucky = !(c.wn > 1e-14 * sqrt(h1[j + 1]));
                c.inv = 1.0 / c.wn;
            }
            __syncthreads();
            // thread 32 takes the new Hessenberg column through the old
            // rotations and forms the new one, while the others form
            // v_{j+1} = w / ||w|| (thread 32 joins them afterwards)
            if (threadIdx.x == 32) {
                GmCtl &c = ctl;
                for (int t = 0; t <= j; t++) hc[t] = hs[t];
                hc[j + 1] = c.wn;
                for (int t = 0; t < j; t++) {
                    const double x0 = hc[t], x1 = hc[t + 1];
                    hc[t] = cs[t] * x0 + sn[t] * x1;
                    hc[t + 1] = -sn[t] * x0 + cs[t] * x1;
                }
                const double den = hypot(hc[j], hc[j + 1]);
                c.stop = 0;
                if (den == 0.0 || !isfinite(den)) {
                    c.status = LS_BREAKDOWN;
                    if (!isfinite(den)) c.nan = 1;
                    c.stop = 1;
                } else {
                    const double cj = hc[j] / den, sj = hc[j + 1] / den;
                    cs[j] = cj;
                    sn[j] = sj;
                    hc[j] = den;
                    hc[j + 1] = 0.0;
                    rinv[j] = 1.0 / den;
                    g[j + 1] = -sj * g[j];
                    g[j] = cj * g[j];
                    c.est = fabs(g[j + 1]);
                    c.k = j + 1;
                    c.total += 1;
                    if (c.est <= c.tol || c.lucky || j + 1 >= m || c.total >= a.max_iter) c.stop = 1;
                }
                double *Hk = H + (size_t)j * m1;
                for (int t = 0; t <= j + 1; t++) Hk[t] = hc[t];
            }
            if (!ctl.lucky) scaled_basis(rv, ctl.inv, j + 1);
            __syncthreads();
            if (ctl.stop) break;
        }
        // end of the cycle: R y = g by columns (warp 0: y_i = g_i / r_ii, then
        // g_t -= r_ti y_i for t < i, lane t), then x += V_k y on this CTA's rows
        const int k = ctl.k;
        if (ctl.status != LS_BREAKDOWN && k > 0) {
            if (warp == 0) {
                for (int i = k - 1; i >= 0; i--) {
                    const double yi = g[i] * rinv[i];
                    if (lane == 0) ys[i] = yi;
                    for (int t = lane; t < i; t += 32) g[t] -= H[(size_t)i * m1 + t] * yi;
                    __syncwarp();
                }
            }
            __syncthreads();
            for (int i = threadIdx.x; i < rows; i += FT) xr[i] += dot4(ys, 1, Vr + i, Rp, k);
        }
        // x published, then the whole x into vh, vl
        for (int i = threadIdx.x; i < rows; i += FT) C.put_row(EX_X, i, xr[i]);
        if (!C.meet()) return;
        load_vec(ex_x, n, nc, false, 1.0, vh, vl, nullptr);
        __syncthreads();
    }
    for (int i = threadIdx.x; i < rows; i += FT) a.x[r0 + i] = xr[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const GmCtl &c = ctl;
        st->bnorm = c.bn;
        st->tol_abs = c.tol;
        st->true_rnorm = c.true_rn;
        st->est = c.est;
        st->rnorm = c.est;
        st->k = c.k;
        st->total = c.total;
        st->iter = c.total;
        st->cycles = c.cycles;
        st->status = c.status;
        if (c.nan) set_err(st, ERRB_NAN);
    }
    C.leave();
}

FusedKernels fused_kernels() {
    FusedKernels K{};
    K.cg = reinterpret_cast<void *>(&cg_fused_kernel<false>);
    K.gmres = reinterpret_cast<void *>(&gm_fused_kernel<false>);
    K.cg_cl = reinterpret_cast<void *>(&cg_fused_kernel<true>);
    K.gmres_cl = reinterpret_cast<void *>(&gm_fused_kernel<true>);
    return K;
}

}  // namespace lsi
