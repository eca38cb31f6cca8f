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

// Sum of slot `slot` over the G CTAs' partials, by the calling warp.  Every
// CTA adds the same values in the same order, and the butterfly leaves the
// same bits in every lane.
template <bool CL>
__device__ __forceinline__ double fsum(const FComm<CL> &C, int slot) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < C.G; b += 32) s += C.get(slot, b);
    return warp_sum(s);
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
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const double t = warp_sum(v[q]);
            if (lane == 0 && s0 + q < count) out[s0 + q] = t;
        }
    }
}

// ---- shared-memory pieces --------------------------------------------------------------
// The first 16-byte boundary at or after p (the float4 region after the FP64 arrays).
__device__ __forceinline__ float *align16(void *p) {
    return reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15);
}

// This CTA's rows of A as the FP32 pair, row-major with row length nc (n
// padded with zeros to a multiple of 4).
__device__ void load_rows(const double *__restrict__ A, long long lda, int r0, int rows, int n, int nc,
                          float *Ah, float *Al) {
    const int total = rows * nc;
    for (int e = threadIdx.x; e < total; e += FT) {
        const int i = e / nc, j = e - i * nc;
        float h = 0.f, l = 0.f;
        if (j < n) split_pair(A[(long long)(r0 + i) * lda + j], h, l);
        Ah[e] = h;
        Al[e] = l;
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
        const DSV d = ds_split(v);
        vh[j] = d.h;
        vl[j] = d.l;
        if (keep) keep[j] = v;
    }
}

// q_i = sum_j (hi_ij + lo_ij) v_j for the CTA's rows i < rows (FP64 out).
// Warp per row, lane l on columns 4 l + 128 t (16-byte shared loads, no bank
// conflicts), two double-single chains per lane joined by a butterfly.
__device__ __forceinline__ void fused_product(const float *Ah, const float *Al, const float *vh, const float *vl,
                                              int rows, int nc, double *q) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n4 = nc >> 2;
    const float4 *xh = reinterpret_cast<const float4 *>(vh);
    const float4 *xl = reinterpret_cast<const float4 *>(vl);
    for (int i = warp; i < rows; i += FW) {
        const float4 *ah = reinterpret_cast<const float4 *>(Ah + (size_t)i * nc);
        const float4 *al = reinterpret_cast<const float4 *>(Al + (size_t)i * nc);
        DSV a0{0.f, 0.f}, a1{0.f, 0.f};
        for (int c = lane; c < n4; c += 32) {
            const float4 h = ah[c], l = al[c], ph = xh[c], pl = xl[c];
            ds_fma(h.x, l.x, DSV{ph.x, pl.x}, a0);
            ds_fma(h.y, l.y, DSV{ph.y, pl.y}, a1);
            ds_fma(h.z, l.z, DSV{ph.z, pl.z}, a0);
            ds_fma(h.w, l.w, DSV{ph.w, pl.w}, a1);
        }
        DSV a = a0 + a1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += shfl_xor_v(a, o);
        if (lane == 0) q[i] = to_double(a);
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
// Shared memory (dynamic): p[nc] (FP64 direction), xr, rr, br, qr (this CTA's
// rows of x, r, b and of the product), ex0, ex1 (cluster form: the rows it
// publishes) [Rp each], psm [FUSED_CG_SLOTS] (cluster form: its partial
// sums), then the FP32 pair of the rows Ah, Al [R nc each] and the split
// vector vh, vl [nc each].
template <bool CL>
__global__ void __launch_bounds__(FT, 1) cg_fused_kernel(FusedArgs a) {
    extern __shared__ __align__(16) unsigned char fsm[];
    __shared__ double sc[4];
    State *st = a.st;
    count_launch(st);
    const int n = a.n, R = a.R, nc = a.nc, Rp = (a.R + 1) & ~1;
    const int r0 = blockIdx.x * R, rows = min(R, n - r0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *p = reinterpret_cast<double *>(fsm);
    double *xr = p + nc, *rr = xr + Rp, *br = rr + Rp, *qr = br + Rp, *ex0 = qr + Rp, *ex1 = ex0 + Rp;
    double *psm = ex1 + Rp;
    float *Ah = align16(psm + FUSED_CG_SLOTS), *Al = Ah + (size_t)R * nc, *vh = Al + (size_t)R * nc,
          *vl = vh + nc;
    FComm<CL> C = make_comm<CL>(a, psm, ex0, ex1);
    auto ex_v = [&](int j) { return C.get_elem(EX_V, j); };
    auto ex_x = [&](int j) { return C.get_elem(EX_X, j); };

    load_rows(a.A, a.lda, r0, rows, n, nc, Ah, Al);
    for (int i = threadIdx.x; i < rows; i += FT) {
        br[i] = a.b[r0 + i];
        xr[i] = a.x0_given ? a.x[r0 + i] : 0.0;
    }
    if (a.x0_given) load_vec([&](int j) { return a.x[j]; }, n, nc, false, 1.0, vh, vl, nullptr);
    __syncthreads();
    // r = b - A x0 (or b); ||b||^2 and ||r||^2
    if (a.x0_given) {
        fused_product(Ah, Al, vh, vl, rows, nc, qr);
        __syncthreads();
    }
    if (warp == 0) {
        double bb = 0.0, r2 = 0.0;
        for (int i = lane; i < rows; i += 32) {
            const double ri = a.x0_given ? br[i] - qr[i] : br[i];
            rr[i] = ri;
            C.put_row(EX_V, i, ri);
            bb += br[i] * br[i];
            r2 += ri * ri;
        }
        bb = warp_sum(bb);
        r2 = warp_sum(r2);
        if (lane == 0) {
            C.put(CS_BB, bb);
            C.put(CS_R0, r2);
        }
    }
    if (!C.meet()) return;
    if (warp == 0) {
        const double b2 = fsum(C, CS_BB), r2 = fsum(C, CS_R0);
        if (lane == 0) {
            sc[0] = b2;
            sc[1] = r2;
        }
    }
    __syncthreads();
    const double b2 = sc[0];
    double rho = sc[1];
    if (b2 == 0.0 && a.x0_given)   // b = 0: x = 0 solves exactly, whatever x0 was
        for (int i = threadIdx.x; i < rows; i += FT) xr[i] = 0.0;
    const double bn = sqrt(b2), tol = a.rtol * bn;
    double rnorm = sqrt(rho), true_rn = sqrt(rho), alpha = 0.0, beta = 0.0, pq = 0.0;
    int iter = 0, cycles = 0, status = 0, nan = 0, conv = 0;
    bool go = true;
    if (!isfinite(b2) || !isfinite(rho)) {
        nan = 1;
        go = false;
    } else if (bn == 0.0 || sqrt(rho) <= tol) {
        status = LS_OK;   // b = 0 (x = 0), or the start already solves
        go = false;
    } else if (a.max_iter <= 0) {
        status = LS_NOT_CONVERGED;
        go = false;
    }
    // p = r: the published rows hold r (x0 given); b equals r otherwise
    if (go) {
        if (a.x0_given) load_vec(ex_v, n, nc, false, 1.0, vh, vl, p);
        else load_vec([&](int j) { return a.b[j]; }, n, nc, false, 1.0, vh, vl, p);
    }
    __syncthreads();

    while (go) {             // residual replacements
        for (;;) {           // CG steps
            // q = A p and this CTA's part of p.q
            fused_product(Ah, Al, vh, vl, rows, nc, qr);
            __syncthreads();
            if (warp == 0) {
                double s = 0.0;
                for (int i = lane; i < rows; i += 32) s += p[r0 + i] * qr[i];
                s = warp_sum(s);
                if (lane == 0) C.put(CS_PQ, s);
            }
            // CS_PQ: its readers finish before they arrive at the r.r meeting
            if (!C.meet()) return;
            if (warp == 0) {
                const double t = fsum(C, CS_PQ);
                if (lane == 0) sc[0] = t;
            }
            __syncthreads();
            pq = sc[0];
            if (!(pq > 0.0)) {   // non-positive curvature: A is not SPD (or NaN)
                status = LS_BREAKDOWN;
                alpha = 0.0;
                break;
            }
            alpha = rho / pq;
            // x += alpha p, r -= alpha q on this CTA's rows; r published
            // (every reader of its previous rows has passed the p.q meeting)
            if (warp == 0) {
                double s = 0.0;
                for (int i = lane; i < rows; i += 32) {
                    xr[i] += alpha * p[r0 + i];
                    const double ri = rr[i] - alpha * qr[i];
                    rr[i] = ri;
                    C.put_row(EX_V, i, ri);
                    s += ri * ri;
                }
                s = warp_sum(s);
                if (lane == 0) C.put(CS_RR, s);
            }
            if (!C.meet()) return;
            // the whole r in flight while warp 0 adds the partial sums
            double rv[FUSED_VEC_REGS];
            prefetch_vec(C, EX_V, n, rv);
            if (warp == 0) {
                const double t = fsum(C, CS_RR);
                if (lane == 0) sc[1] = t;
            }
            __syncthreads();
            const double rho_new = sc[1];
            const bool finite = isfinite(rho_new);
            conv = finite && sqrt(rho_new) <= tol;
            beta = rho_new / rho;
            if (finite && !conv) {   // p = r + beta p, the whole vector in every CTA
#pragma unroll
                for (int k = 0; k < FUSED_VEC_REGS; k++) {
                    const int j = threadIdx.x + k * FT;
                    if (j < n) {
                        const double pj = rv[k] + beta * p[j];
                        p[j] = pj;
                        const DSV d = ds_split(pj);
                        vh[j] = d.h;
                        vl[j] = d.l;
                    }
                }
            }
            rho = rho_new;
            rnorm = sqrt(rho_new);
            iter++;
            if (!finite) nan = 1;
            __syncthreads();
            if (!finite || conv || iter >= a.max_iter) break;
        }
        // the true residual b - A x: x published
        for (int i = threadIdx.x; i < rows; i += FT) C.put_row(EX_X, i, xr[i]);
        if (!C.meet()) return;
        load_vec(ex_x, n, nc, false, 1.0, vh, vl, nullptr);
        __syncthreads();
        fused_product(Ah, Al, vh, vl, rows, nc, qr);
        __syncthreads();
        // t = b - A x published: the last readers of r (the p update) have
        // passed the meeting above
        if (warp == 0) {
            double s = 0.0;
            for (int i = lane; i < rows; i += 32) {
                const double ti = br[i] - qr[i];
                qr[i] = ti;
                C.put_row(EX_V, i, ti);
                s += ti * ti;
            }
            s = warp_sum(s);
            if (lane == 0) C.put(CS_TT, s);
        }
        if (!C.meet()) return;
        if (warp == 0) {
            const double t = fsum(C, CS_TT);
            if (lane == 0) sc[2] = t;
        }
        __syncthreads();
        const double t = sqrt(sc[2]);
        true_rn = t;
        cycles++;
        if (nan || !isfinite(t)) {
            nan = 1;
            break;
        }
        if (status == LS_BREAKDOWN) break;
        if (t <= tol) {
            status = LS_OK;
            break;
        }
        if (iter >= a.max_iter) {
            status = LS_NOT_CONVERGED;
            break;
        }
        // restart from the true residual: r = p = b - A x
        for (int i = threadIdx.x; i < rows; i += FT) rr[i] = qr[i];
        load_vec(ex_v, n, nc, false, 1.0, vh, vl, p);
        rho = t * t;
        rnorm = t;
        conv = 0;
        __syncthreads();
    }
    for (int i = threadIdx.x; i < rows; i += FT) a.x[r0 + i] = xr[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->bnorm = bn;
        st->tol_abs = tol;
        st->rho = rho;
        st->rnorm = rnorm;
        st->true_rnorm = true_rn;
        st->alpha = alpha;
        st->beta = beta;
        st->pq = pq;
        st->iter = iter;
        st->cycles = cycles;
        st->conv = conv;
        st->status = status;
        if (nan) set_err(st, ERRB_NAN);
    }
    C.leave();
}

// ============================================================================
// GMRES(m) (paper, GMRES pseudocode and restart paragraph; least squares by
// Givens rotations)
// ============================================================================
// Shared memory (dynamic): Vr [(m + 1) Rp] (this CTA's rows of the basis,
// column j at Vr + j Rp), xr, br, wr, ex0, ex1 [Rp each], h1, h2, hs, g, hc
// [m + 2 each], cs, sn, ys [m + 1 each], psm [FUSED_PART_SLOTS], then (when
// h_smem) the rotated Hessenberg matrix Hs [(m + 1) m], then Ah, Al [R nc
// each] and vh, vl [nc each].  Every CTA keeps its own copy of the rotated
// Hessenberg matrix (in shared memory, or at a.H + blockIdx.x (m + 1) m,
// column-major); all copies are equal because every CTA applies the same
// rotations to the same numbers.
template <bool CL>
__global__ void __launch_bounds__(FT, 1) gm_fused_kernel(FusedArgs a) {
    extern __shared__ __align__(16) unsigned char fsm[];
    __shared__ double sc[4];
    __shared__ int flag_s[2];
    State *st = a.st;
    count_launch(st);
    const int n = a.n, R = a.R, nc = a.nc, m = a.m, Rp = (a.R + 1) & ~1;
    const int r0 = blockIdx.x * R, rows = min(R, n - r0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *Vr = reinterpret_cast<double *>(fsm);
    double *xr = Vr + (size_t)(m + 1) * Rp, *br = xr + Rp, *wr = br + Rp, *ex0 = wr + Rp, *ex1 = ex0 + Rp;
    double *h1 = ex1 + Rp, *h2 = h1 + (m + 2), *hs = h2 + (m + 2), *g = hs + (m + 2), *hc = g + (m + 2);
    double *cs = hc + (m + 2), *sn = cs + (m + 1), *ys = sn + (m + 1), *psm = ys + (m + 1);
    double *Hs = psm + FUSED_PART_SLOTS;
    double *H = a.h_smem ? Hs : a.H + (size_t)blockIdx.x * (m + 1) * m;
    float *Ah = align16(a.h_smem ? Hs + (size_t)(m + 1) * m : Hs);
    float *Al = Ah + (size_t)R * nc, *vh = Al + (size_t)R * nc, *vl = vh + nc;
    const int m1 = m + 1;
    FComm<CL> C = make_comm<CL>(a, psm, ex0, ex1);
    auto ex_x = [&](int j) { return C.get_elem(EX_X, j); };

    load_rows(a.A, a.lda, r0, rows, n, nc, Ah, Al);
    for (int i = threadIdx.x; i < rows; i += FT) {
        br[i] = a.b[r0 + i];
        xr[i] = a.x0_given ? a.x[r0 + i] : 0.0;
    }
    if (a.x0_given) load_vec([&](int j) { return a.x[j]; }, n, nc, false, 1.0, vh, vl, nullptr);
    else
        for (int j = threadIdx.x; j < nc; j += FT) vh[j] = vl[j] = 0.f;
    __syncthreads();

    double bn = 0.0, tol = 0.0, true_rn = 0.0, est = 0.0;
    int total = 0, cycles = 0, status = 0, nan = 0, k = 0;
    bool first = true;
    double rv[FUSED_VEC_REGS];
    for (;;) {   // cycles: each starts from the true residual
        // r = b - A x (x is in vh, vl), published: the last readers of the
        // previous contents (v_{k+1} of the previous cycle) have passed the
        // meeting that published x
        fused_product(Ah, Al, vh, vl, rows, nc, wr);
        __syncthreads();
        if (warp == 0) {
            double s = 0.0, bb = 0.0;
            for (int i = lane; i < rows; i += 32) {
                const double ri = br[i] - wr[i];
                wr[i] = ri;
                C.put_row(EX_V, i, ri);
                s += ri * ri;
                bb += br[i] * br[i];
            }
            s = warp_sum(s);
            bb = warp_sum(bb);
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
            if (lane == 0) {
                sc[0] = t;
                sc[1] = b2;
            }
        }
        __syncthreads();
        if (first) {
            const double b2 = sc[1];
            bn = sqrt(b2);
            tol = a.rtol * bn;
            if (!isfinite(b2)) {
                nan = 1;
                break;
            }
            if (bn == 0.0) {   // b = 0: x = 0 solves exactly
                for (int i = threadIdx.x; i < rows; i += FT) xr[i] = 0.0;
                status = LS_OK;
                true_rn = 0.0;
                break;
            }
            first = false;
        }
        const double beta = sqrt(sc[0]);
        true_rn = beta;
        if (nan || !isfinite(beta)) {
            nan = 1;
            break;
        }
        if (status == LS_BREAKDOWN) break;
        if (beta <= tol) {
            status = LS_OK;
            break;
        }
        if (total >= a.max_iter) {
            status = LS_NOT_CONVERGED;
            break;
        }
        // v_0 = r / beta: the whole vector (from the prefetched r) and this CTA's rows
        cycles++;
#pragma unroll
        for (int q = 0; q < FUSED_VEC_REGS; q++) {
            const int j = threadIdx.x + q * FT;
            if (j < nc) {
                const DSV d = ds_split(j < n ? rv[q] / beta : 0.0);
                vh[j] = d.h;
                vl[j] = d.l;
            }
        }
        for (int i = threadIdx.x; i < rows; i += FT) Vr[i] = wr[i] / beta;
        if (threadIdx.x == 0) g[0] = beta;
        est = beta;
        k = 0;
        __syncthreads();

        for (int j = 0;; j++) {   // Arnoldi steps; v_j is in vh, vl
            fused_product(Ah, Al, vh, vl, rows, nc, wr);
            __syncthreads();
            // first pass: V_j^T w and ||w||^2 over this CTA's rows (thread t: column t)
            for (int t = threadIdx.x; t <= j + 1; t += FT) {
                double s = 0.0;
                if (t <= j)
                    for (int i = 0; i < rows; i++) s += Vr[(size_t)t * Rp + i] * wr[i];
                else
                    for (int i = 0; i < rows; i++) s += wr[i] * wr[i];
                C.put(gs1(t), s);
            }
            if (!C.meet()) return;
            fsum_slots(C, gs1(0), j + 2, h1);
            __syncthreads();
            const double wnorm0 = h1[j + 1];
            // w -= V_j h, published (its readers of the last step have passed
            // the meeting above); the second-pass dots and ||w||^2 published
            // with it
            for (int i = threadIdx.x; i < rows; i += FT) {
                double wi = wr[i];
                for (int t = 0; t <= j; t++) wi -= h1[t] * Vr[(size_t)t * Rp + i];
                wr[i] = wi;
                C.put_row(EX_V, i, wi);
            }
            __syncthreads();
            for (int t = threadIdx.x; t <= j + 1; t += FT) {
                double s = 0.0;
                if (t <= j)
                    for (int i = 0; i < rows; i++) s += Vr[(size_t)t * Rp + i] * wr[i];
                else
                    for (int i = 0; i < rows; i++) s += wr[i] * wr[i];
                C.put(gs2(m, t), s);
            }
            if (!C.meet()) return;
            // w in flight while the sums are formed.  When the second pass
            // runs, a CTA that has taken its decision may overwrite its rows
            // while another still loads them; those loads are discarded and
            // the vector is loaded again after the next meeting.
            prefetch_vec(C, EX_V, n, rv);
            fsum_slots(C, gs2(m, 0), j + 2, h2);
            for (int t = threadIdx.x; t <= j; t += FT) hs[t] = h1[t];
            __syncthreads();
            double wn2 = h2[j + 1];
            // a second pass only when cancellation lost accuracy (or always if asked)
            if (a.reorth || wn2 < 0.49 * wnorm0) {
                if (warp == 0) {
                    double s = 0.0;
                    for (int i = lane; i < rows; i += 32) {
                        double wi = wr[i];
                        for (int t = 0; t <= j; t++) wi -= h2[t] * Vr[(size_t)t * Rp + i];
                        wr[i] = wi;
                        C.put_row(EX_V, i, wi);
                        s += wi * wi;
                    }
                    s = warp_sum(s);
                    if (lane == 0) C.put(gs3(m), s);
                }
                for (int t = threadIdx.x; t <= j; t += FT) hs[t] += h2[t];
                if (!C.meet()) return;
                prefetch_vec(C, EX_V, n, rv);
                if (warp == 0) {
                    const double v = fsum(C, gs3(m));
                    if (lane == 0) sc[2] = v;
                }
                __syncthreads();
                wn2 = sc[2];
            }
            const double wn = sqrt(wn2);
            const bool lucky = !(wn > 1e-14 * sqrt(wnorm0));
            if (!lucky) {   // v_{j+1} = w / ||w||, the whole vector, and this CTA's rows of it
#pragma unroll
                for (int q = 0; q < FUSED_VEC_REGS; q++) {
                    const int jj = threadIdx.x + q * FT;
                    if (jj < nc) {
                        const DSV d = ds_split(jj < n ? rv[q] / wn : 0.0);
                        vh[jj] = d.h;
                        vl[jj] = d.l;
                    }
                }
                for (int i = threadIdx.x; i < rows; i += FT) Vr[(size_t)(j + 1) * Rp + i] = wr[i] / wn;
            }
            // the new Hessenberg column, the old rotations, the new one (one
            // thread, in shared memory), then the column into this CTA's copy
            if (threadIdx.x == 0) {
                for (int t = 0; t <= j; t++) hc[t] = hs[t];
                hc[j + 1] = wn;
                for (int t = 0; t < j; t++) {
                    const double x0 = hc[t], x1 = hc[t + 1];
                    hc[t] = cs[t] * x0 + sn[t] * x1;
                    hc[t + 1] = -sn[t] * x0 + cs[t] * x1;
                }
                const double den = hypot(hc[j], hc[j + 1]);
                int stop = 0, brk = 0;
                if (den == 0.0 || !isfinite(den)) {
                    brk = isfinite(den) ? 1 : 2;
                    stop = 1;
                } else {
                    const double c = hc[j] / den, s = hc[j + 1] / den;
                    cs[j] = c;
                    sn[j] = s;
                    hc[j] = den;
                    hc[j + 1] = 0.0;
                    g[j + 1] = -s * g[j];
                    g[j] = c * g[j];
                    sc[3] = fabs(g[j + 1]);
                    if (sc[3] <= tol || lucky || j + 1 >= m || total + 1 >= a.max_iter) stop = 1;
                }
                double *Hk = H + (size_t)j * m1;
                for (int t = 0; t <= j + 1; t++) Hk[t] = hc[t];
                flag_s[0] = stop;
                flag_s[1] = brk;
            }
            __syncthreads();
            if (flag_s[1]) {
                status = LS_BREAKDOWN;
                if (flag_s[1] == 2) nan = 1;
                break;
            }
            k = j + 1;
            total++;
            est = sc[3];
            if (flag_s[0]) break;
        }
        // end of the cycle: R y = g (one warp, from this CTA's copy of R), x += V_k y
        if (status != LS_BREAKDOWN && k > 0) {
            if (warp == 0) {
                for (int i = k - 1; i >= 0; i--) {
                    double s = 0.0;
                    for (int t = i + 1 + lane; t < k; t += 32) s += H[(size_t)t * m1 + i] * ys[t];
                    s = warp_sum(s);
                    if (lane == 0) ys[i] = (g[i] - s) / H[(size_t)i * m1 + i];
                    __syncwarp();
                }
            }
            __syncthreads();
            for (int i = threadIdx.x; i < rows; i += FT) {
                double xi = xr[i];
                for (int t = 0; t < k; t++) xi += Vr[(size_t)t * Rp + i] * ys[t];
                xr[i] = xi;
            }
        }
        // x published, then the whole x into vh, vl
        for (int i = threadIdx.x; i < rows; i += FT) C.put_row(EX_X, i, xr[i]);
        if (!C.meet()) return;
        load_vec(ex_x, n, nc, false, 1.0, vh, vl, nullptr);
        __syncthreads();
    }
    for (int i = threadIdx.x; i < rows; i += FT) a.x[r0 + i] = xr[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->bnorm = bn;
        st->tol_abs = tol;
        st->true_rnorm = true_rn;
        st->est = est;
        st->rnorm = est;
        st->k = k;
        st->total = total;
        st->iter = total;
        st->cycles = cycles;
        st->status = status;
        if (nan) set_err(st, ERRB_NAN);
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
