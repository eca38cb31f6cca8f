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
// grid-wide barriers over every SM.  Here one cooperative launch of G CTAs
// runs the whole solve:
//  * CTA c owns rows [c R, c R + R) of A; it splits them into the FP32 pair
//    once, at the start, and keeps them in shared memory for the whole solve,
//    so A is read from HBM once per solve, not once per step;
//  * every CTA holds the full vector that multiplies A (the CG direction p,
//    the Arnoldi vector v_j, or x for a residual) as its (hi, lo) split in
//    shared memory, and its own rows of the other vectors (x, r, b, the rows
//    of the Krylov basis V);
//  * a product is warp per row, lanes along the row, double-single
//    accumulation and a butterfly reduction;
//  * the vector a step produces row by row (r, w) is exchanged through a
//    global buffer: each CTA writes its rows, meets the others at a grid
//    barrier, and reads the whole vector back from L2;
//  * a scalar reduction: each CTA publishes its partial sum into a slot,
//    meets the others at a barrier, and every CTA adds the G partials of the
//    slot in the same fixed order, so all CTAs hold the same bits and take
//    the same decisions without further communication;
//  * the grid barrier counts arrivals on three counters in turn (see
//    fbar_sync) with a bounded wait.
// A CG step takes two barriers (p.Ap; r.r together with the exchange of r);
// an Arnoldi step two (V^T w with ||w||^2; ||w - V h||^2 with the exchange of
// w and the speculative second-pass dots), three when the second
// Gram-Schmidt pass runs.
//
// Partial-sum slots and exchange buffers are reused step after step.  Each
// is written before a barrier and read after it; its next write comes after
// a later barrier, which no CTA reaches before it has finished reading, so
// no double buffering is needed (the argument for each buffer is at its use).
#include <cuda_runtime.h>

#include "ls_device.cuh"
#include "ls_ds.cuh"
#include "ls_internal.h"
#include "split_pair.h"

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
}  // namespace

// ---- grid barrier ------------------------------------------------------------------
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

// Sum of slot `slot` over the G CTAs' partials (layout [slot][G]), by the
// calling warp.  Every CTA adds the same values in the same order, and the
// butterfly leaves the same bits in every lane.
__device__ __forceinline__ double fsum(const double *part, int slot, int G) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < G; b += 32) s += __ldcg(&part[(size_t)slot * G + b]);
    return warp_sum(s);
}
__device__ __forceinline__ void fput(double *part, int slot, double v) {
    part[(size_t)slot * gridDim.x + blockIdx.x] = v;
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

// (vh, vl) = split of the full vector: src[j] / scale (or src[j] when
// scale_it is false), read from L2 (src was written by other CTAs or by the
// host); zero padding up to nc.  Optionally keeps the FP64 values in keep[].
__device__ __forceinline__ void load_vec(const double *src, int n, int nc, bool scale_it, double scale,
                                         float *vh, float *vl, double *keep) {
    for (int j = threadIdx.x; j < nc; j += FT) {
        double v = 0.0;
        if (j < n) {
            v = __ldcg(&src[j]);
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

// ============================================================================
// CG (paper, CG paragraph; Hestenes-Stiefel form)
// ============================================================================
// Shared memory (dynamic): p[nc] (FP64 direction), xr, rr, br, qr [Rp each]
// (this CTA's rows of x, r, b and of the product), then the FP32 pair of the
// rows Ah, Al [R nc each] and the split vector vh, vl [nc each].
__global__ void __launch_bounds__(FT, 1) cg_fused_kernel(FusedArgs a) {
    extern __shared__ __align__(16) unsigned char fsm[];
    __shared__ double sc[4];
    State *st = a.st;
    count_launch(st);
    const int n = a.n, R = a.R, nc = a.nc, G = gridDim.x, Rp = (a.R + 1) & ~1;
    const int r0 = blockIdx.x * R, rows = min(R, n - r0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *p = reinterpret_cast<double *>(fsm);
    double *xr = p + nc, *rr = xr + Rp, *br = rr + Rp, *qr = br + Rp;
    float *Ah = align16(qr + Rp), *Al = Ah + (size_t)R * nc, *vh = Al + (size_t)R * nc,
          *vl = vh + nc;
    unsigned e = 0;   // barriers passed

    load_rows(a.A, a.lda, r0, rows, n, nc, Ah, Al);
    for (int i = threadIdx.x; i < rows; i += FT) {
        br[i] = a.b[r0 + i];
        xr[i] = a.x0_given ? a.x[r0 + i] : 0.0;
    }
    if (a.x0_given) load_vec(a.x, n, nc, false, 1.0, vh, vl, nullptr);
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
            a.xch[r0 + i] = ri;
            bb += br[i] * br[i];
            r2 += ri * ri;
        }
        bb = warp_sum(bb);
        r2 = warp_sum(r2);
        if (lane == 0) {
            fput(a.part, CS_BB, bb);
            fput(a.part, CS_R0, r2);
        }
    }
    if (!fbar_sync(a.bar, e, st)) return;
    if (warp == 0) {
        const double b2 = fsum(a.part, CS_BB, G), r2 = fsum(a.part, CS_R0, G);
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
    // p = r: the exchange buffer holds r (x0 given) and b equals r otherwise
    if (go) load_vec(a.x0_given ? a.xch : a.b, n, nc, false, 1.0, vh, vl, p);
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
                if (lane == 0) fput(a.part, CS_PQ, s);
            }
            // CS_PQ: its readers finish before they arrive at the next r.r barrier
            if (!fbar_sync(a.bar, e, st)) return;
            if (warp == 0) {
                const double t = fsum(a.part, CS_PQ, G);
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
            // x += alpha p, r -= alpha q on this CTA's rows; r to the exchange
            // buffer (every reader of its previous contents has passed the
            // p.q barrier just met)
            if (warp == 0) {
                double s = 0.0;
                for (int i = lane; i < rows; i += 32) {
                    xr[i] += alpha * p[r0 + i];
                    const double ri = rr[i] - alpha * qr[i];
                    rr[i] = ri;
                    a.xch[r0 + i] = ri;
                    s += ri * ri;
                }
                s = warp_sum(s);
                if (lane == 0) fput(a.part, CS_RR, s);
            }
            if (!fbar_sync(a.bar, e, st)) return;
            if (warp == 0) {
                const double t = fsum(a.part, CS_RR, G);
                if (lane == 0) sc[1] = t;
            }
            __syncthreads();
            const double rho_new = sc[1];
            const bool finite = isfinite(rho_new);
            conv = finite && sqrt(rho_new) <= tol;
            beta = rho_new / rho;
            if (finite && !conv) {   // p = r + beta p, the whole vector in every CTA
                for (int j = threadIdx.x; j < n; j += FT) {
                    const double pj = __ldcg(&a.xch[j]) + beta * p[j];
                    p[j] = pj;
                    const DSV d = ds_split(pj);
                    vh[j] = d.h;
                    vl[j] = d.l;
                }
            }
            rho = rho_new;
            rnorm = sqrt(rho_new);
            iter++;
            if (!finite) nan = 1;
            __syncthreads();
            if (!finite || conv || iter >= a.max_iter) break;
        }
        // the true residual b - A x: x to the second exchange buffer
        for (int i = threadIdx.x; i < rows; i += FT) a.xch2[r0 + i] = xr[i];
        if (!fbar_sync(a.bar, e, st)) return;
        load_vec(a.xch2, n, nc, false, 1.0, vh, vl, nullptr);
        __syncthreads();
        fused_product(Ah, Al, vh, vl, rows, nc, qr);
        __syncthreads();
        // t = b - A x to the exchange buffer: its last readers (the p update)
        // have passed the barrier above
        if (warp == 0) {
            double s = 0.0;
            for (int i = lane; i < rows; i += 32) {
                const double ti = br[i] - qr[i];
                qr[i] = ti;
                a.xch[r0 + i] = ti;
                s += ti * ti;
            }
            s = warp_sum(s);
            if (lane == 0) fput(a.part, CS_TT, s);
        }
        if (!fbar_sync(a.bar, e, st)) return;
        if (warp == 0) {
            const double t = fsum(a.part, CS_TT, G);
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
        load_vec(a.xch, n, nc, false, 1.0, vh, vl, p);
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
}

// ============================================================================
// GMRES(m) (paper, GMRES pseudocode and restart paragraph; least squares by
// Givens rotations)
// ============================================================================
// Shared memory (dynamic): Vr [(m + 1) Rp] (this CTA's rows of the basis,
// column j at Vr + j Rp), xr, br, wr [Rp each], h1, h2, hs, g [m + 2 each],
// cs, sn, ys [m + 1 each], then Ah, Al [R nc each] and vh, vl [nc each].
// Each CTA keeps its own copy of the rotated Hessenberg matrix in global
// memory (a.H + blockIdx.x (m + 1) m, column-major), written and read by
// this CTA only; all copies are equal because every CTA applies the same
// rotations to the same numbers.
__global__ void __launch_bounds__(FT, 1) gm_fused_kernel(FusedArgs a) {
    extern __shared__ __align__(16) unsigned char fsm[];
    __shared__ double sc[4];
    __shared__ int flag_s[2];
    State *st = a.st;
    count_launch(st);
    const int n = a.n, R = a.R, nc = a.nc, G = gridDim.x, m = a.m, Rp = (a.R + 1) & ~1;
    const int r0 = blockIdx.x * R, rows = min(R, n - r0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *Vr = reinterpret_cast<double *>(fsm);
    double *xr = Vr + (size_t)(m + 1) * Rp, *br = xr + Rp, *wr = br + Rp;
    double *h1 = wr + Rp, *h2 = h1 + (m + 2), *hs = h2 + (m + 2), *g = hs + (m + 2);
    double *cs = g + (m + 2), *sn = cs + (m + 1), *ys = sn + (m + 1);
    float *Ah = align16(ys + (m + 1));
    float *Al = Ah + (size_t)R * nc, *vh = Al + (size_t)R * nc, *vl = vh + nc;
    double *H = a.H + (size_t)blockIdx.x * (m + 1) * m;
    const int m1 = m + 1;
    unsigned e = 0;   // barriers passed

    load_rows(a.A, a.lda, r0, rows, n, nc, Ah, Al);
    for (int i = threadIdx.x; i < rows; i += FT) {
        br[i] = a.b[r0 + i];
        xr[i] = a.x0_given ? a.x[r0 + i] : 0.0;
    }
    if (a.x0_given) load_vec(a.x, n, nc, false, 1.0, vh, vl, nullptr);
    else
        for (int j = threadIdx.x; j < nc; j += FT) vh[j] = vl[j] = 0.f;
    __syncthreads();

    double bn = 0.0, tol = 0.0, true_rn = 0.0, est = 0.0;
    int total = 0, cycles = 0, status = 0, nan = 0, k = 0;
    bool first = true;
    for (;;) {   // cycles: each starts from the true residual
        // r = b - A x (x is in vh, vl) to the exchange buffer, whose last
        // readers (v_{k+1} of the previous cycle) have passed the x barrier
        fused_product(Ah, Al, vh, vl, rows, nc, wr);
        __syncthreads();
        if (warp == 0) {
            double s = 0.0, bb = 0.0;
            for (int i = lane; i < rows; i += 32) {
                const double ri = br[i] - wr[i];
                wr[i] = ri;
                a.xch[r0 + i] = ri;
                s += ri * ri;
                bb += br[i] * br[i];
            }
            s = warp_sum(s);
            bb = warp_sum(bb);
            if (lane == 0) {
                fput(a.part, gsr(m), s);
                if (first) fput(a.part, gsb(m), bb);
            }
        }
        if (!fbar_sync(a.bar, e, st)) return;
        if (warp == 0) {
            const double t = fsum(a.part, gsr(m), G);
            const double b2 = first ? fsum(a.part, gsb(m), G) : 0.0;
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
        // v_0 = r / beta
        cycles++;
        load_vec(a.xch, n, nc, true, beta, vh, vl, nullptr);
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
                fput(a.part, gs1(t), s);
            }
            if (!fbar_sync(a.bar, e, st)) return;
            for (int t = warp; t <= j + 1; t += FW) {
                const double v = fsum(a.part, gs1(t), G);
                if (lane == 0) h1[t] = v;
            }
            __syncthreads();
            const double wnorm0 = h1[j + 1];
            // w -= V_j h; w to the exchange buffer (its readers of the last
            // step have passed the barrier above); the second-pass dots and
            // ||w||^2 published with it
            for (int i = threadIdx.x; i < rows; i += FT) {
                double wi = wr[i];
                for (int t = 0; t <= j; t++) wi -= h1[t] * Vr[(size_t)t * Rp + i];
                wr[i] = wi;
                a.xch[r0 + i] = wi;
            }
            __syncthreads();
            for (int t = threadIdx.x; t <= j + 1; t += FT) {
                double s = 0.0;
                if (t <= j)
                    for (int i = 0; i < rows; i++) s += Vr[(size_t)t * Rp + i] * wr[i];
                else
                    for (int i = 0; i < rows; i++) s += wr[i] * wr[i];
                fput(a.part, gs2(m, t), s);
            }
            if (!fbar_sync(a.bar, e, st)) return;
            if (warp == 0) {
                const double v = fsum(a.part, gs2(m, j + 1), G);
                if (lane == 0) sc[2] = v;
            }
            for (int t = threadIdx.x; t <= j; t += FT) hs[t] = h1[t];
            __syncthreads();
            double wn2 = sc[2];
            // a second pass only when cancellation lost accuracy (or always if asked)
            if (a.reorth || wn2 < 0.49 * wnorm0) {
                for (int t = warp; t <= j; t += FW) {
                    const double v = fsum(a.part, gs2(m, t), G);
                    if (lane == 0) h2[t] = v;
                }
                __syncthreads();
                // nobody reads the exchange buffer between the last barrier and the next
                if (warp == 0) {
                    double s = 0.0;
                    for (int i = lane; i < rows; i += 32) {
                        double wi = wr[i];
                        for (int t = 0; t <= j; t++) wi -= h2[t] * Vr[(size_t)t * Rp + i];
                        wr[i] = wi;
                        a.xch[r0 + i] = wi;
                        s += wi * wi;
                    }
                    s = warp_sum(s);
                    if (lane == 0) fput(a.part, gs3(m), s);
                }
                for (int t = threadIdx.x; t <= j; t += FT) hs[t] += h2[t];
                if (!fbar_sync(a.bar, e, st)) return;
                if (warp == 0) {
                    const double v = fsum(a.part, gs3(m), G);
                    if (lane == 0) sc[2] = v;
                }
                __syncthreads();
                wn2 = sc[2];
            }
            const double wn = sqrt(wn2);
            const bool lucky = !(wn > 1e-14 * sqrt(wnorm0));
            if (!lucky) {   // v_{j+1} = w / ||w||, the whole vector, and this CTA's rows of it
                load_vec(a.xch, n, nc, true, wn, vh, vl, nullptr);
                for (int i = threadIdx.x; i < rows; i += FT) Vr[(size_t)(j + 1) * Rp + i] = wr[i] / wn;
            }
            // the new Hessenberg column, the old rotations, the new one (one thread)
            if (threadIdx.x == 0) {
                double *Hk = H + (size_t)j * m1;
                for (int t = 0; t <= j; t++) Hk[t] = hs[t];
                Hk[j + 1] = wn;
                for (int t = 0; t < j; t++) {
                    const double x0 = Hk[t], x1 = Hk[t + 1];
                    Hk[t] = cs[t] * x0 + sn[t] * x1;
                    Hk[t + 1] = -sn[t] * x0 + cs[t] * x1;
                }
                const double den = hypot(Hk[j], Hk[j + 1]);
                int stop = 0, brk = 0;
                if (den == 0.0 || !isfinite(den)) {
                    brk = isfinite(den) ? 1 : 2;
                    stop = 1;
                } else {
                    const double c = Hk[j] / den, s = Hk[j + 1] / den;
                    cs[j] = c;
                    sn[j] = s;
                    Hk[j] = den;
                    Hk[j + 1] = 0.0;
                    g[j + 1] = -s * g[j];
                    g[j] = c * g[j];
                    sc[3] = fabs(g[j + 1]);
                    if (sc[3] <= tol || lucky || j + 1 >= m || total + 1 >= a.max_iter) stop = 1;
                }
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
        // x to the second exchange buffer, then the whole x into vh, vl
        for (int i = threadIdx.x; i < rows; i += FT) a.xch2[r0 + i] = xr[i];
        if (!fbar_sync(a.bar, e, st)) return;
        load_vec(a.xch2, n, nc, false, 1.0, vh, vl, nullptr);
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
}

FusedKernels fused_kernels() {
    FusedKernels K{};
    K.cg = reinterpret_cast<void *>(&cg_fused_kernel);
    K.gmres = reinterpret_cast<void *>(&gm_fused_kernel);
    return K;
}

}  // namespace lsi
