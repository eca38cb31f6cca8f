// k_engine.cu -- kernels of the batched / served solve engine (ls_engine.h).
//
// Per slot (one dense system, s right-hand sides solved column by column):
//   refinement (FP64 accuracy): R = B - A X; stop when every
//     ||R_j|| <= rtol ||B_j||;
//   inner solve (FP32 on the FP32 copy of A) of A z = R_j / ||R_j||:
//     SPD systems: conjugate gradient (paper: CG paragraph), the columns sharing
//       one block product Q = Ahat P per step;
//     other systems: one GMRES(m) cycle (paper: GMRES pseudocode, Arnoldi with
//       classical Gram-Schmidt; Givens least squares), one block product
//       W = Ahat V_k per Arnoldi step;
//   correction: X += ||R_j|| z_j.
// All cross-row sums are reduced per slot in a fixed task order.
#include <cuda_runtime.h>

#include "ls_device.cuh"
#include "ls_engine.h"
#include "ls_internal.h"

namespace lsi {

constexpr int RED_T = 64;
constexpr int P32_T = 256;            // threads of eng_prod (both task kinds)
constexpr int VEC_T = 256;

__device__ __forceinline__ void eng_count(const EngineDev &E) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(E.launches, 1ull);
}

// Tasks are claimed one at a time from a per-tick counter, so CTAs that draw
// large tasks do not hold up the tick while others sit idle.
__device__ __forceinline__ int claim(int *counter, int *slot_s) {
    __syncthreads();
    if (threadIdx.x == 0) *slot_s = atomicAdd(counter, 1);
    __syncthreads();
    return *slot_s;
}

// ============================================================================
// eng_red: one block per slot; thread j < 32 owns column j
// ============================================================================
__global__ void __launch_bounds__(RED_T) eng_red_kernel(const EngineDev *Ep, cudaGraphConditionalHandle h) {
    const EngineDev &E = *Ep;
    __shared__ int all_stop, newphase_s;
    const int sl = blockIdx.x < E.nslots ? blockIdx.x : 0;
    const int j = threadIdx.x;
    eng_count(E);
    const SlotDesc &D = E.desc[sl];
    SlotState &S = E.st[sl];
    const int ph = blockIdx.x < E.nslots ? S.phase : PH_FREE;
    const bool colv = j < D.s;
    int newphase = ph;
    if (threadIdx.x == 0) all_stop = 1;
    __syncthreads();

    if (ph != PH_FREE && ph != PH_DONE && colv) {
        if (ph == PH_START) {
            double b2 = 0.0;
            for (int t = D.tv; t < D.tv + D.nv; t++) b2 += E.partv[(size_t)t * 32 + j];
            S.bnorm[j] = sqrt(b2);
            S.rn[j] = sqrt(b2);
            S.conv[j] = (b2 == 0.0);
            if (!isfinite(b2)) atomicOr(&S.err, ERRB_NAN);
            if (!S.conv[j]) atomicAnd(&all_stop, 0);
        } else if (ph == PH_RESID) {
            double r2 = 0.0;
            for (int t = D.t64; t < D.t64 + D.n64; t++) r2 += E.part64[(size_t)t * 32 + j];
            S.rn[j] = sqrt(r2);
            if (!isfinite(r2)) atomicOr(&S.err, ERRB_NAN);
            S.conv[j] = sqrt(r2) <= D.rtol * S.bnorm[j];
            if (!S.conv[j]) atomicAnd(&all_stop, 0);
        } else if (ph == PH_INIT) {
            double f2 = 0.0;
            for (int t = D.tv; t < D.tv + D.nv; t++) f2 += E.partv[(size_t)t * 32 + j];
            S.colstop[j] = S.conv[j] || !(f2 > 0.0);
            S.rho[j] = f2;
            S.rho0[j] = f2;
            S.beta[j] = 0.0;
            S.gbeta[j] = sqrt(f2);
            S.hnorm[j] = sqrt(f2);
            E.gm[sl].g[j][0] = sqrt(f2);
        } else if (ph == PH_CG) {
            if (!S.colstop[j]) {
                double pq = 0.0, rr = 0.0;
                for (int b = D.b32; b < D.b32 + D.nb32; b++)
                    pq += E.part32[((size_t)b * E_PS + 0) * 32 + j];
                for (int t = D.tv; t < D.tv + D.nv; t++) rr += E.partv[(size_t)t * 32 + j];
                if (!(pq > 0.0) || !isfinite(rr)) {
                    S.colstop[j] = 1;              // breakdown: keep the iterate
                } else if (rr <= (double)D.inner_tol * D.inner_tol * S.rho0[j]) {
                    S.colstop[j] = 1;
                } else {
                    S.beta[j] = rr / S.rho[j];
                    S.rho[j] = rr;
                }
            }
            if (!S.colstop[j]) atomicAnd(&all_stop, 0);
        } else if (ph == PH_GM) {
            const int k = S.it;                    // Arnoldi step just completed
            if (!S.colstop[j]) {
                SlotGm &G = E.gm[sl];
                double *Hk = G.H[j] + (size_t)k * (E_MAXM + 1);
                for (int i = 0; i <= k; i++) {
                    double hs = 0.0;
                    for (int b = D.b32; b < D.b32 + D.nb32; b++)
                        hs += E.part32[((size_t)b * E_PS + i) * 32 + j];
                    Hk[i] = hs;
                }
                double w2 = 0.0;
                for (int t = D.tv; t < D.tv + D.nv; t++) w2 += E.partv[(size_t)t * 32 + j];
                const double hk1 = sqrt(w2);
                Hk[k + 1] = hk1;
                for (int i = 0; i < k; i++) {      // earlier rotations
                    const double a = Hk[i], c = Hk[i + 1];
                    Hk[i] = G.cs[j][i] * a + G.sn[j][i] * c;
                    Hk[i + 1] = -G.sn[j][i] * a + G.cs[j][i] * c;
                }
                const double den = hypot(Hk[k], Hk[k + 1]);
                if (!(den > 0.0) || !isfinite(den)) {
                    S.colstop[j] = 1;              // breakdown: solve with the first k steps
                    S.hnorm[j] = 1.0;
                } else {
                    const double c = Hk[k] / den, s = Hk[k + 1] / den;
                    G.cs[j][k] = c;
                    G.sn[j][k] = s;
                    Hk[k] = den;
                    Hk[k + 1] = 0.0;
                    G.g[j][k + 1] = -s * G.g[j][k];
                    G.g[j][k] = c * G.g[j][k];
                    S.alpha[j] = k + 1;            // steps taken by this column
                    const double est = fabs(G.g[j][k + 1]);
                    if (est <= (double)D.inner_tol * S.gbeta[j] || !(hk1 > 1e-14 * den))
                        S.colstop[j] = 1;
                    S.hnorm[j] = hk1 > 0.0 ? hk1 : 1.0;
                }
            }
            if (!S.colstop[j]) atomicAnd(&all_stop, 0);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && ph != PH_FREE && ph != PH_DONE) {
        switch (ph) {
            case PH_ADMIT:
                newphase = PH_START;
                break;
            case PH_START:
                newphase = (all_stop || S.err) ? PH_DONE : PH_INIT;
                if (newphase == PH_DONE) S.status = S.err ? LS_ERR_NAN : LS_OK;
                break;
            case PH_RESID:
                S.outer += 1;
                if (S.err) { newphase = PH_DONE; S.status = LS_ERR_NAN; }
                else if (all_stop) { newphase = PH_DONE; S.status = LS_OK; }
                else if (S.outer >= D.max_outer) { newphase = PH_DONE; S.status = LS_NOT_CONVERGED; }
                else newphase = PH_INIT;
                break;
            case PH_INIT:
                S.it = 0;
                newphase = D.method == LS_METHOD_CG ? PH_CG : PH_GM;
                break;
            case PH_CG:
                S.it += 1;
                S.inner_total += 1;
                newphase = (all_stop || S.it >= D.inner_iters) ? PH_UPDATE : PH_CG;
                break;
            case PH_GM:
                S.it += 1;
                S.inner_total += 1;
                newphase = (all_stop || S.it >= D.m) ? PH_UPDATE : PH_GM;
                break;
            case PH_UPDATE:
                newphase = PH_RESID;
                break;
        }
        S.ticks += 1;
        if (S.ticks > 1000000 && newphase != PH_DONE) {   // never loop forever
            newphase = PH_DONE;
            S.status = LS_NOT_CONVERGED;
        }
        newphase_s = newphase;
    }
    __syncthreads();
    // GMRES cycle ends: back-solve R y = g per column (thread j)
    if (ph == PH_GM && threadIdx.x < 32) {
        if (newphase_s == PH_UPDATE && colv) {
            const SlotGm &G = E.gm[sl];
            const int kj = (int)S.alpha[j];       // steps with a valid rotation
            for (int i = kj - 1; i >= 0; i--) {
                double sacc = G.g[j][i];
                for (int q = i + 1; q < kj; q++) sacc -= G.H[j][(size_t)q * (E_MAXM + 1) + i] * S.yv[j][q];
                S.yv[j][i] = sacc / G.H[j][(size_t)i * (E_MAXM + 1) + i];
            }
            for (int i = kj; i < E_MAXM; i++) S.yv[j][i] = 0.0;
        }
    }
    if (ph == PH_INIT && threadIdx.x < 32 && colv) S.alpha[j] = 0.0;   // GMRES step counters
    if (threadIdx.x == 0) {
        int act = 0;
        if (ph != PH_FREE && ph != PH_DONE) {
            S.phase = newphase_s;
            act = (newphase_s != PH_DONE);
        }
        if (act) atomicAdd(&E.active[0], 1);
        __threadfence();
        const int tk = atomicAdd(&E.active[1], 1);
        if (tk == (int)gridDim.x - 1) {       // last block: loop control
            __threadfence();
            const int total = atomicAdd(&E.active[0], 0);
            const int ticks = E.active[3] + 1;
            E.active[3] = ticks;
            const int go = total > 0 && ticks < E.tick_limit;
            if (E.host_loop) E.active[4] = go;
            else cudaGraphSetConditional(h, go);
            E.active[0] = 0;
            E.active[1] = 0;
            E.active[2] = total;
            E.active[5] = 0;   // task claim counters of prod / vec
            E.active[7] = 0;
        }
    }
}

// ============================================================================
// eng_prod, FP32 block product task: Y = Ahat P for 256 rows and the task's
// K chunk of up to 512 columns of A, all sp columns, register-blocked: each
// thread owns an (sp/4)-row x 4-column tile of Y.  The A chunk (32 columns of
// the task's rows) sits transposed in shared memory; the next chunk is
// prefetched into registers meanwhile.  When a row block has several K
// chunks, each task stores its partial product and the last one to finish
// sums them in chunk order (so the result does not depend on which task came
// last) and runs the epilogue: Y rows and partial dots.
// ============================================================================
template <int SP>
__device__ __forceinline__ void prod32_task(const EngineDev &E, const Task &T, float *As, float *Ps,
                                            double *Red, float *colscale, int *colstop, int *flag_s) {
    constexpr int RB = E_RB32, KC = E_KC32;
    constexpr int RPT = SP / 4;                 // rows per thread
    constexpr int NCG = SP / 4;                 // column groups of 4
    constexpr int RBP = RB + 4;                 // padded row stride of the transposed tile
    constexpr int AV = RB * KC / 4 / P32_T;     // float4 loads of A per thread per chunk (8)
    constexpr int PV = (KC * SP + P32_T - 1) / P32_T;
    static_assert((RB / RPT) * NCG == P32_T, "thread grid");
    static_assert(E_KS32 % KC == 0 && E_KS32 % RB == 0, "K chunks hold whole row blocks");
    const SlotDesc &D = E.desc[T.slot];
    const SlotState &S = E.st[T.slot];
    const int ph = S.phase;
    const int n = D.n, s = D.s, it = S.it;
    const long long nsp = (long long)n * SP;
    const int r0 = T.r0, r1 = T.r1, nrow = r1 - r0;
    const int tid = threadIdx.x, rg = tid / NCG, cg = tid % NCG;
    const float *src, *src2 = nullptr;
    float *dst, *out;
    if (ph == PH_CG) {
        src = D.Rf;                                             // P = Rf + beta P'
        src2 = it > 0 ? D.P + ((it + 1) & 1) * nsp : nullptr;
        dst = D.P + (it & 1) * nsp;
        out = D.Q;
    } else {
        src = D.W + (it & 1) * nsp;                             // V_k = W / h
        dst = D.V + (long long)it * nsp;
        out = D.W + ((it + 1) & 1) * nsp;
    }
    if (tid < 32) {
        float sc = 0.0f;
        const int stp = tid < s ? S.colstop[tid] : 1;
        if (!stp) sc = ph == PH_CG ? (float)S.beta[tid] : (float)(1.0 / S.hnorm[tid]);
        colscale[tid] = sc;
        colstop[tid] = stp;
    }
    __syncthreads();
    const float *A = D.A32;
    const long long lda = D.ld32;
    float4 areg[AV];
    float preg[PV];
    // lane l of warp w loads rows 32*(w % 8) + l ... : all lanes of a warp hold
    // the same k-quad, so the transposed stores hit 32 different banks
    auto a_index = [&](int v, int &rr, int &q) {
        const int e = tid + v * P32_T;                          // 0 .. RB*KC/4 - 1
        rr = (e & 31) + 32 * ((e >> 5) % (RB / 32));
        q = (e >> 5) / (RB / 32);
    };
    auto prefetch = [&](int k0) {
#pragma unroll
        for (int v = 0; v < AV; v++) {
            int rr, q;
            a_index(v, rr, q);
            const int gr = r0 + rr, gk = k0 + 4 * q;
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gr < r1) {
                const float *ap = A + (long long)gr * lda + gk;
                if (gk + 3 < n) x = *reinterpret_cast<const float4 *>(ap);
                else {
                    if (gk < n) x.x = ap[0];
                    if (gk + 1 < n) x.y = ap[1];
                    if (gk + 2 < n) x.z = ap[2];
                }
            }
            areg[v] = x;
        }
#pragma unroll
        for (int v = 0; v < PV; v++) {
            const int e = tid + v * P32_T;
            float val = 0.0f;
            if (e < KC * SP) {
                const int kk = e / SP, c = e % SP, gk = k0 + kk;
                if (gk < n && c < s) {
                    const long long o = (long long)gk * SP + c;
                    if (ph == PH_CG)
                        val = colstop[c] ? 0.0f : (src2 ? fmaf(colscale[c], src2[o], src[o]) : src[o]);
                    else
                        val = src[o] * colscale[c];
                    if (gk >= r0 && gk < r1) dst[o] = val;      // this task owns row gk
                }
            }
            preg[v] = val;
        }
    };
    auto store = [&]() {
#pragma unroll
        for (int v = 0; v < AV; v++) {
            int rr, q;
            a_index(v, rr, q);
            As[(4 * q + 0) * RBP + rr] = areg[v].x;
            As[(4 * q + 1) * RBP + rr] = areg[v].y;
            As[(4 * q + 2) * RBP + rr] = areg[v].z;
            As[(4 * q + 3) * RBP + rr] = areg[v].w;
        }
#pragma unroll
        for (int v = 0; v < PV; v++) {
            const int e = tid + v * P32_T;
            if (e < KC * SP) Ps[e] = preg[v];
        }
    };
    float acc[RPT][4];
#pragma unroll
    for (int r = 0; r < RPT; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[r][c] = 0.0f;
    prefetch(T.k0);
    for (int k0 = T.k0; k0 < T.k1; k0 += KC) {
        store();
        __syncthreads();
        if (k0 + KC < T.k1) prefetch(k0 + KC);                  // overlaps with the math below
#pragma unroll 8
        for (int kk = 0; kk < KC; kk++) {
            float av[RPT];
            const float *ar = As + kk * RBP + rg * RPT;
            if constexpr (RPT == 1) {
                av[0] = ar[0];
            } else if constexpr (RPT == 2) {
                const float2 a2 = *reinterpret_cast<const float2 *>(ar);
                av[0] = a2.x;
                av[1] = a2.y;
            } else {
#pragma unroll
                for (int r4 = 0; r4 < RPT; r4 += 4) {
                    const float4 a4 = *reinterpret_cast<const float4 *>(ar + r4);
                    av[r4] = a4.x;
                    av[r4 + 1] = a4.y;
                    av[r4 + 2] = a4.z;
                    av[r4 + 3] = a4.w;
                }
            }
            const float4 pv = *reinterpret_cast<const float4 *>(Ps + kk * SP + cg * 4);
            const float pc[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
            for (int r = 0; r < RPT; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) acc[r][c] = fmaf(av[r], pc[c], acc[r][c]);
        }
        __syncthreads();
    }
    const int kc32 = (n + E_KS32 - 1) / E_KS32;
    if (kc32 > 1) {
        // publish this chunk's partial product; the last task of the row block
        // adds all chunks in chunk order
        float *yk = D.Yk + (long long)T.kc * nsp;
#pragma unroll
        for (int r = 0; r < RPT; r++) {
            const int row = rg * RPT + r;
            if (row < nrow)
                __stcg(reinterpret_cast<float4 *>(yk + (long long)(r0 + row) * SP + cg * 4),
                       make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]));
        }
        __threadfence();
        __syncthreads();
        const int rbl = r0 / E_RB32;
        if (tid == 0) *flag_s = atomicAdd(D.ticket + rbl, 1) == kc32 - 1;
        __syncthreads();
        if (!*flag_s) return;
        __threadfence();
        if (tid == 0) D.ticket[rbl] = 0;                        // ready for the next tick
#pragma unroll
        for (int r = 0; r < RPT; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[r][c] = 0.0f;
        for (int q = 0; q < kc32; q++) {
            const float *yq = D.Yk + (long long)q * nsp;
#pragma unroll
            for (int r = 0; r < RPT; r++) {
                const int row = rg * RPT + r;
                if (row < nrow) {
                    const float4 v = __ldcg(reinterpret_cast<const float4 *>(yq + (long long)(r0 + row) * SP + cg * 4));
                    acc[r][0] += v.x;
                    acc[r][1] += v.y;
                    acc[r][2] += v.z;
                    acc[r][3] += v.w;
                }
            }
        }
    }
    // Y rows of this row block
#pragma unroll
    for (int r = 0; r < RPT; r++) {
        const int row = rg * RPT + r;
        if (row < nrow)
            *reinterpret_cast<float4 *>(out + (long long)(r0 + row) * SP + cg * 4) =
                make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
    }
    // partial dots over this row block: CG p.q; GMRES v_i.w for i <= it
    // (the new direction's rows may come from another task: read through L2)
    const int nd = ph == PH_CG ? 1 : it + 1;
    constexpr int NRG = RB / RPT;               // row groups
    constexpr int NG = P32_T / SP;              // second-level groups per column
    for (int i = 0; i < nd; i++) {
        const float *vi = ph == PH_CG ? dst : D.V + (long long)i * nsp;
        double pc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int r = 0; r < RPT; r++) {
            const int row = rg * RPT + r;
            if (row < nrow) {
                const float4 v = __ldcg(reinterpret_cast<const float4 *>(vi + (long long)(r0 + row) * SP + cg * 4));
                pc[0] += (double)v.x * acc[r][0];
                pc[1] += (double)v.y * acc[r][1];
                pc[2] += (double)v.z * acc[r][2];
                pc[3] += (double)v.w * acc[r][3];
            }
        }
#pragma unroll
        for (int c = 0; c < 4; c++) Red[rg * SP + cg * 4 + c] = pc[c];
        __syncthreads();
        {   // thread (group g, column c) sums row groups g, g + NG, ... (fixed order)
            const int c = tid % SP, g = tid / SP;
            double sacc = 0.0;
            for (int q = g; q < NRG; q += NG) sacc += Red[q * SP + c];
            __syncthreads();
            Red[g * SP + c] = sacc;
        }
        __syncthreads();
        if (tid < 32) {
            double sacc = 0.0;
            if (tid < SP)
                for (int g = 0; g < NG; g++) sacc += Red[g * SP + tid];
            E.part32[((size_t)T.rb * E_PS + i) * 32 + tid] = sacc;
        }
        __syncthreads();
    }
}

// ============================================================================
// eng_prod, refinement residual task: R = B - A X for 8 rows, to about FP64
// accuracy on the FP32 pipe.  A = A32 + A32lo and X = Xh + Xl are fp32 pairs;
// each term a x = ah xh + ah xl + al xh (+ al xl, below 2^-48 |a x|, dropped)
// is accumulated in a (hi, lo) pair: ah xh = p + e exactly (product error by
// FMA), hi += p exactly with the rounding error moved to lo (two-sum, Knuth),
// lo also takes e and the cross terms.  Warp w owns row w, lane l the k = l
// (mod 32) part of it; the pairs are reduced across the warp in the same
// arithmetic and the total is formed in FP64.
// ============================================================================
struct DS {
    float h, l;
};

// (hi, lo) + (hi, lo): the high parts by two-sum, all errors into lo.
__device__ __forceinline__ DS ds_add(DS a, DS b) {
    const float s = __fadd_rn(a.h, b.h);
    const float bv = __fsub_rn(s, a.h);
    const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bv)), __fsub_rn(b.h, bv));
    return DS{s, __fadd_rn(e, __fadd_rn(a.l, b.l))};
}

__device__ __forceinline__ DS ds_shfl_xor(DS v, int o) {
    return DS{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
}

// Butterfly transpose-reduction over the warp: each round a lane keeps half of
// its columns and adds the partner's copy of them; afterwards lane l holds the
// warp total of column l >> (5 - log2 N0).
template <int N, int OFF, int N0>
__device__ __forceinline__ void ds_butterfly(DS (&acc)[N0], int lane) {
    if constexpr (OFF >= 1) {
        if constexpr (N > 1) {
            constexpr int H = N / 2;
            const bool upper = (lane & OFF) != 0;
#pragma unroll
            for (int i = 0; i < H; i++) {
                const DS send = upper ? acc[i] : acc[i + H];
                const DS keep = upper ? acc[i + H] : acc[i];
                acc[i] = ds_add(keep, ds_shfl_xor(send, OFF));
            }
            ds_butterfly<H, OFF / 2>(acc, lane);
        } else {
            acc[0] = ds_add(acc[0], ds_shfl_xor(acc[0], OFF));
            ds_butterfly<1, OFF / 2>(acc, lane);
        }
    }
}

template <int N>
__host__ __device__ constexpr int ilog2() { return N <= 1 ? 0 : 1 + ilog2<N / 2>(); }

template <int SP>
__device__ __forceinline__ void res_task(const EngineDev &E, const Task &T, int t, float *sm,
                                         double (*red)[33]) {
    constexpr int KC = 1024 / SP;               // k per chunk: 32 terms per thread per chunk
    constexpr int AP = KC + 1;                  // padded row stride of the A chunk
    constexpr int XS = SP + 1;                  // odd stride: conflict-free column reads
    constexpr int AV = E_RB64 * KC / P32_T;     // A floats (each of hi / lo) per thread per chunk
    constexpr int XV = KC * SP / P32_T;         // X floats (each of hi / lo) per thread per chunk
    static_assert(E_RB64 * 32 == P32_T, "a warp per row");
    float *Ah = sm, *Al = Ah + E_RB64 * AP, *Xh = Al + E_RB64 * AP, *Xl = Xh + KC * XS;
    const SlotDesc &D = E.desc[T.slot];
    const int n = D.n, s = D.s;
    const int r0 = T.r0, r1 = T.r1, nrow = r1 - r0;
    const int tid = threadIdx.x, row = tid >> 5, lane = tid & 31;
    const float *A = D.A32, *Alo = D.A32lo, *XH = D.Xh, *XL = D.Xl;
    const long long lda = D.ld32;
    float ahr[AV], alr[AV], xhr[XV], xlr[XV];
    auto prefetch = [&](int k0) {
#pragma unroll
        for (int v = 0; v < AV; v++) {
            const int e = tid + v * P32_T;
            const int rr = e / KC, kk = e % KC;
            const int gr = r0 + rr, gk = k0 + kk;
            const bool in = gr < r1 && gk < n;
            const long long o = (long long)gr * lda + gk;
            ahr[v] = in ? A[o] : 0.0f;
            alr[v] = in ? Alo[o] : 0.0f;
        }
#pragma unroll
        for (int v = 0; v < XV; v++) {
            const int e = tid + v * P32_T;             // the chunk is contiguous: rows k0.. of n x SP
            const bool in = k0 + e / SP < n;
            const long long o = (long long)k0 * SP + e;
            xhr[v] = in ? XH[o] : 0.0f;
            xlr[v] = in ? XL[o] : 0.0f;
        }
    };
    auto store = [&]() {
#pragma unroll
        for (int v = 0; v < AV; v++) {
            const int e = tid + v * P32_T;
            Ah[(e / KC) * AP + e % KC] = ahr[v];
            Al[(e / KC) * AP + e % KC] = alr[v];
        }
#pragma unroll
        for (int v = 0; v < XV; v++) {
            const int e = tid + v * P32_T;
            Xh[(e / SP) * XS + e % SP] = xhr[v];
            Xl[(e / SP) * XS + e % SP] = xlr[v];
        }
    };
    DS acc[SP];
#pragma unroll
    for (int c = 0; c < SP; c++) acc[c] = DS{0.0f, 0.0f};
    prefetch(0);
    for (int k0 = 0; k0 < n; k0 += KC) {
        store();
        __syncthreads();
        if (k0 + KC < n) prefetch(k0 + KC);
        if (row < nrow) {
#pragma unroll
            for (int i = 0; i < KC / 32; i++) {
                const int kk = lane + 32 * i;
                const float ah = Ah[row * AP + kk], al = Al[row * AP + kk];
                const float *xh = Xh + kk * XS, *xl = Xl + kk * XS;
#pragma unroll
                for (int c = 0; c < SP; c++) {
                    if (c < s) {
                        const float xhc = xh[c];
                        const float p = __fmul_rn(ah, xhc);
                        const float pe = fmaf(ah, xhc, -p);             // ah xh - p, exact
                        const float tc = fmaf(al, xhc, fmaf(ah, xl[c], pe));
                        const float sh = __fadd_rn(acc[c].h, p);
                        const float bv = __fsub_rn(sh, acc[c].h);
                        const float er = __fadd_rn(__fsub_rn(acc[c].h, __fsub_rn(sh, bv)), __fsub_rn(p, bv));
                        acc[c].h = sh;
                        acc[c].l = __fadd_rn(acc[c].l, __fadd_rn(tc, er));
                    }
                }
            }
        }
        __syncthreads();
    }
    ds_butterfly<SP, 16>(acc, lane);
    constexpr int LG = ilog2<SP>();
    if ((lane & ((32 >> LG) - 1)) == 0) {
        const int c = lane >> (5 - LG);
        double v = 0.0;
        if (row < nrow) {
            const long long o = (long long)(r0 + row) * SP + c;
            const double rv = c < s ? D.B[o] - ((double)acc[0].h + (double)acc[0].l) : 0.0;
            D.R[o] = rv;
            v = rv * rv;
        }
        red[row][c] = v;
    }
    __syncthreads();
    if (tid < 32) {
        double sacc = 0.0;
        if (tid < SP)
            for (int rr = 0; rr < nrow; rr++) sacc += red[rr][tid];
        E.part64[(size_t)t * 32 + tid] = sacc;
    }
    __syncthreads();
}

// One queue per tick: the refinement-residual tasks first, then the FP32
// product tasks; tasks of slots in other phases are skipped.
__global__ void __launch_bounds__(P32_T, 2) eng_prod_kernel(const EngineDev *Ep) {
    const EngineDev &E = *Ep;
    extern __shared__ __align__(16) unsigned char esm[];
    float *As = reinterpret_cast<float *>(esm);                         // [KC][RB + 4]
    float *Ps = As + E_KC32 * (E_RB32 + 4);                             // [KC][SP]
    double *Red = reinterpret_cast<double *>(Ps + E_KC32 * 32);         // [row groups][SP]
    __shared__ double red64[E_RB64][33];
    __shared__ float colscale[32];
    __shared__ int colstop[32];
    __shared__ int claim_s, flag_s;
    eng_count(E);
    const int total = E.n64 + E.n32;
    for (int u = claim(E.active + 5, &claim_s); u < total; u = claim(E.active + 5, &claim_s)) {
        if (u < E.n64) {
            const Task T = E.t64[u];
            if (T.slot < 0) continue;                                   // unused entry
            if (E.st[T.slot].phase != PH_RESID) continue;
            float *sm = reinterpret_cast<float *>(esm);
            switch (E.desc[T.slot].sp) {
                case 4: res_task<4>(E, T, u, sm, red64); break;
                case 8: res_task<8>(E, T, u, sm, red64); break;
                case 16: res_task<16>(E, T, u, sm, red64); break;
                default: res_task<32>(E, T, u, sm, red64); break;
            }
        } else {
            const Task T = E.t32[u - E.n64];
            if (T.slot < 0) continue;
            const int ph = E.st[T.slot].phase;
            if (ph != PH_CG && ph != PH_GM) continue;
            switch (E.desc[T.slot].sp) {
                case 4: prod32_task<4>(E, T, As, Ps, Red, colscale, colstop, &flag_s); break;
                case 8: prod32_task<8>(E, T, As, Ps, Red, colscale, colstop, &flag_s); break;
                case 16: prod32_task<16>(E, T, As, Ps, Red, colscale, colstop, &flag_s); break;
                default: prod32_task<32>(E, T, As, Ps, Red, colscale, colstop, &flag_s); break;
            }
        }
        __syncthreads();
    }
}

// ============================================================================
// eng_vec: vector updates of one 256-row task.  The task's n x sp block is
// walked as a flat array: thread t always sees column t % sp (sp divides the
// block size), so loads are coalesced and each thread's partial sum belongs
// to one column.
// ============================================================================
__global__ void __launch_bounds__(VEC_T) eng_vec_kernel(const EngineDev *Ep) {
    const EngineDev &E = *Ep;
    __shared__ double psum[VEC_T];
    __shared__ double hsm[E_MAXM + 1][32];
    __shared__ double colv_s[32];
    __shared__ int claim_s;
    eng_count(E);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int t = claim(E.active + 7, &claim_s); t < E.nv; t = claim(E.active + 7, &claim_s)) {
        const Task T = E.tv[t];
        if (T.slot < 0) continue;                                       // unused entry
        const SlotDesc &D = E.desc[T.slot];
        const SlotState &S = E.st[T.slot];
        const int ph = S.phase;
        if (ph != PH_START && ph != PH_INIT && ph != PH_CG && ph != PH_GM && ph != PH_UPDATE) continue;
        const int n = D.n, s = D.s, sp = D.sp, it = S.it;
        const long long nsp = (long long)n * sp;
        // per-column scalars needed by this phase
        if (tid < 32) {
            double cv = 0.0;
            if (tid < s) {
                if (ph == PH_CG) {
                    double pq = 0.0;
                    for (int u = D.b32; u < D.b32 + D.nb32; u++)
                        pq += E.part32[((size_t)u * E_PS + 0) * 32 + tid];
                    cv = (S.colstop[tid] || !(pq > 0.0)) ? 0.0 : S.rho[tid] / pq;
                } else if (ph == PH_INIT || ph == PH_UPDATE) {
                    cv = (ph == PH_UPDATE && S.conv[tid]) ? 0.0 : S.rn[tid];
                }
            }
            colv_s[tid] = cv;
        }
        if (ph == PH_GM) {
            for (int e = tid; e < (it + 1) * 32; e += VEC_T) {
                const int ii = e / 32, c = e % 32;
                double hs = 0.0;
                if (c < s && !S.colstop[c])
                    for (int u = D.b32; u < D.b32 + D.nb32; u++)
                        hs += E.part32[((size_t)u * E_PS + ii) * 32 + c];
                hsm[ii][c] = hs;
            }
        }
        if (ph == PH_START) {   // A = A32 + A32lo for this task's rows, a warp per row
            for (int r = T.r0 + warp; r < T.r1; r += VEC_T / 32) {
                const double *a = D.A64 + (long long)r * D.lda64;
                float *a32 = D.A32 + (long long)r * D.ld32;
                float *alo = D.A32lo + (long long)r * D.ld32;
                for (int k = lane; k < n; k += 32) {
                    const double v = a[k];
                    const float hi = __double2float_rn(v);
                    a32[k] = hi;
                    alo[k] = __double2float_rn(v - (double)hi);
                }
            }
            if (T.r0 == 0)      // split-K tickets of the FP32 product start at zero
                for (int b = tid; b < D.nb32; b += VEC_T) D.ticket[b] = 0;
        }
        __syncthreads();
        const long long e0 = (long long)T.r0 * sp, e1 = (long long)T.r1 * sp;
        const int c = tid % sp;                                        // fixed for this thread
        const bool live = c < s;
        double part = 0.0;
        if (ph == PH_START) {
            for (long long e = e0 + tid; e < e1; e += VEC_T) {
                const double b = D.B[e];
                D.X[e] = 0.0;
                D.Xh[e] = 0.0f;
                D.Xl[e] = 0.0f;
                D.R[e] = b;
                part += b * b;
            }
        } else if (ph == PH_INIT) {
            const bool on = live && !S.conv[c];
            const double rn = colv_s[c];
            for (long long e = e0 + tid; e < e1; e += VEC_T) {
                const float f = on ? (float)(D.R[e] / rn) : 0.0f;
                D.Rf[e] = f;
                D.Z[e] = 0.0f;
                if (D.method != LS_METHOD_CG) D.W[e] = f;               // W buffer 0
                part += (double)f * (double)f;
            }
        } else if (ph == PH_CG) {
            const float al = (float)colv_s[c];
            const float *p = D.P + (it & 1) * nsp;
            for (long long e = e0 + tid; e < e1; e += VEC_T) {
                D.Z[e] = fmaf(al, p[e], D.Z[e]);
                const float rv = fmaf(-al, D.Q[e], D.Rf[e]);
                D.Rf[e] = rv;
                part += (double)rv * (double)rv;
            }
        } else if (ph == PH_GM) {
            float *w = D.W + ((it + 1) & 1) * nsp;
            for (long long e = e0 + tid; e < e1; e += VEC_T) {
                double wv = w[e];
                for (int q = 0; q <= it; q++) wv -= hsm[q][c] * (double)D.V[(long long)q * nsp + e];
                const float wf = (float)wv;
                w[e] = wf;
                part += (double)wf * (double)wf;
            }
        } else if (ph == PH_UPDATE) {
            const double rn = colv_s[c];
            if (live && rn != 0.0) {
                const int kj = D.method == LS_METHOD_CG ? 0 : (int)S.alpha[c];
                for (long long e = e0 + tid; e < e1; e += VEC_T) {
                    double d;
                    if (D.method == LS_METHOD_CG) {
                        d = (double)D.Z[e];
                    } else {
                        d = 0.0;
                        for (int q = 0; q < kj; q++) d += S.yv[c][q] * (double)D.V[(long long)q * nsp + e];
                    }
                    const double xn = D.X[e] + rn * d;
                    const float xh = __double2float_rn(xn);
                    D.X[e] = xn;
                    D.Xh[e] = xh;
                    D.Xl[e] = __double2float_rn(xn - (double)xh);
                }
            }
        }
        // partial column sums over this task's rows (fixed order)
        if (ph != PH_UPDATE) {
            psum[tid] = part;
            __syncthreads();
            if (tid < 32) {
                double sacc = 0.0;
                if (tid < sp)
                    for (int q = tid; q < VEC_T; q += sp) sacc += psum[q];
                E.partv[(size_t)t * 32 + tid] = sacc;
            }
        }
        __syncthreads();
    }
}

// ============================================================================
// admission / completion helpers
// ============================================================================
// B (column-major, ldb) -> the slot's row-major n x sp block (zero padding).
__global__ void eng_admit_kernel(const EngineDev *Ep, const double *const *Bsrc, const long long *ldb,
                                 int first, int count) {
    const EngineDev &E = *Ep;
    for (int q = blockIdx.y; q < count; q += gridDim.y) {
        const int sl = first + q;
        const SlotDesc &D = E.desc[sl];
        const double *b = Bsrc[q];
        const long long total = (long long)D.n * D.sp;
        for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
             e += (long long)gridDim.x * blockDim.x) {
            const int i = (int)(e / D.sp), c = (int)(e % D.sp);
            D.B[e] = c < D.s ? b[(long long)c * ldb[q] + i] : 0.0;
        }
    }
}

// X (row-major) -> column-major destination (ldx).
__global__ void eng_finish_kernel(const EngineDev *Ep, double *const *Xdst, const long long *ldx, int first,
                                  int count) {
    const EngineDev &E = *Ep;
    for (int q = blockIdx.y; q < count; q += gridDim.y) {
        const int sl = first + q;
        const SlotDesc &D = E.desc[sl];
        double *x = Xdst[q];
        const long long total = (long long)D.n * D.s;
        for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
             e += (long long)gridDim.x * blockDim.x) {
            const int c = (int)(e / D.n), i = (int)(e % D.n);
            x[(long long)c * ldx[q] + i] = D.X[(long long)i * D.sp + c];
        }
    }
}

EngineKernels engine_kernels() {
    EngineKernels K{};
    K.red = reinterpret_cast<void *>(&eng_red_kernel);
    K.prod = reinterpret_cast<void *>(&eng_prod_kernel);
    K.vec = reinterpret_cast<void *>(&eng_vec_kernel);
    K.admit = reinterpret_cast<void *>(&eng_admit_kernel);
    K.finish = reinterpret_cast<void *>(&eng_finish_kernel);
    K.red_threads = RED_T;
    K.prod_threads = P32_T;
    K.vec_threads = VEC_T;
    // FP32 product: transposed A chunk (+ padding), operand chunk, reduction
    // scratch (P32_T x 4 doubles); the residual tasks reuse the same bytes
    K.prod_smem = (size_t)E_KC32 * (E_RB32 + 4) * 4 + E_KC32 * 32 * 4 + (size_t)E_RB32 * 32 / 4 * 8;
    return K;
}

}  // namespace lsi
