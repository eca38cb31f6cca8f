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
#include "ls_ds.cuh"
#include "ls_engine.h"
#include "ls_internal.h"
#include "ls_tc.cuh"
#include "split_pair.h"

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
    __shared__ int all_stop, newphase_s, cnt_s, first_s, base_s, cntv_s, basev_s, res_s;
    const int sl = blockIdx.x < E.nslots ? E.order[blockIdx.x] : 0;
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
            for (int b = D.b32; b < D.b32 + D.nb32; b++) r2 += E.part64[(size_t)b * 32 + j];
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
    // this tick's runnable tasks of the slot go to the work lists of the
    // tick's parity (eng_prod and eng_vec claim from those lists only)
    const int par = E.active[A_TICKS] & 1;
    if (threadIdx.x == 0) {
        const int np = (ph != PH_FREE && ph != PH_DONE) ? newphase_s : PH_FREE;
        int cnt = 0, first = 0, cntv = 0, res = 0;
        if (np == PH_RESID) {          // the longest tasks: listed apart, claimed first
            cnt = D.n64;
            first = D.t64;
            res = 1;
        } else if (np == PH_CG || np == PH_GM || np == PH_START) {   // START: A32 / A32lo split
            cnt = D.n32;
            first = E.n64 + D.t32;
        }
        if (np == PH_START || np == PH_INIT || np == PH_CG || np == PH_GM || np == PH_UPDATE) cntv = D.nv;
        cnt_s = cnt;
        first_s = first;
        cntv_s = cntv;
        res_s = res;
        base_s = cnt ? atomicAdd(&E.active[(res ? A_LEN_RES : A_LEN_PROD) + par], cnt) : 0;
        basev_s = cntv ? atomicAdd(&E.active[A_LEN_VEC + par], cntv) : 0;
    }
    __syncthreads();
    {
        int *wp = E.work[par] + (res_s ? E.wres : 0);
        for (int i = threadIdx.x; i < cnt_s; i += RED_T) wp[base_s + i] = first_s + i;
        int *wv = E.work[par] + E.wvec;
        for (int i = threadIdx.x; i < cntv_s; i += RED_T) wv[basev_s + i] = D.tv + i;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int act = 0;
        if (ph != PH_FREE && ph != PH_DONE) {
            S.phase = newphase_s;
            act = (newphase_s != PH_DONE);
        }
        if (act) atomicAdd(&E.active[A_COUNT], 1);
        __threadfence();
        const int tk = atomicAdd(&E.active[A_TICKET], 1);
        if (tk == (int)gridDim.x - 1) {       // last block: loop control
            __threadfence();
            const int total = atomicAdd(&E.active[A_COUNT], 0);
            const int ticks = E.active[A_TICKS] + 1;
            E.active[A_TICKS] = ticks;
            const int go = total > 0 && ticks < E.tick_limit;
            if (E.host_loop) E.active[A_GO] = go;
            else cudaGraphSetConditional(h, go);
            E.active[A_COUNT] = 0;
            E.active[A_TICKET] = 0;
            E.active[A_LAST] = total;
            E.active[A_CLAIM_PROD] = 0;    // task claim counters of eng_prod / eng_vec
            E.active[A_CLAIM_VEC] = 0;
            E.active[A_LEN_PROD + (par ^ 1)] = 0;   // lists of the next tick
            E.active[A_LEN_RES + (par ^ 1)] = 0;
            E.active[A_LEN_VEC + (par ^ 1)] = 0;
        }
    }
}

// ============================================================================
// eng_prod: one CTA per SM, warp-specialised.  The producer warp claims the
// tick's runnable tasks and streams, for every 32-column chunk of an FP32
// product task, the 256 x 32 tile of A32 (2-D TMA, 128-byte swizzle) and the
// operand inputs (1-D bulk copies of the rows k0 .. k0+31 of the n x sp
// blocks) into a ring of shared-memory stages, across task boundaries; the
// eight consumer warps multiply.  Refinement-residual tasks stream the same
// way (A32 and A32lo tiles, Xh and Xl rows); A-split tasks pass through the
// ring as one header-only stage each and are run by the consumers with
// ordinary loads.
// ============================================================================
constexpr int PC_W = P32_T / 32;                     // consumer warps
constexpr int PROD_T = P32_T + 64;                   // + the producer warp and the MMA warp
constexpr int PSTAGES = 3;                           // ring stages
constexpr int PREFETCH = 4;                          // tiles of a task brought into L2 ahead of their copy
constexpr int TILE_B = E_RB32 * E_KC32 * 4;          // 32 KB A tile
constexpr int OPR_B = E_KC32 * 32 * 4;               // one raw operand chunk (widest slot)
constexpr int BOP_B = E_MAXS * E_KC32 * 4;           // one K-major tensor-core B operand (4 KB)
constexpr int TMEM_COLS = 256;                       // two 128-row halves of the tile:
constexpr int TC_HALF_COLS = 128;                    // per half Ah [Bh | Bt] (2 sp columns), then At Bh (sp)
static_assert(E_KC32 * 4 == 128, "a tile row is one 128-byte swizzle row");

struct StageHdr {
    int kind, u, k0, flags;
    int slot, sp, pad_[2];
    float colscale[32];
    int colstop[32];
};
enum : int { SK_STOP = 0, SK_PROD = 1, SK_GENERIC = 2, SK_RES = 3 };
enum : int { SF_FIRST = 1, SF_LAST = 2, SF_SRC2 = 4 };

constexpr size_t align_c(size_t v, size_t a) { return (v + a - 1) / a * a; }
constexpr size_t OFF_TILE = 0;                                         // 1024-aligned tiles
constexpr size_t OFF_CVT = OFF_TILE + (size_t)PSTAGES * TILE_B;        // [2] tensor-core tail tiles
constexpr size_t OFF_BOP = OFF_CVT + 2 * (size_t)TILE_B;               // [2] B operands [head; tail] /
                                                                       // the FP32 path's two operand chunks
constexpr size_t OFF_OPR = OFF_BOP + 4 * (size_t)BOP_B;                // [stage][2][OPR_B]
constexpr size_t OFF_HDR = OFF_OPR + (size_t)PSTAGES * 2 * OPR_B;
// barriers: full[PSTAGES], empty[PSTAGES], mma[2], conv[2]
constexpr size_t OFF_BAR = align_c(OFF_HDR + PSTAGES * sizeof(StageHdr), 16);
constexpr size_t OFF_TCQ = OFF_BAR + (2 * PSTAGES + 4) * sizeof(uint64_t);   // 2 hand-over entries
constexpr size_t OFF_TSLOT = OFF_TCQ + 2 * 16;
constexpr size_t OFF_RED = align_c(OFF_TSLOT + 16, 16);                // 1024 doubles
constexpr size_t PROD_SMEM = OFF_RED + 1024 * sizeof(double) + 1024;  // + alignment slack
static_assert(OFF_CVT % 1024 == 0 && OFF_BOP % 1024 == 0, "swizzled operands need 1024-byte alignment");
static_assert(PROD_SMEM <= 232448, "shared memory of one CTA");
static_assert(BOP_B == OPR_B, "the FP32 path's operand buffer aliases a B operand");

struct TcQ;
struct ProdSmem {
    unsigned char *base;
    __device__ float *tile(int st) const { return reinterpret_cast<float *>(base + OFF_TILE + (size_t)st * TILE_B); }
    __device__ float *opr(int st, int w) const {
        return reinterpret_cast<float *>(base + OFF_OPR + ((size_t)st * 2 + w) * OPR_B);
    }
    __device__ StageHdr *hdr(int st) const { return reinterpret_cast<StageHdr *>(base + OFF_HDR) + st; }
    __device__ uint64_t *full(int st) const { return reinterpret_cast<uint64_t *>(base + OFF_BAR) + st; }
    __device__ uint64_t *empty(int st) const {
        return reinterpret_cast<uint64_t *>(base + OFF_BAR) + PSTAGES + st;
    }
    // tensor-core path: products of buffer parity b done / chunk of parity b handed over
    __device__ uint64_t *mma(int b) const { return reinterpret_cast<uint64_t *>(base + OFF_BAR) + 2 * PSTAGES + b; }
    __device__ uint64_t *conv(int b) const {
        return reinterpret_cast<uint64_t *>(base + OFF_BAR) + 2 * PSTAGES + 2 + b;
    }
    __device__ struct TcQ *tcq() const { return reinterpret_cast<struct TcQ *>(base + OFF_TCQ); }
    __device__ uint32_t *tslot() const { return reinterpret_cast<uint32_t *>(base + OFF_TSLOT); }
    // FP32 path: operand chunk b (32 rows x sp, row-major)
    __device__ float *ps(int b) const { return reinterpret_cast<float *>(base + OFF_BOP + (size_t)b * BOP_B); }
    // tensor-core path, buffer parity b: the TF32 tail of the A tile (its head is written over
    // the stage's tile) and the B operand, 2 sp rows of 128 bytes: the operand's head, then its tail
    __device__ float *tail(int b) const { return reinterpret_cast<float *>(base + OFF_CVT + (size_t)b * TILE_B); }
    __device__ float *bop(int b) const { return reinterpret_cast<float *>(base + OFF_BOP + (size_t)b * 2 * BOP_B); }
    __device__ double *red() const { return reinterpret_cast<double *>(base + OFF_RED); }
};

__device__ __forceinline__ void release_stage(const ProdSmem &M, int st) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(M.empty(st));
}

// ----------------------------------------------------------------------------
// consumers: one FP32 product task, Y = Ahat P for 256 rows x D.ks32
// columns of A, all SP columns.  Each thread owns RPT rows (rg + NRG r) x 4
// columns (cg); per 4 k it reads each row's 4 A values with one 16-byte load
// from the swizzled tile and 4 operand quads, then does 16 RPT multiply-adds
// in increasing k.  The first stage was waited for by the caller.  When the
// row block has several K chunks, each task stores its partial product and
// the last one to finish sums them in chunk order and runs the epilogue: Y
// rows and the partial dots.  Returns false on a timeout (all consumers
// together).
// ----------------------------------------------------------------------------
// ----------------------------------------------------------------------------
// The end of an FP32 product task, given the task's accumulators acc (thread
// (rg, cg) holds rows rg + NRG r, columns 4 cg .. 4 cg + 3): split-K partials,
// the Y rows of the row block and its partial dots.
// ----------------------------------------------------------------------------
template <int SP>
__device__ bool prod_epilogue(const EngineDev &E, const ProdSmem &M, const Task &T, int ph, int it,
                              const float *dst, float *out, float (&acc)[SP / 4][4], int *flag_s) {
    constexpr int RPT = SP / 4, NCG = SP / 4, NRG = E_RB32 / RPT;
    const int tid = threadIdx.x, rg = tid / NCG, cg = tid % NCG;
    const SlotDesc &D = E.desc[T.slot];
    const int n = D.n;
    const long long nsp = (long long)n * SP;
    const int r0 = T.r0, nrow = T.r1 - T.r0;
    const int kc32 = (n + D.ks32 - 1) / D.ks32;
    if (kc32 > 1) {
        // publish this chunk's partial product; the last task of the row block
        // adds all chunks in chunk order
        float *yk = D.Yk + (long long)T.kc * nsp;
#pragma unroll
        for (int r = 0; r < RPT; r++) {
            const int row = rg + NRG * r;
            if (row < nrow)
                __stcg(reinterpret_cast<float4 *>(yk + (long long)(r0 + row) * SP + cg * 4),
                       make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]));
        }
        named_bar(1, P32_T);
        const int rbl = r0 / E_RB32;
        if (tid == 0) {     // the CTA's stores are ordered before this by the barrier
            const int last = atom_add_acq_rel(D.ticket + rbl, 1) == kc32 - 1;
            if (last) D.ticket[rbl] = 0;                        // ready for the next tick
            *flag_s = last;
        }
        named_bar(1, P32_T);
        if (!*flag_s) return true;
#pragma unroll
        for (int r = 0; r < RPT; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[r][c] = 0.0f;
        for (int q = 0; q < kc32; q++) {
            const float *yq = D.Yk + (long long)q * nsp;
#pragma unroll
            for (int r = 0; r < RPT; r++) {
                const int row = rg + NRG * r;
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
        const int row = rg + NRG * r;
        if (row < nrow)
            *reinterpret_cast<float4 *>(out + (long long)(r0 + row) * SP + cg * 4) =
                make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
    }
    // partial dots over this row block: CG p.q; GMRES v_i.w for i <= it
    // (the new direction's rows may come from another task: read through L2).
    // Per dot: a shuffle tree over the warp's row groups, then the 8 warps'
    // sums in warp order; the two halves of Red alternate between dots.  The
    // sums run in double-single arithmetic (each product of two FP32 values
    // exact, about 48 bits kept) on the FP32 pipe: a warp's FP64 instruction
    // takes about 64 cycles of its scheduler's FP64 unit on this GPU, and a
    // GMRES epilogue forms up to m dots of RPT x 4 products per thread.
    float2 *Red = reinterpret_cast<float2 *>(M.red());
    const int nd = ph == PH_CG ? 1 : it + 1;
    const int lane = tid & 31, warp = tid >> 5;
    for (int i = 0; i < nd; i++) {
        const float *vi = ph == PH_CG ? dst : D.V + (long long)i * nsp;
        DSV pc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
        for (int r = 0; r < RPT; r++) {
            const int row = rg + NRG * r;
            if (row < nrow) {
                const float4 v = __ldcg(reinterpret_cast<const float4 *>(vi + (long long)(r0 + row) * SP + cg * 4));
                ds_fma(v.x, 0.0f, DSV{acc[r][0], 0.0f}, pc[0]);
                ds_fma(v.y, 0.0f, DSV{acc[r][1], 0.0f}, pc[1]);
                ds_fma(v.z, 0.0f, DSV{acc[r][2], 0.0f}, pc[2]);
                ds_fma(v.w, 0.0f, DSV{acc[r][3], 0.0f}, pc[3]);
            }
        }
#pragma unroll
        for (int o = NCG; o < 32; o <<= 1)
#pragma unroll
            for (int c = 0; c < 4; c++) pc[c] += shfl_xor_v(pc[c], o);
        float2 *Rb = Red + (i & 1) * (PC_W * 32);
        if (lane < NCG)
#pragma unroll
            for (int c = 0; c < 4; c++) Rb[warp * 32 + lane * 4 + c] = make_float2(pc[c].h, pc[c].l);
        named_bar(1, P32_T);
        if (tid < 32) {
            DSV sacc{0.f, 0.f};
            if (tid < SP)
                for (int w = 0; w < PC_W; w++) {
                    const float2 t = Rb[w * 32 + tid];
                    sacc += DSV{t.x, t.y};
                }
            E.part32[((size_t)T.rb * E_PS + i) * 32 + tid] = to_double(sacc);
        }
    }
    named_bar(1, P32_T);        // Red free for the next task
    return true;
}

template <int SP>
__device__ bool prod_task(const EngineDev &E, const ProdSmem &M, int &seq, int *flag_s) {
    constexpr int KC = E_KC32;
    constexpr int RPT = SP / 4;                 // rows per thread
    constexpr int NCG = SP / 4;                 // column groups of 4
    constexpr int NRG = E_RB32 / RPT;           // row groups
    static_assert(NRG * NCG == P32_T, "thread grid");
    static_assert(NRG % 8 == 0, "a thread's rows share one swizzle phase");
    const int tid = threadIdx.x, rg = tid / NCG, cg = tid % NCG;
    const StageHdr &H0 = *M.hdr(seq % PSTAGES);
    const int u = H0.u;
    const Task T = E.t32[u - E.n64];
    const SlotDesc &D = E.desc[T.slot];
    const SlotState &S = E.st[T.slot];
    const int ph = S.phase;
    const int n = D.n, s = D.s, it = S.it;
    const long long nsp = (long long)n * SP;
    const int r0 = T.r0, r1 = T.r1;
    float *dst, *out;
    if (ph == PH_CG) {
        dst = D.P + (it & 1) * nsp;
        out = D.Q;
    } else {
        dst = D.V + (long long)it * nsp;
        out = D.W + ((it + 1) & 1) * nsp;
    }
    float acc[RPT][4];
#pragma unroll
    for (int r = 0; r < RPT; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[r][c] = 0.0f;
    const int nch = (T.k1 - T.k0 + KC - 1) / KC;
    for (int ch = 0; ch < nch; ch++) {
        const int st = seq % PSTAGES;
        const bool ok = ch == 0 || mbar_wait(M.full(st), (seq / PSTAGES) & 1);
        float *Ps = M.ps(ch & 1);
        if (ok) {   // the operand chunk: P = Rf + beta P' (CG) or V_k = W / h (GMRES)
            // thread tid always builds column tid % SP (SP divides the block)
            const StageHdr &H = *M.hdr(st);
            const float *o1 = M.opr(st, 0), *o2 = M.opr(st, 1);
            const bool two = (H.flags & SF_SRC2) != 0;
            const int k0 = H.k0, c = tid % SP;
            const bool live = c < s && !(ph == PH_CG && H.colstop[c]);
            const float cs = H.colscale[c];
            const bool own = k0 < r1 && k0 + KC > r0;           // the chunk holds rows of this block
#pragma unroll
            for (int j = 0; j < (KC * SP + P32_T - 1) / P32_T; j++) {
                const int e = tid + j * P32_T;
                if (KC * SP % P32_T == 0 || e < KC * SP) {
                    const int gk = k0 + e / SP;
                    float val = 0.0f;
                    if (live && gk < n) {
                        if (ph == PH_CG) val = two ? fmaf(cs, o2[e], o1[e]) : o1[e];
                        else val = o1[e] * cs;
                        if (own && gk >= r0 && gk < r1) dst[(long long)gk * SP + c] = val;   // owned rows
                    }
                    Ps[e] = val;
                }
            }
        }
        if (named_bar_or(1, P32_T, !ok)) return false;
        // rows rg + NRG r share the swizzle phase rg & 7 (NRG is a multiple
        // of 8): one chunk offset per k quad, fixed offsets between the rows.
        // The next quad's operands are loaded before this quad's FMAs.
        const float *At = M.tile(st) + rg * KC;
        const int sw = rg & 7;
        float4 a[2][RPT], p[2][4];
        auto load_q = [&](int kq, int b) {
            const float *Aq = At + ((kq ^ sw) << 2);
#pragma unroll
            for (int r = 0; r < RPT; r++) a[b][r] = *reinterpret_cast<const float4 *>(Aq + r * NRG * KC);
#pragma unroll
            for (int j = 0; j < 4; j++) p[b][j] = *reinterpret_cast<const float4 *>(Ps + (4 * kq + j) * SP + cg * 4);
        };
        load_q(0, 0);
#pragma unroll
        for (int kq = 0; kq < KC / 4; kq++) {
            const int b = kq & 1;
            if (kq + 1 < KC / 4) load_q(kq + 1, b ^ 1);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const float pc[4] = {p[b][j].x, p[b][j].y, p[b][j].z, p[b][j].w};
#pragma unroll
                for (int r = 0; r < RPT; r++) {
                    const float av = j == 0 ? a[b][r].x : j == 1 ? a[b][r].y : j == 2 ? a[b][r].z : a[b][r].w;
#pragma unroll
                    for (int c = 0; c < 4; c++) acc[r][c] = fmaf(av, pc[c], acc[r][c]);
                }
            }
        }
        release_stage(M, st);
        seq++;
    }
    return prod_epilogue<SP>(E, M, T, ph, it, dst, out, acc, flag_s);
}

// ----------------------------------------------------------------------------
// Tensor-core form of the FP32 product task (sp = 16 or 32).  The consumers
// build each chunk's operand as in the FP32 form; then every FP32 value v of
// the chunk and of the 256 x 32 tile of A is split into a TF32 head h = rn(v)
// and a TF32 tail t = rn(v - h) (v = h + t to about 2^-24 |v|): the tile's
// head is written over the tile, its tail into the tail tile of the buffer
// parity, the operand's head and tail as the two halves of one K-major
// 128-byte-swizzled B operand [Bh; Bt] of 2 sp rows.  The chunk is then
// handed to the MMA warp, which issues, per 8-column step of K and per
// 128-row half of the tile (tcgen05.mma kind::tf32, FP32 accumulators in
// tensor memory),
//     D1 += Ah [Bh | Bt]   (N = 2 sp: A's head is read once for both)
//     D2 += At Bh          (N = sp)
// so that Y = D1[:, :sp] + D1[:, sp:] + D2 (the dropped At Bt is below
// 2^-24 |A||P|), and commits twice: to the stage's "empty" barrier (the
// stage goes back to the producer when the products that read it are done)
// and to the parity's "done" barrier (the consumers may then overwrite that
// parity's tail tile and B operand, two chunks later).  The consumers wait
// for the tensor core only before reusing a buffer parity and for the task's
// last chunk; the accumulators then come back through tcgen05.ld, summed,
// through a shared-memory staging copy into the FP32 form's register layout,
// and the task ends as the FP32 form does.
// ----------------------------------------------------------------------------
struct TcQ {                 // a chunk handed to the MMA warp
    int st;                  // ring stage holding the tile's head
    int sp;                  // 16 or 32
    int first;               // first chunk of its task (accumulators start from zero)
    int stop;                // no more chunks in this launch
};

struct TcCtx {
    uint32_t tmem;           // accumulators: half h at column 128 h (D1: 2 sp columns, then D2: sp)
    unsigned cseq;           // chunks handed to the MMA warp by this CTA
    int *fail_s;             // a wait gave up: every later wait returns at once
};

// Bounded wait that also gives up at once after an earlier failure (so a
// failed task cannot queue one time limit after another).
__device__ __forceinline__ bool tc_wait(uint64_t *bar, unsigned parity, int *fail_s) {
    if (*(volatile int *)fail_s) return false;
    if (mbar_wait(bar, parity)) return true;
    *(volatile int *)fail_s = 1;
    return false;
}

template <int SP>
__device__ bool prod_task_tc(const EngineDev &E, const ProdSmem &M, int &seq, int *flag_s, TcCtx &tc) {
    constexpr int KC = E_KC32;
    constexpr int RPT = SP / 4, NCG = SP / 4, NRG = E_RB32 / RPT;
    constexpr int KQ = KC / 4;                  // 16-byte quads of K per chunk
    constexpr int F4 = SP / 4, SWM = F4 - 1;    // staging: float4 per row, swizzle mask
    static_assert(SP == 16 || SP == 32, "M = 128 needs N a multiple of 16");
    static_assert(3 * SP <= TC_HALF_COLS && 2 * TC_HALF_COLS <= TMEM_COLS, "D1 and D2 of both halves");
    static_assert(2 * SP * KC * 4 <= 2 * BOP_B, "B operand [head; tail]");
    static_assert(E_RB32 * SP * 4 <= TILE_B, "the staging copy fits a tail tile");
    const int tid = threadIdx.x, rg = tid / NCG, cg = tid % NCG;
    const int warp = tid >> 5, lane = tid & 31;
    const StageHdr &H0 = *M.hdr(seq % PSTAGES);
    const int u = H0.u;
    const Task T = E.t32[u - E.n64];
    const SlotDesc &D = E.desc[T.slot];
    const SlotState &S = E.st[T.slot];
    const int ph = S.phase;
    const int n = D.n, s = D.s, it = S.it;
    const long long nsp = (long long)n * SP;
    const int r0 = T.r0, r1 = T.r1;
    float *dst, *out;
    if (ph == PH_CG) {
        dst = D.P + (it & 1) * nsp;
        out = D.Q;
    } else {
        dst = D.V + (long long)it * nsp;
        out = D.W + ((it + 1) & 1) * nsp;
    }
    const int nch = (T.k1 - T.k0 + KC - 1) / KC;
    for (int ch = 0; ch < nch; ch++) {
        const int st = seq % PSTAGES;
        bool ok = ch == 0 || tc_wait(M.full(st), (seq / PSTAGES) & 1, tc.fail_s);
        const unsigned q = tc.cseq;
        const int b = q & 1;
        // the tail tile and B operand of parity b were last read by chunk q - 2
        if (q >= 2) ok = tc_wait(M.mma(b), ((q - 2) >> 1) & 1, tc.fail_s) && ok;
        if (ok) {
            const StageHdr &H = *M.hdr(st);
            const float *o1 = M.opr(st, 0), *o2 = M.opr(st, 1);
            const bool two = (H.flags & SF_SRC2) != 0;
            const int k0 = H.k0;
            float *Bo = M.bop(b);
            // thread (c, kq): rows 4 kq .. 4 kq + 3 of operand column c
            for (int e = tid; e < SP * KQ; e += P32_T) {
                const int c = e % SP, kq = e / SP;
                const bool live = c < s && !(ph == PH_CG && H.colstop[c]);
                const float cs = H.colscale[c];
                float hv[4], tv[4];
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int kl = 4 * kq + j, gk = k0 + kl;
                    float val = 0.0f;
                    if (live && gk < n) {
                        const int oe = kl * SP + c;
                        if (ph == PH_CG) val = two ? fmaf(cs, o2[oe], o1[oe]) : o1[oe];
                        else val = o1[oe] * cs;
                        if (gk >= r0 && gk < r1) dst[(long long)gk * SP + c] = val;   // owned rows
                    }
                    hv[j] = tf32_rn(val);
                    tv[j] = tf32_rn(val - hv[j]);
                }
                const int pos = c * KC + ((kq ^ (c & 7)) << 2);      // rows c and SP + c: same swizzle phase
                *reinterpret_cast<float4 *>(Bo + pos) = make_float4(hv[0], hv[1], hv[2], hv[3]);
                *reinterpret_cast<float4 *>(Bo + SP * KC + pos) = make_float4(tv[0], tv[1], tv[2], tv[3]);
            }
            float4 *Ah4 = reinterpret_cast<float4 *>(M.tile(st));
            float4 *At4 = reinterpret_cast<float4 *>(M.tail(b));
#pragma unroll 4
            for (int e = tid; e < TILE_B / 16; e += P32_T) {
                const float4 a = Ah4[e];
                const float4 h = make_float4(tf32_rn(a.x), tf32_rn(a.y), tf32_rn(a.z), tf32_rn(a.w));
                Ah4[e] = h;
                At4[e] = make_float4(tf32_rn(a.x - h.x), tf32_rn(a.y - h.y), tf32_rn(a.z - h.z), tf32_rn(a.w - h.w));
            }
        }
        if (tid == 0) {
            TcQ &Q = M.tcq()[b];
            Q.st = st;
            Q.sp = SP;
            Q.first = ch == 0;
            Q.stop = 0;
        }
        fence_async_smem();          // this thread's shared-memory writes, before the tensor core reads them
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(M.conv(b));
            if (warp != PC_W - 1) mbar_arrive(M.empty(st));   // the eighth arrival: the MMA warp's commit
        }
        tc.cseq++;
        seq++;
    }
    // the task's last products
    const unsigned lq = tc.cseq - 1;
    bool ok = tc_wait(M.mma(lq & 1), (lq >> 1) & 1, tc.fail_s);
    if (named_bar_or(1, P32_T, !ok)) return false;
    tc_fence_after();
    {   // accumulators -> registers (D1 head + D1 tail + D2) -> staging copy
        // (row-major, float4 f of row r at f ^ (r & SWM))
        const int h = warp >> 2, qw = warp & 3;
        const int row = h * 128 + qw * 32 + lane;
        const uint32_t ta = tc.tmem + ((uint32_t)(qw * 32) << 16) + (uint32_t)(TC_HALF_COLS * h);
        float4 *Ys = reinterpret_cast<float4 *>(M.tail(0));
#pragma unroll
        for (int c0 = 0; c0 < SP; c0 += 16) {
            float v1[16], v2[16], v3[16];
            tmem_ld16(ta + c0, v1);
            tmem_ld16(ta + SP + c0, v2);
            tmem_ld16(ta + 2 * SP + c0, v3);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int f = c0 / 4 + j;
                float y[4];
#pragma unroll
                for (int c = 0; c < 4; c++) y[c] = (v1[4 * j + c] + v2[4 * j + c]) + v3[4 * j + c];
                Ys[row * F4 + (f ^ (row & SWM))] = make_float4(y[0], y[1], y[2], y[3]);
            }
        }
    }
    tc_fence_before();
    named_bar(1, P32_T);
    float acc[RPT][4];
    {
        const float4 *Ys = reinterpret_cast<const float4 *>(M.tail(0));
#pragma unroll
        for (int r = 0; r < RPT; r++) {
            const int row = rg + NRG * r;
            const float4 v = Ys[row * F4 + (cg ^ (row & SWM))];
            acc[r][0] = v.x;
            acc[r][1] = v.y;
            acc[r][2] = v.z;
            acc[r][3] = v.w;
        }
    }
    return prod_epilogue<SP>(E, M, T, ph, it, dst, out, acc, flag_s);
}

// Consumers leaving the launch: a stop entry for the MMA warp (once it has
// taken the entry two places back, so the barrier phases stay in step).
__device__ __forceinline__ void tc_send_stop(const ProdSmem &M, TcCtx &tc) {
    const unsigned q = tc.cseq;
    const int b = q & 1;
    if (q >= 2) tc_wait(M.mma(b), ((q - 2) >> 1) & 1, tc.fail_s);
    if (threadIdx.x == 0) M.tcq()[b].stop = 1;
    named_bar(1, P32_T);
    if ((threadIdx.x & 31) == 0) mbar_arrive(M.conv(b));
}

// The MMA warp: one lane issues every chunk's products in hand-over order.
// Returns the number of chunks it issued.
__device__ unsigned tc_mma_warp(const EngineDev &E, const ProdSmem &M, uint32_t tmem) {
    const int lane = threadIdx.x & 31;
    unsigned j = 0;
    for (;;) {
        const int b = j & 1;
        const bool ok = __all_sync(0xffffffffu, mbar_wait(M.conv(b), (j >> 1) & 1));
        if (!ok) {
            if (lane == 0) atomicExch(E.active + A_ERR, 1);
            break;
        }
        const TcQ Q = M.tcq()[b];
        if (Q.stop) break;
        if (lane == 0) {
            tc_fence_after();
            const uint32_t ah = smem_u32(M.tile(Q.st)), at = smem_u32(M.tail(b)), bo = smem_u32(M.bop(b));
            const int sp = Q.sp;
            const uint32_t id1 = tc_idesc_tf32(128, 2 * sp), id2 = tc_idesc_tf32(128, sp);
#pragma unroll
            for (int kk = 0; kk < E_KC32 / 8; kk++) {
                const uint64_t db = tc_desc_sw128(bo + kk * 32);     // [Bh; Bt], and Bh its first sp rows
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const uint32_t d1 = tmem + TC_HALF_COLS * h, d2 = d1 + 2 * sp;
                    const uint32_t ao = h * (TILE_B / 2) + kk * 32;
                    const bool acc = !Q.first || kk > 0;
                    tc_mma_tf32(d1, tc_desc_sw128(ah + ao), db, id1, acc);
                    tc_mma_tf32(d2, tc_desc_sw128(at + ao), db, id2, acc);
                }
            }
            tc_commit(M.empty(Q.st));
            tc_commit(M.mma(b));
        }
        __syncwarp();
        j++;
    }
    return j;
}

// ----------------------------------------------------------------------------
// consumers: one refinement-residual task, R = B - A X for 256 rows and the
// task's ks64(SP) columns of A, to about FP64 accuracy on the FP32 pipe.
// A = A32 + A32lo and X = Xh + Xl are fp32 pairs; each 32-column chunk comes
// as two stages (A32 tile + Xh rows, then A32lo tile + Xl rows).  Each term
// a x = ah xh + ah xl + al xh (+ al xl, below 2^-48 |a x|, dropped) is
// accumulated in a (hi, lo) pair: ah xh = p + e exactly (product error by
// FMA), hi += p exactly with the rounding error moved to lo (two-sum, Knuth),
// lo also takes e and the cross terms.  Thread tile: RPT rows x 4 columns as
// in the FP32 product.  The (hi, lo) totals are formed in FP64; split-K
// partials are added in chunk order by the last task of the row block, which
// also stores R and the partial ||R_j||^2 of its rows.
// ----------------------------------------------------------------------------
template <int SP>
__device__ bool res_task(const EngineDev &E, const ProdSmem &M, int &seq, int *flag_s) {
    constexpr int KC = E_KC32;
    constexpr int RPT = SP / 4, NCG = SP / 4, NRG = E_RB32 / RPT;
    static_assert(NRG * NCG == P32_T && NRG % 8 == 0, "thread grid");
    static_assert(ks64(SP) % KC == 0, "K chunks hold whole shared-memory chunks");
    const int tid = threadIdx.x, rg = tid / NCG, cg = tid % NCG;
    const int u = M.hdr(seq % PSTAGES)->u;
    const Task T = E.t64[u];
    const SlotDesc &D = E.desc[T.slot];
    const int n = D.n, s = D.s;
    const long long nsp = (long long)n * SP;
    const int r0 = T.r0, nrow = T.r1 - T.r0;
    float hi[RPT][4], lo[RPT][4];
#pragma unroll
    for (int r = 0; r < RPT; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) hi[r][c] = lo[r][c] = 0.0f;
    const int sw = rg & 7;
    const int nch = (T.k1 - T.k0 + KC - 1) / KC;
    for (int ch = 0; ch < nch; ch++) {
        const int sa = seq % PSTAGES, sb = (seq + 1) % PSTAGES;
        bool ok = ch == 0 || mbar_wait(M.full(sa), (seq / PSTAGES) & 1);
        ok = ok && mbar_wait(M.full(sb), ((seq + 1) / PSTAGES) & 1);
        if (named_bar_or(1, P32_T, !ok)) return false;
        const int rows = min(KC, n - M.hdr(sa)->k0);         // operand rows present
        const float *Ah = M.tile(sa) + rg * KC, *Al = M.tile(sb) + rg * KC;
        const float *Xh = M.opr(sa, 0) + cg * 4, *Xl = M.opr(sb, 0) + cg * 4;
#pragma unroll 4
        for (int kk = 0; kk < KC; kk++) {
            const int off = (((kk >> 2) ^ sw) << 2) + (kk & 3);
            float ah[RPT], al[RPT];
#pragma unroll
            for (int r = 0; r < RPT; r++) {
                ah[r] = Ah[off + r * NRG * KC];
                al[r] = Al[off + r * NRG * KC];
            }
            float4 xh4 = make_float4(0.f, 0.f, 0.f, 0.f), xl4 = xh4;
            if (kk < rows) {                                    // beyond n the rows were not copied
                xh4 = *reinterpret_cast<const float4 *>(Xh + kk * SP);
                xl4 = *reinterpret_cast<const float4 *>(Xl + kk * SP);
            }
            const float xh[4] = {xh4.x, xh4.y, xh4.z, xh4.w}, xl[4] = {xl4.x, xl4.y, xl4.z, xl4.w};
#pragma unroll
            for (int r = 0; r < RPT; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const float p = __fmul_rn(ah[r], xh[c]);
                    const float pe = fmaf(ah[r], xh[c], -p);            // ah xh - p, exact
                    const float tc = fmaf(al[r], xh[c], fmaf(ah[r], xl[c], pe));
                    const float sh = __fadd_rn(hi[r][c], p);
                    const float bv = __fsub_rn(sh, hi[r][c]);
                    const float er = __fadd_rn(__fsub_rn(hi[r][c], __fsub_rn(sh, bv)), __fsub_rn(p, bv));
                    hi[r][c] = sh;
                    lo[r][c] = __fadd_rn(lo[r][c], __fadd_rn(tc, er));
                }
        }
        release_stage(M, sa);
        release_stage(M, sb);
        seq += 2;
    }
    double v[RPT][4];
#pragma unroll
    for (int r = 0; r < RPT; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) v[r][c] = (double)hi[r][c] + (double)lo[r][c];
    const int kc64 = (n + ks64(SP) - 1) / ks64(SP);
    if (kc64 > 1) {
        double *rk = D.Rk + (long long)T.kc * nsp;
#pragma unroll
        for (int r = 0; r < RPT; r++) {
            const int row = rg + NRG * r;
            if (row < nrow) {
                double *q = rk + (long long)(r0 + row) * SP + cg * 4;
                __stcg(reinterpret_cast<double2 *>(q), make_double2(v[r][0], v[r][1]));
                __stcg(reinterpret_cast<double2 *>(q + 2), make_double2(v[r][2], v[r][3]));
            }
        }
        named_bar(1, P32_T);
        const int rbl = r0 / E_RB32;
        if (tid == 0) {     // the CTA's stores are ordered before this by the barrier
            const int last = atom_add_acq_rel(D.ticket + rbl, 1) == kc64 - 1;
            if (last) D.ticket[rbl] = 0;                        // ready for the next tick
            *flag_s = last;
        }
        named_bar(1, P32_T);
        if (!*flag_s) return true;
#pragma unroll
        for (int r = 0; r < RPT; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) v[r][c] = 0.0;
        for (int q = 0; q < kc64; q++) {
            const double *rq = D.Rk + (long long)q * nsp;
#pragma unroll
            for (int r = 0; r < RPT; r++) {
                const int row = rg + NRG * r;
                if (row < nrow) {
                    const double *pq = rq + (long long)(r0 + row) * SP + cg * 4;
                    const double2 a = __ldcg(reinterpret_cast<const double2 *>(pq));
                    const double2 b = __ldcg(reinterpret_cast<const double2 *>(pq + 2));
                    v[r][0] += a.x;
                    v[r][1] += a.y;
                    v[r][2] += b.x;
                    v[r][3] += b.y;
                }
            }
        }
    }
    // R = B - A X for the row block, partial ||R_j||^2 (shuffle tree over the
    // warp's row groups, then the 8 warps in order)
    double pc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int r = 0; r < RPT; r++) {
        const int row = rg + NRG * r;
        if (row < nrow) {
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const long long o = (long long)(r0 + row) * SP + cg * 4 + c;
                const double rv = cg * 4 + c < s ? D.B[o] - v[r][c] : 0.0;
                D.R[o] = rv;
                pc[c] += rv * rv;
            }
        }
    }
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int o = NCG; o < 32; o <<= 1)
#pragma unroll
        for (int c = 0; c < 4; c++) pc[c] += __shfl_xor_sync(0xffffffffu, pc[c], o);
    double *Rb = M.red();
    if (lane < NCG)
#pragma unroll
        for (int c = 0; c < 4; c++) Rb[warp * 32 + lane * 4 + c] = pc[c];
    named_bar(1, P32_T);
    if (tid < 32) {
        double sacc = 0.0;
        if (tid < SP)
            for (int w = 0; w < PC_W; w++) sacc += Rb[w * 32 + tid];
        E.part64[(size_t)T.rb * 32 + tid] = sacc;
    }
    named_bar(1, P32_T);        // Red free for the next task
    return true;
}

// At admission (START), the FP32 product tasks' parts of A are split instead:
// A = A32 + A32lo for the task's rows and columns, written in the tile-major
// layout of a32_tile (the task that ends at column n also writes the zero
// columns up to a32_ncols(n)).  A warp takes 128 columns (four tiles' rows)
// of one row at a time, a lane four consecutive columns, four such pieces in
// flight per warp; split_pair works on the bit pattern with integer
// operations, off the FP64 pipe.
__device__ __forceinline__ void convert_task(const SlotDesc &D, const Task &T) {
    constexpr int NW = P32_T / 32, U = 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = D.n;
    const int kw = T.k1 == n ? (int)a32_ncols(n) : T.k1;
    const int nseg = (kw - T.k0 + 127) / 128;
    const int items = (T.r1 - T.r0) * nseg;
    const bool vec = (D.lda64 & 1) == 0 && ((uintptr_t)D.A64 & 15) == 0;
    for (int base = warp; base < items; base += U * NW) {
        double v[U][4];
        int rr[U], kk[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int item = base + u * NW;
            rr[u] = T.r0 + item / nseg;
            kk[u] = T.k0 + (item % nseg) * 128 + 4 * lane;
            if (item >= items) kk[u] = kw;             // nothing to do
            const double *a = D.A64 + (long long)rr[u] * D.lda64 + kk[u];
            if (kk[u] < kw && vec && kk[u] + 3 < n) {
                const double2 x = __ldcs(reinterpret_cast<const double2 *>(a));
                const double2 y = __ldcs(reinterpret_cast<const double2 *>(a) + 1);
                v[u][0] = x.x;
                v[u][1] = x.y;
                v[u][2] = y.x;
                v[u][3] = y.y;
            } else {
#pragma unroll
                for (int c = 0; c < 4; c++) v[u][c] = kk[u] < kw && kk[u] + c < n ? __ldcs(a + c) : 0.0;
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (kk[u] >= kw) continue;
            float h[4], l[4];
#pragma unroll
            for (int c = 0; c < 4; c++) split_pair(v[u][c], h[c], l[c]);
            const long long at = a32_tile(n, T.r0, kk[u] & ~(E_KC32 - 1)) + a32_pos(rr[u] - T.r0, kk[u] & (E_KC32 - 1));
            *reinterpret_cast<float4 *>(D.A32 + at) = make_float4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<float4 *>(D.A32lo + at) = make_float4(l[0], l[1], l[2], l[3]);
        }
    }
}

// Bring the next tiles of a task into L2 ahead of their copy to shared memory
// (no shared memory used, no completion tracking): more bytes in flight.
__device__ __forceinline__ void l2_prefetch(const void *p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// ----------------------------------------------------------------------------
// producer: fills one stage (header by all 32 lanes, copies by lane 0).
// ----------------------------------------------------------------------------
// Lane 0 waits until the consumers have released the stage of sequence
// number seq's previous use; the outcome is the same in every lane.
__device__ __forceinline__ bool wait_empty(const ProdSmem &M, int seq) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0 && seq >= PSTAGES)
        ok = mbar_wait(M.empty(seq % PSTAGES), ((seq / PSTAGES) - 1) & 1);
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__global__ void __launch_bounds__(PROD_T, 1) eng_prod_kernel(const EngineDev *Ep) {
    const EngineDev &E = *Ep;
    extern __shared__ __align__(16) unsigned char esm[];
    ProdSmem M;
    M.base = esm + ((1024 - (smem_u32(esm) & 1023)) & 1023);             // 1024-aligned tiles
    __shared__ int flag_s;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    eng_count(E);
    if (threadIdx.x == 0) {
        for (int st = 0; st < PSTAGES; st++) {
            mbar_init(M.full(st), 32);
            mbar_init(M.empty(st), PC_W);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(M.mma(b), 1);
            mbar_init(M.conv(b), PC_W);
        }
        fence_mbar_init();
    }
    if (warp == 0) {             // tensor memory for the accumulators (one CTA per SM)
        tmem_alloc(M.tslot(), TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const int par = (E.active[A_TICKS] - 1) & 1;               // list set of this tick
    if (warp == PC_W + 1) {
        // ---------------- MMA warp ----------------
        const unsigned issued = tc_mma_warp(E, M, *M.tslot());
        if (issued > 0 && (threadIdx.x & 31) == 0 && !mbar_wait(M.mma((issued - 1) & 1), ((issued - 1) >> 1) & 1))
            atomicExch(E.active + A_ERR, 1);
        __syncwarp();
    } else if (warp == PC_W) {
        // ---------------- producer warp ----------------
        const int nres = E.active[A_LEN_RES + par];
        const int total = nres + E.active[A_LEN_PROD + par];
        const int *wp = E.work[par], *wr = E.work[par] + E.wres;
        int seq = 0;
        bool fail = false;
        auto push_marker = [&](int kind, int u) -> bool {
            if (!wait_empty(M, seq)) return false;
            StageHdr *H = M.hdr(seq % PSTAGES);
            if (lane == 0) {
                H->kind = kind;
                H->u = u;
                H->flags = 0;
            }
            mbar_arrive(M.full(seq % PSTAGES));
            seq++;
            return true;
        };
        for (;;) {
            int w = 0;
            if (lane == 0) w = atomicAdd(E.active + A_CLAIM_PROD, 1);
            w = __shfl_sync(0xffffffffu, w, 0);
            if (w >= total) break;
            const int u = w < nres ? wr[w] : wp[w - nres];
            const Task T = u < E.n64 ? E.t64[u] : E.t32[u - E.n64];
            if (T.slot < 0) continue;                                   // unused entry
            const int ph = E.st[T.slot].phase;
            if (u >= E.n64 && ph == PH_START) {                         // A split: run by the consumers
                if (!push_marker(SK_GENERIC, u)) { fail = true; break; }
                continue;
            }
            if (u < E.n64) {                                            // refinement residual
                if (ph != PH_RESID) continue;
                const SlotDesc &D = E.desc[T.slot];
                const int n = D.n, sp = D.sp;
                const unsigned tb = (unsigned)(min(E_RB32, n - T.r0) * E_KC32 * 4);   // one tile
                if (lane == 0)
                    for (int i = 1; i <= PREFETCH; i++)
                        if (T.k0 + i * E_KC32 < T.k1) {
                            l2_prefetch(D.A32 + a32_tile(n, T.r0, T.k0 + i * E_KC32), tb);
                            l2_prefetch(D.A32lo + a32_tile(n, T.r0, T.k0 + i * E_KC32), tb);
                        }
                for (int k0 = T.k0; k0 < T.k1 && !fail; k0 += E_KC32) {
                    if (lane == 0 && k0 + (PREFETCH + 1) * E_KC32 < T.k1) {
                        l2_prefetch(D.A32 + a32_tile(n, T.r0, k0 + (PREFETCH + 1) * E_KC32), tb);
                        l2_prefetch(D.A32lo + a32_tile(n, T.r0, k0 + (PREFETCH + 1) * E_KC32), tb);
                    }
                    const unsigned ob = (unsigned)(min(E_KC32, n - k0) * sp * 4);
                    for (int half = 0; half < 2; half++) {              // A32 + Xh, then A32lo + Xl
                        if (!wait_empty(M, seq)) { fail = true; break; }
                        const int st = seq % PSTAGES;
                        if (lane == 0) {
                            StageHdr *H = M.hdr(st);
                            H->kind = SK_RES;
                            H->u = u;
                            H->k0 = k0;
                            H->flags = 0;
                            H->slot = T.slot;
                            H->sp = sp;
                            mbar_arrive_expect_tx(M.full(st), tb + ob);
                            bulk_load_1d(M.tile(st), (half ? D.A32lo : D.A32) + a32_tile(n, T.r0, k0), tb,
                                         M.full(st));
                            bulk_load_1d(M.opr(st, 0), (half ? D.Xl : D.Xh) + (long long)k0 * sp, ob, M.full(st));
                        } else {
                            mbar_arrive(M.full(st));
                        }
                        seq++;
                    }
                }
                if (fail) break;
                continue;
            }
            if (ph != PH_CG && ph != PH_GM) continue;
            const SlotDesc &D = E.desc[T.slot];
            const SlotState &S = E.st[T.slot];
            const int n = D.n, sp = D.sp, it = S.it;
            const long long nsp = (long long)n * sp;
            const float *src, *src2 = nullptr;
            if (ph == PH_CG) {
                src = D.Rf;                                             // P = Rf + beta P'
                src2 = it > 0 ? D.P + ((it + 1) & 1) * nsp : nullptr;
            } else {
                src = D.W + (it & 1) * nsp;                             // V_k = W / h
            }
            const int stp = lane < D.s ? S.colstop[lane] : 1;
            float sc = 0.0f;
            if (!stp) sc = ph == PH_CG ? (float)S.beta[lane] : (float)(1.0 / S.hnorm[lane]);
            const unsigned tb = (unsigned)(min(E_RB32, n - T.r0) * E_KC32 * 4);   // one tile
            if (lane == 0)
                for (int i = 1; i <= PREFETCH; i++)
                    if (T.k0 + i * E_KC32 < T.k1) l2_prefetch(D.A32 + a32_tile(n, T.r0, T.k0 + i * E_KC32), tb);
            for (int k0 = T.k0; k0 < T.k1; k0 += E_KC32) {
                if (lane == 0 && k0 + (PREFETCH + 1) * E_KC32 < T.k1)
                    l2_prefetch(D.A32 + a32_tile(n, T.r0, k0 + (PREFETCH + 1) * E_KC32), tb);
                if (!wait_empty(M, seq)) { fail = true; break; }
                const int st = seq % PSTAGES;
                StageHdr *H = M.hdr(st);
                H->colscale[lane] = sc;
                H->colstop[lane] = stp;
                const int rows = min(E_KC32, n - k0);
                const unsigned ob = (unsigned)(rows * sp * 4);
                if (lane == 0) {
                    H->kind = SK_PROD;
                    H->u = u;
                    H->k0 = k0;
                    H->flags = (k0 == T.k0 ? SF_FIRST : 0) | (k0 + E_KC32 >= T.k1 ? SF_LAST : 0) |
                               (src2 ? SF_SRC2 : 0);
                    H->slot = T.slot;
                    H->sp = sp;
                    mbar_arrive_expect_tx(M.full(st), tb + ob + (src2 ? ob : 0));
                    bulk_load_1d(M.tile(st), D.A32 + a32_tile(n, T.r0, k0), tb, M.full(st));
                    bulk_load_1d(M.opr(st, 0), src + (long long)k0 * sp, ob, M.full(st));
                    if (src2) bulk_load_1d(M.opr(st, 1), src2 + (long long)k0 * sp, ob, M.full(st));
                } else {
                    mbar_arrive(M.full(st));
                }
                seq++;
            }
            if (fail) break;
        }
        if (!fail && !push_marker(SK_STOP, 0)) fail = true;
        if (fail && lane == 0) atomicExch(E.active + A_ERR, 1);     // the consumers time out too
        // never leave with copies in flight
        if (lane == 0)
            for (int i = seq > PSTAGES ? seq - PSTAGES : 0; i < seq; i++)
                if (!mbar_wait(M.full(i % PSTAGES), (i / PSTAGES) & 1)) atomicExch(E.active + A_ERR, 1);
        __syncwarp();
    } else {
        // ---------------- consumer warps ----------------
        int seq = 0;
        __shared__ int fail_s;
        if (threadIdx.x == 0) fail_s = 0;
        named_bar(1, P32_T);
        TcCtx tc{*M.tslot(), 0u, &fail_s};
        for (;;) {
            const int st = seq % PSTAGES;
            const bool ok = mbar_wait(M.full(st), (seq / PSTAGES) & 1);
            if (named_bar_or(1, P32_T, !ok)) {
                if (threadIdx.x == 0) atomicExch(E.active + A_ERR, 1);
                break;
            }
            const StageHdr &H = *M.hdr(st);
            const int kind = H.kind;
            if (kind == SK_STOP) break;
            if (kind == SK_GENERIC) {
                const int u = H.u;
                named_bar(1, P32_T);                                    // header read by all
                release_stage(M, st);
                seq++;
                const Task T = E.t32[u - E.n64];
                convert_task(E.desc[T.slot], T);
                continue;
            }
            if (kind == SK_RES) {
                bool good;
                switch (H.sp) {
                    case 4: good = res_task<4>(E, M, seq, &flag_s); break;
                    case 8: good = res_task<8>(E, M, seq, &flag_s); break;
                    case 16: good = res_task<16>(E, M, seq, &flag_s); break;
                    default: good = res_task<32>(E, M, seq, &flag_s); break;
                }
                if (!good) {
                    if (threadIdx.x == 0) atomicExch(E.active + A_ERR, 1);
                    break;
                }
                continue;
            }
            bool good;
            switch (H.sp) {
                case 4: good = prod_task<4>(E, M, seq, &flag_s); break;
                case 8: good = prod_task<8>(E, M, seq, &flag_s); break;
                case 16:
                    good = E.desc[H.slot].tc ? prod_task_tc<16>(E, M, seq, &flag_s, tc)
                                             : prod_task<16>(E, M, seq, &flag_s);
                    break;
                default:
                    good = E.desc[H.slot].tc ? prod_task_tc<32>(E, M, seq, &flag_s, tc)
                                             : prod_task<32>(E, M, seq, &flag_s);
                    break;
            }
            if (!good) {
                if (threadIdx.x == 0) atomicExch(E.active + A_ERR, 1);
                break;
            }
        }
        tc_send_stop(M, tc);
    }
    // tensor memory is freed once every product has completed: the MMA warp
    // waits (bounded) for its last commit before the whole block meets
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(*M.tslot(), TMEM_COLS);
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
    const int tid = threadIdx.x;
    const int par = (E.active[A_TICKS] - 1) & 1;               // list set of this tick
    const int total = E.active[A_LEN_VEC + par];
    const int *wv = E.work[par] + E.wvec;
    for (int w = claim(E.active + A_CLAIM_VEC, &claim_s); w < total;
         w = claim(E.active + A_CLAIM_VEC, &claim_s)) {
        const int t = wv[w];
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
        if (ph == PH_START && T.r0 == 0)   // split-K tickets of the FP32 product start at zero
            for (int b = tid; b < D.nb32; b += VEC_T) D.ticket[b] = 0;
        __syncthreads();
        // The task's rows form one contiguous stretch of the n x sp block;
        // thread t always sees column t % sp (sp divides VEC_T).  Elements are
        // handled VU at a time, all loads first, so they are in flight
        // together (the stores may alias the loads as far as the compiler
        // knows, so it would not batch them itself).
        constexpr int VU = 4;
        const long long e0 = (long long)T.r0 * sp, e1 = (long long)T.r1 * sp;
        const int c = tid % sp;                                        // fixed for this thread
        const bool live = c < s;
        double part = 0.0;    // PH_START (FP64 b)
        DSV pds{0.0f, 0.0f};  // the other phases: squares of FP32 values, double-single
        if (ph == PH_START) {
            for (long long eb = e0 + tid; eb < e1; eb += VU * VEC_T) {
                double b[VU];
#pragma unroll
                for (int u = 0; u < VU; u++) {
                    const long long e = eb + (long long)u * VEC_T;
                    b[u] = e < e1 ? D.B[e] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < VU; u++) {
                    const long long e = eb + (long long)u * VEC_T;
                    if (e < e1) {
                        D.X[e] = 0.0;
                        D.Xh[e] = 0.0f;
                        D.Xl[e] = 0.0f;
                        D.R[e] = b[u];
                        part += b[u] * b[u];
                    }
                }
            }
        } else if (ph == PH_INIT) {
            const bool on = live && !S.conv[c];
            const double rinv = on ? 1.0 / colv_s[c] : 0.0;   // one division per thread
            const bool gm = D.method != LS_METHOD_CG;
            for (long long eb = e0 + tid; eb < e1; eb += VU * VEC_T) {
                double r[VU];
#pragma unroll
                for (int u = 0; u < VU; u++) {
                    const long long e = eb + (long long)u * VEC_T;
                    r[u] = e < e1 ? D.R[e] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < VU; u++) {
                    const long long e = eb + (long long)u * VEC_T;
                    if (e < e1) {
                        const float f = on ? (float)(r[u] * rinv) : 0.0f;
                        D.Rf[e] = f;
                        D.Z[e] = 0.0f;
                        if (gm) D.W[e] = f;                             // W buffer 0
                        ds_fma(f, 0.0f, DSV{f, 0.0f}, pds);
                    }
                }
            }
        } else if (ph == PH_CG) {
            const float al = (float)colv_s[c];
            const float *p = D.P + (it & 1) * nsp;
            for (long long eb = e0 + tid; eb < e1; eb += VU * VEC_T) {
                float z[VU], pv[VU], q[VU], r[VU];
#pragma unroll
                for (int u = 0; u < VU; u++) {
                    const long long e = eb + (long long)u * VEC_T;
                    const bool in = e < e1;
                    z[u] = in ? D.Z[e] : 0.0f;
                    pv[u] = in ? __ldcg(p + e) : 0.0f;                 // written by other CTAs
                    q[u] = in ? __ldcg(D.Q + e) : 0.0f;
                    r[u] = in ? D.Rf[e] : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < VU; u++) {
                    const long long e = eb + (long long)u * VEC_T;
                    if (e < e1) {
                        D.Z[e] = fmaf(al, pv[u], z[u]);
                        const float rv = fmaf(-al, q[u], r[u]);
                        D.Rf[e] = rv;
                        ds_fma(rv, 0.0f, DSV{rv, 0.0f}, pds);
                    }
                }
            }
        } else if (ph == PH_GM) {
            float *w = D.W + ((it + 1) & 1) * nsp;
            for (long long eb = e0 + tid; eb < e1; eb += VU * VEC_T) {
                DSV wv[VU];   // w - sum_q h_q v_q in double-single (about 48 bits)
#pragma unroll
                for (int u = 0; u < VU; u++) {
                    const long long e = eb + (long long)u * VEC_T;
                    wv[u] = DSV{e < e1 ? __ldcg(w + e) : 0.0f, 0.0f};
                }
                for (int q = 0; q <= it; q++) {
                    const float *vq = D.V + (long long)q * nsp;
                    float hh, hl;
                    split_pair(-hsm[q][c], hh, hl);
#pragma unroll
                    for (int u = 0; u < VU; u++) {
                        const long long e = eb + (long long)u * VEC_T;
                        if (e < e1) ds_fma(hh, hl, DSV{__ldcg(vq + e), 0.0f}, wv[u]);
                    }
                }
#pragma unroll
                for (int u = 0; u < VU; u++) {
                    const long long e = eb + (long long)u * VEC_T;
                    if (e < e1) {
                        const float wf = __fadd_rn(wv[u].h, wv[u].l);
                        w[e] = wf;
                        ds_fma(wf, 0.0f, DSV{wf, 0.0f}, pds);
                    }
                }
            }
        } else if (ph == PH_UPDATE) {
            const double rn = colv_s[c];
            if (live && rn != 0.0) {
                const bool cgm = D.method == LS_METHOD_CG;
                const int kj = cgm ? 0 : (int)S.alpha[c];
                for (long long eb = e0 + tid; eb < e1; eb += VU * VEC_T) {
                    double x[VU];
                    DSV d[VU];   // the correction direction in double-single
#pragma unroll
                    for (int u = 0; u < VU; u++) {
                        const long long e = eb + (long long)u * VEC_T;
                        const bool in = e < e1;
                        x[u] = in ? D.X[e] : 0.0;
                        d[u] = DSV{(in && cgm) ? D.Z[e] : 0.0f, 0.0f};
                    }
                    for (int q = 0; q < kj; q++) {
                        const float *vq = D.V + (long long)q * nsp;
                        float yh, yl;
                        split_pair(S.yv[c][q], yh, yl);
#pragma unroll
                        for (int u = 0; u < VU; u++) {
                            const long long e = eb + (long long)u * VEC_T;
                            if (e < e1) ds_fma(yh, yl, DSV{vq[e], 0.0f}, d[u]);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < VU; u++) {
                        const long long e = eb + (long long)u * VEC_T;
                        if (e < e1) {
                            const double xn = x[u] + rn * to_double(d[u]);
                            float xh, xl;
                            split_pair(xn, xh, xl);
                            D.X[e] = xn;
                            D.Xh[e] = xh;
                            D.Xl[e] = xl;
                        }
                    }
                }
            }
        }
        // partial column sums over this task's rows (fixed order)
        if (ph != PH_UPDATE) {
            psum[tid] = part + to_double(pds);
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

// Columns [c0, c0 + k) of a slot's X (row-major n x sp) -> a column-major
// destination (ldx), one item per (slot, column range).
__global__ void eng_finish_kernel(const EngineDev *Ep, double *const *Xdst, const long long *ldx,
                                  const int *slot, const int *c0, const int *k, int count) {
    const EngineDev &E = *Ep;
    for (int q = blockIdx.y; q < count; q += gridDim.y) {
        const SlotDesc &D = E.desc[slot[q]];
        double *x = Xdst[q];
        const int cb = c0[q];
        const long long total = (long long)D.n * k[q];
        for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
             e += (long long)gridDim.x * blockDim.x) {
            const int c = (int)(e / D.n), i = (int)(e % D.n);
            x[(long long)c * ldx[q] + i] = D.X[(long long)i * D.sp + cb + c];
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
    K.prod_threads = PROD_T;
    K.vec_threads = VEC_T;
    K.prod_smem = PROD_SMEM;
    return K;
}

}  // namespace lsi
