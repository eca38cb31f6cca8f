// ls_engine.h -- the batched / served solve engine: many independent dense
// systems (each with up to 32 right-hand sides) advance together on the
// device, one "tick" at a time.  Every tick runs three kernels over all
// resident slots:
//   eng_red   per slot: finish the reductions of the previous tick, run the
//             scalar recurrences (CG alpha/beta, GMRES Givens and back-solve),
//             choose the slot's next phase;
//   eng_prod  block products, both kinds claimed from one queue:
//             R = B - A X to FP64 accuracy (refinement residual), evaluated
//             on the FP32 pipe with error-free transformations on the split
//             A = A32 + A32lo, X = Xh + Xl (GB300 runs FP32 64x faster than
//             FP64), or Y = Ahat P in FP32 on Ahat = A32 (inner Krylov step),
//             split along K with a fixed-order fix-up, fused partial dots;
//   eng_vec   vector updates of each slot's rows, with partial dot products.
// Each slot follows its own phase sequence (refinement residual -> inner
// CG or GMRES(m) steps on every unconverged column -> correction of X),
// so slots can be admitted and retired between any two ticks (continuous
// batching).  A slot's arithmetic and reduction order depend only on its own
// n and s, never on the other slots, so a result is bitwise the same alone
// or in a mix.
#pragma once

#include <cuda_runtime.h>

#include "ls_internal.h"

namespace lsi {

constexpr int E_MAXS = LS_BATCH_MAX_RHS;   // right-hand sides per slot (32)
constexpr int E_MAXM = 32;                 // GMRES restart length in the engine
constexpr int E_RB32 = 256;                // rows per FP32 product task (any width)
constexpr int E_KS32 = 512;                // columns of A per FP32 product task (split K)
constexpr int E_KC32 = 32;                 // k per shared-memory chunk of the FP32 product
constexpr int E_RB64 = 8;                  // rows per refinement-residual task
constexpr int E_RBV = 256;                 // rows per vector task
constexpr int E_PS = E_MAXM + 2;           // partial-dot slots per FP32 row block

// slot phases: what eng_prod / eng_vec do in the current tick
enum : int {
    PH_FREE = 0,
    PH_START = 1,     // vec: X = 0, R = B, partial ||B||^2
    PH_RESID = 2,     // prod (FP64): R = B - A X, partial ||R||^2
    PH_INIT = 3,      // vec: Rf = R / ||R||, Z = 0 (GMRES: W0 = Rf), partial ||Rf||^2
    PH_CG = 4,        // prod: P = Rf + beta P', Q = Ahat P, partial P.Q; vec: Z, Rf, ||Rf||^2
    PH_GM = 5,        // prod: V_k = W / h, W' = Ahat V_k, partial V_i.W'; vec: W' -= V h, ||W'||^2
    PH_UPDATE = 6,    // vec: X += ||R|| (Z or V y)
    PH_DONE = 7,
    PH_ADMIT = 8,     // just admitted: eng_red turns it into START (nothing to reduce yet)
};

// Work decomposition of one slot of size n (the same for any s, so a slot's
// reduction order never depends on its neighbours).
struct SlotTasks {
    int rb32;        // FP32 row blocks (E_RB32 rows each)
    int kc32;        // K chunks per row block (E_KS32 columns of A each)
    int t32;         // FP32 product tasks = rb32 * kc32
    int t64;         // residual tasks (E_RB64 rows each)
    int tv;          // vector tasks (E_RBV rows each)
};
__host__ __device__ inline SlotTasks slot_tasks(int n) {
    SlotTasks t;
    n = n > 0 ? n : 0;
    t.rb32 = (n + E_RB32 - 1) / E_RB32;
    t.kc32 = n > 0 ? (n + E_KS32 - 1) / E_KS32 : 0;
    t.t32 = t.rb32 * t.kc32;
    t.t64 = (n + E_RB64 - 1) / E_RB64;
    t.tv = (n + E_RBV - 1) / E_RBV;
    return t;
}

struct SlotDesc {                // written at admission
    int n, s;                    // size and right-hand sides (s <= 32)
    int sp;                      // row stride of the n x sp row-major blocks: 4, 8, 16 or 32
    int method;                  // LS_METHOD_CG / LS_METHOD_GMRES
    int m;                       // GMRES restart (<= E_MAXM)
    int inner_iters;             // inner iterations per refinement step
    int max_outer;               // refinement steps
    float inner_tol;             // inner relative tolerance
    double rtol;                 // outer (FP64) relative tolerance
    const double *A64;           // FP64 A (row-major)
    long long lda64;
    float *A32;                  // fp32(A) (row-major, ld32): the inner solves' matrix
    float *A32lo;                // fp32(A - fp32(A)): with A32, A to about 48 bits
    long long ld32;
    double *X, *B, *R;           // n x sp row-major FP64
    float *Xh, *Xl;              // X = Xh + Xl (fp32 pair), refreshed with X
    float *Yk;                   // split-K partial products: kc32 x n x sp (kc32 > 1)
    int *ticket;                 // per FP32 row block: K-chunk tasks finished this tick
    float *Rf, *Z, *Q;           // n x sp row-major FP32
    float *P;                    // CG: two n x sp buffers (current / previous direction)
    float *W;                    // GMRES: two n x sp buffers (unnormalised new vector)
    float *V;                    // GMRES: (m + 1) normalised n x sp blocks
    int t32, n32;                // FP32 product tasks [t32, t32 + n32)
    int b32, nb32;               // FP32 row blocks (partial-dot rows) [b32, b32 + nb32)
    int t64, n64;                // residual tasks
    int tv, nv;                  // vector tasks
};

struct SlotState {               // mutable, per slot
    int phase;
    int it;                      // inner iteration (CG) or Arnoldi step k (GMRES)
    int outer;                   // refinement residuals computed
    int status;                  // LS_* once done
    int err;
    int inner_total;             // inner iterations over all refinement steps
    int ticks;
    int pad_;
    double bnorm[E_MAXS], rn[E_MAXS];
    double rho[E_MAXS], rho0[E_MAXS], beta[E_MAXS], alpha[E_MAXS];
    double hnorm[E_MAXS];        // GMRES: normaliser of the pending vector
    double gbeta[E_MAXS];        // GMRES: ||Rf|| at the start of the cycle
    double yv[E_MAXS][E_MAXM];   // GMRES: least-squares solution, per column
    int colstop[E_MAXS];         // inner loop finished for this column
    int conv[E_MAXS];            // outer tolerance met
};

struct SlotGm {                  // GMRES small dense state, per slot and column
    double H[E_MAXS][(E_MAXM + 1) * E_MAXM];   // rotated Hessenberg, column-major
    double cs[E_MAXS][E_MAXM], sn[E_MAXS][E_MAXM];
    double g[E_MAXS][E_MAXM + 1];
};

struct Task {
    int slot;
    int r0, r1;                  // rows [r0, r1)
    int k0, k1;                  // FP32 product: columns of A [k0, k1)
    int kc;                      // FP32 product: K chunk index (0 .. kc32 - 1)
    int rb;                      // FP32 product: global row-block index (partial dots)
    int pad_;
};

struct EngineDev {               // pointers handed to every engine kernel
    SlotDesc *desc;
    SlotState *st;
    SlotGm *gm;
    int nslots;
    Task *t32, *t64, *tv;        // task tables
    int n32, n64, nv;            // table sizes
    double *part32;              // [row block][E_PS][32]
    double *part64;              // [task64][32]
    double *partv;               // [taskv][32]
    int *active;                 // [0] count, [1] ticket, [2] last count, [3] ticks run
    int tick_limit;              // ticks per graph launch (loop control)
    int host_loop;               // 1: no graph; eng_red writes the loop condition to active[4]
    unsigned long long *launches;
};

struct EngineKernels {
    void *red, *prod, *vec, *admit, *finish;
    int prod_threads, vec_threads, red_threads;
    size_t prod_smem;
};
EngineKernels engine_kernels();

}  // namespace lsi
