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
constexpr int E_KS32 = 512;                // default columns of A per FP32 product task (split K)
constexpr int E_KS32_MIN = 256;            // smallest task width the tuner may choose
constexpr int E_KC32 = 32;                 // k per shared-memory chunk of the FP32 product
constexpr int E_VEL = 8192;                // elements of the n x sp block per vector task
constexpr int E_PS = E_MAXM + 2;           // partial-dot slots per FP32 row block

// slot phases: what eng_prod / eng_vec do in the current tick
enum : int {
    PH_FREE = 0,
    PH_START = 1,     // prod: A = A32 + A32lo; vec: X = 0, R = B, partial ||B||^2
    PH_RESID = 2,     // prod (FP64): R = B - A X, partial ||R||^2
    PH_INIT = 3,      // vec: Rf = R / ||R||, Z = 0 (GMRES: W0 = Rf), partial ||Rf||^2
    PH_CG = 4,        // prod: P = Rf + beta P', Q = Ahat P, partial P.Q; vec: Z, Rf, ||Rf||^2
    PH_GM = 5,        // prod: V_k = W / h, W' = Ahat V_k, partial V_i.W'; vec: W' -= V h, ||W'||^2
    PH_UPDATE = 6,    // vec: X += ||R|| (Z or V y)
    PH_DONE = 7,
    PH_ADMIT = 8,     // just admitted: eng_red turns it into START (nothing to reduce yet)
};

// Columns of A per refinement-residual task (256 rows): the double-single
// arithmetic costs 12 FP32 operations per term, so about the same time per
// task for every width.
__host__ __device__ constexpr int ks64(int sp) { return 4096 / (sp > 0 ? sp : 32); }

// Rows per vector task: the same number of elements for any width.
__host__ __device__ constexpr int rbv(int sp) { return E_VEL / (sp > 0 ? sp : 32); }

// Storage of a slot's FP32 matrices (A32, A32lo) on the device: tile-major,
// in the order eng_prod streams them.  Row block b (rows 256 b .. 256 b +
// nr - 1, nr = min(256, n - 256 b)) holds ceil(n / 32) column tiles of nr x
// 32 floats, each contiguous; inside a tile, row r is 128 bytes whose
// 16-byte pieces are stored XOR-swizzled by r & 7 (piece j at position
// j ^ (r & 7)), which is the image the tensor core and the FP32 path expect
// in shared memory, so one tile is one contiguous bulk copy.  Columns past
// n are stored as zeros; the last row block stores only its nr rows.
__host__ __device__ inline long long a32_ncols(int n) { return (long long)(n + E_KC32 - 1) / E_KC32 * E_KC32; }
// Offset (floats) of the tile holding rows r0 .. (r0 a multiple of 256) and
// columns k0 .. k0 + 31 (k0 a multiple of 32).
__host__ __device__ inline long long a32_tile(int n, int r0, int k0) {
    const int nr = n - r0 < E_RB32 ? n - r0 : E_RB32;
    return (long long)r0 * a32_ncols(n) + (long long)(k0 / E_KC32) * nr * E_KC32;
}
// Position of element (r, k) of a tile (r < 256, k < 32).
__host__ __device__ inline int a32_pos(int r, int k) { return r * E_KC32 + ((((k >> 2) ^ (r & 7))) << 2) + (k & 3); }

// Work decomposition of one slot of size n and padded width sp (it depends on
// nothing else, so a slot's reduction order never depends on its neighbours).
struct SlotTasks {
    int rb32;        // FP32 row blocks (E_RB32 rows each)
    int kc32;        // K chunks per row block (ks32(sp) columns of A each)
    int t32;         // FP32 product tasks = rb32 * kc32
    int kc64;        // K chunks per row block of the residual (ks64(sp) columns each)
    int t64;         // residual tasks = rb32 * kc64
    int tv;          // vector tasks (rbv(sp) rows each)
};
// ks32: columns of A per FP32 product task (a multiple of E_KC32, chosen per
// slot class by the tuner).
__host__ __device__ inline SlotTasks slot_tasks(int n, int sp, int ks32) {
    SlotTasks t;
    n = n > 0 ? n : 0;
    t.rb32 = (n + E_RB32 - 1) / E_RB32;
    t.kc32 = n > 0 ? (n + ks32 - 1) / ks32 : 0;
    t.t32 = t.rb32 * t.kc32;
    t.kc64 = n > 0 ? (n + ks64(sp) - 1) / ks64(sp) : 0;
    t.t64 = t.rb32 * t.kc64;
    t.tv = (n + rbv(sp) - 1) / rbv(sp);
    return t;
}

struct SlotDesc {                // written at admission
    int n, s;                    // size and right-hand sides (s <= 32)
    int sp;                      // row stride of the n x sp row-major blocks: 4, 8, 16 or 32
    int method;                  // LS_METHOD_CG / LS_METHOD_GMRES
    int m;                       // GMRES restart (<= E_MAXM)
    int ks32;                    // columns of A per FP32 product task
    int tc;                      // FP32 products on the tensor cores (sp = 16 or 32 only)
    int inner_iters;             // inner iterations per refinement step
    int max_outer;               // refinement steps
    float inner_tol;             // inner relative tolerance
    double rtol;                 // outer (FP64) relative tolerance
    const double *A64;           // FP64 A (row-major)
    long long lda64;
    float *A32;                  // fp32(A), tile-major (a32_tile): the inner solves' matrix
    float *A32lo;                // fp32(A - fp32(A)), same layout: with A32, A to about 48 bits
    long long ld32;              // padded column count a32_ncols(n)
    double *X, *B, *R;           // n x sp row-major FP64
    float *Xh, *Xl;              // X = Xh + Xl (fp32 pair), refreshed with X
    float *Yk;                   // split-K partial products: kc32 x n x sp (kc32 > 1)
    double *Rk;                  // split-K partial residual products: kc64 x n x sp (kc64 > 1)
    int *ticket;                 // per FP32 row block: K-chunk tasks finished this tick
    float *Rf, *Z, *Q;           // n x sp row-major FP32
    float *P;                    // CG: two n x sp buffers (current / previous direction)
    float *W;                    // GMRES: two n x sp buffers (unnormalised new vector)
    float *V;                    // GMRES: (m + 1) normalised n x sp blocks
    int t32, n32;                // FP32 product tasks [t32, t32 + n32)
    int b32, nb32;               // row blocks (partial-dot / residual-norm rows) [b32, b32 + nb32)
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
    double *part64;              // [row block][32]
    double *partv;               // [taskv][32]
    int *order;                  // eng_red block b handles slot order[b] (costliest first)
    int *work[2];                // per tick parity: runnable FP32 product tasks, then the
                                 // residual tasks at work[p] + wres, the vector tasks at
                                 // work[p] + wvec
    int wres, wvec;              // offsets of the residual and vector lists in work[p]
    int *active;                 // engine counters, see the A_* indices
    int tick_limit;              // ticks per graph launch (loop control)
    int host_loop;               // 1: no graph; eng_red writes the loop condition to active[4]
    unsigned long long *launches;
};

// indices into EngineDev::active
enum : int {
    A_COUNT = 0,      // slots still active after this tick's eng_red
    A_TICKET = 1,     // eng_red blocks finished
    A_LAST = 2,       // active slots seen by the last loop test
    A_TICKS = 3,      // ticks run by this launch
    A_GO = 4,         // host-loop mode: the loop condition
    A_CLAIM_PROD = 5, // eng_prod task claims this tick
    A_CLAIM_VEC = 6,  // eng_vec task claims this tick
    A_ERR = 7,        // a bounded wait in eng_prod gave up (the launch's results are void)
    A_LEN_PROD = 8,   // [8 + parity]: runnable eng_prod tasks listed by eng_red
    A_LEN_VEC = 10,   // [10 + parity]: runnable eng_vec tasks
    A_LEN_RES = 12,   // [12 + parity]: runnable refinement-residual tasks (claimed first)
    A_SIZE = 16
};

struct EngineKernels {
    void *red, *prod, *vec, *admit, *finish;
    int prod_threads, vec_threads, red_threads;
    size_t prod_smem;
};
EngineKernels engine_kernels();

}  // namespace lsi
