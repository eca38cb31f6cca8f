// ls_internal.h -- structures shared by the host drivers and the kernels.
#pragma once

#include <cuda.h>            // CUtensorMap (type only; the driver is reached by entry point)
#include <cuda_runtime.h>
#include <stdint.h>

#include "ls.h"

namespace lsi {

// storage formats of A
// DT_DS: an FP64 matrix split once into an FP32 pair A = hi + lo (hi = fp32(A),
// lo = fp32(A - hi), about 48 significant bits), multiplied in double-single
// arithmetic on the FP32 pipe; vectors and results stay FP64.
enum DType : int { DT_F64 = 0, DT_BF16 = 1, DT_FP8 = 2, DT_F32 = 3, DT_DS = 4 };

// ---- GEMV geometry ----------------------------------------------------------
// A tile of TR rows x TC columns is one TMA box.  Consumer warps form a
// WR x WC grid over the tile: each lane holds VEC consecutive columns and
// RW rows (TR = WR * RW, TC = WC * 32 * VEC).
constexpr int GEMV_CONSUMER_WARPS = 4;
constexpr int GEMV_THREADS = (GEMV_CONSUMER_WARPS + 1) * 32;
constexpr int GEMV_STAGES = 6;
constexpr int GEMV_MAX_TR = 64;
constexpr int MAX_GRID = 2048;     // upper bound on CTAs of any persistent launch

// ---- device-resident matrix descriptor ---------------------------------------
struct alignas(128) MatDesc {
    CUtensorMap tmap;        // 2-D tiled TMA map of A (valid when use_tma)
    CUtensorMap tmap_lo;     // DT_DS: the same for the low part
    const void *ptr;         // A (row-major); DT_DS: the high part
    const void *ptr_lo;      // DT_DS: the low part (same layout)
    const float *scale;      // FP8 row scales (else nullptr)
    long long lda;           // elements
    int rows, cols;
    int dtype;
    int use_tma;
    int pad_[8];
};

// error bits
enum : int { ERRB_TIMEOUT = 1, ERRB_NAN = 2 };

// stop reasons / status written by the kernels (same values as LS_*)
// State lives in device memory; one per context.
constexpr int LS_COND_SLOTS = 4;

struct State {
    // CG / common
    double rho;          // r.r
    double alpha, beta;
    double omega;        // BiCGSTAB stabilisation step
    double pq;           // p.Ap
    double bnorm;        // ||b||
    double tol_abs;      // rtol * ||b||
    double rnorm;        // recursive residual norm
    double true_rnorm;   // ||b - A x|| at the last check
    double dot;          // scratch result of FIN_STORE
    // GMRES
    double est;          // |g_{k+1}|
    double wnorm0;       // ||A v_k||^2 before orthogonalisation
    // mixed precision (inner FP32 loop, outer FP64 loop)
    double in_rho, in_alpha, in_pq, in_rho0;
    double prn;          // p.r partial total (FCG)
    double outer_rn;     // ||r|| at the start of the outer step
    int iter;            // method matvecs (inner ones for the mixed path)
    int max_iter;
    int status;          // 0 running/converged, LS_NOT_CONVERGED, LS_BREAKDOWN
    int err;             // ERRB_* bits
    int conv;            // recursive residual passed the test
    int k;               // GMRES: Arnoldi steps in the current cycle
    int m;               // GMRES restart length
    int reorth;          // GMRES: 1 = always two passes
    int total;           // GMRES: Arnoldi steps over all cycles
    int cycles;          // GMRES cycles / mixed outer steps
    int in_iter, in_max; // inner loop counters
    int outer, max_outer;
    int nstored;         // FCG directions stored
    int in_stop;
    int skip;            // BiCGSTAB: the rest of the step is skipped (s passed, or stop)
    float in_tol2;       // inner (rtol^2 * rho0), <0 = fixed count
    int launches_lo;     // kernels executed (low word; counted by block 0)
    int hostloop;        // 1: loop conditions go to cond[] instead of graph handles
    unsigned cond[LS_COND_SLOTS];
    unsigned long long launches;
};

// GMRES small dense state (device)
struct GmresSmall {
    double H[(LS_MAX_RESTART + 1) * LS_MAX_RESTART];  // rotated Hessenberg, column-major
    double cs[LS_MAX_RESTART], sn[LS_MAX_RESTART];
    double g[LS_MAX_RESTART + 1];
    double y[LS_MAX_RESTART];
    double h[LS_MAX_RESTART + 1];                     // current column (projection)
};

// ---- per-launch scratch of the persistent GEMV --------------------------------
struct GemvScratch {
    unsigned ticket;                                 // last-CTA detection (self-resetting)
    unsigned pad_[31];
    unsigned bticket[MAX_GRID];                      // per shared row tile (self-resetting)
    double cta_dot[MAX_GRID];                        // per-CTA dot contributions
    double fixdot[MAX_GRID];                         // dot of shared row tiles, by first CTA
    double fix[MAX_GRID * 2 * GEMV_MAX_TR];          // partial row sums of shared row tiles
};

// epilogues: what is done with a finished row sum s_i
enum : int {
    EPI_STORE = 0,      // y_i = s_i
    EPI_DOT = 1,        // y_i = s_i; dot += z_i y_i
    EPI_RESID = 2,      // y_i = b_i - s_i; dot += y_i^2
    EPI_NRM = 3,        // y_i = s_i; dot += y_i^2
    EPI_JACOBI = 4,     // r_i = b_i - s_i; y_i = x_i + z_i r_i (z = D^-1); dot += r_i^2
};
// finalisers run by the last CTA on the reduced dot
enum : int {
    FIN_STORE = 0,      // st->dot = dot (and *dot_out if given)
    FIN_CG_ALPHA = 1,   // pq = dot; alpha = rho / pq; breakdown if !(pq > 0)
    FIN_TRUE_RES = 2,   // true_rnorm = sqrt(dot)
    FIN_WNORM0 = 3,     // wnorm0 = dot
    FIN_INNER_ALPHA = 4,// in_pq = dot; in_alpha = in_rho / in_pq (inner stop on breakdown)
    FIN_FCG_D = 5,      // pq = dot (p.Ap of the outer direction)
    FIN_BS_ALPHA = 6,   // BiCGSTAB: pq = r^.v; alpha = rho / pq; breakdown if pq = 0
    FIN_JACOBI = 7,     // rnorm = ||b - A x||; iter++; stop test -> skip
};

struct GemvArgs {
    const void *x;       // input vector (double for F64, float otherwise)
    void *y;             // output vector (same type as x)
    const int *kptr;     // if set: x += (*kptr) * kstride, y += (*kptr + kyoff) * kstride
    long long kstride;   // (elements) -- lets one graph node walk a stored basis
    int kyoff;           // GMRES: 1 (w = A v_k goes to column k+1); FCG: 0
    int z_is_x;          // EPI_DOT with z = x (after the k offset)
    const double *b;     // EPI_RESID, EPI_JACOBI
    const void *z;       // EPI_DOT; EPI_JACOBI: 1 / a_ii
    double *dot_out;     // optional copy of the final dot
    State *st;
    GemvScratch *scr;
    int epi, fin;
};

// ---- launchers (k_gemv.cu) -------------------------------------------------------
struct GemvLaunch {
    void *func;          // kernel entry
    int grid, block;
    size_t smem;
};
// Choose the kernel for a matrix (TMA or plain-load variant) and epilogue.
GemvLaunch gemv_plan(int dtype, bool use_tma, int epi, int num_sms);
// Raise a kernel's dynamic shared-memory limit to at least smem bytes on the
// current device.  The attribute is per device: it is set again only for a
// new (kernel, device) pair or a larger size.  Safe from several host threads.
cudaError_t set_smem_limit(const void *func, size_t smem);
cudaError_t gemv_launch(const GemvLaunch &L, const MatDesc *dA, const GemvArgs &a,
                        cudaStream_t s);
// Fill the TMA map of a matrix descriptor (host side); returns false when the
// layout cannot be streamed by TMA (alignment), in which case use_tma = 0.
bool make_tensor_map(MatDesc *h, int dtype, const void *ptr, int rows, int cols, long long lda);
// DT_DS descriptor of the FP32 pair (hi, lo), both row-major with leading dimension ld.
bool make_tensor_map_ds(MatDesc *h, const float *hi, const float *lo, int rows, int cols, long long ld);
// hi = fp32(A), lo = fp32(A - hi), row-major with leading dimension ld (a multiple of 4).
cudaError_t split_f64_launch(int rows, int cols, const double *A, long long lda, float *hi, float *lo,
                             long long ld, int num_sms, cudaStream_t s);
// FP32 row-major rows x cols (leading dimension ld) read in box_rows x box_cols
// tiles with the 128-byte swizzle; `map` is 128 bytes, 64-byte aligned.
bool encode_f32_tile_map_sw128(void *map, const float *ptr, int rows, int cols, long long ld,
                               int box_cols, int box_rows);
int gemv_tile_rows(int dtype);
cudaError_t quantize_launch(int dtype, int rows, int cols, const double *A, long long lda,
                            void *Q, long long ldq, float *scale, int num_sms, cudaStream_t s);

// ---- FP64 solver vectors (workspace) ---------------------------------------------
struct GridBar;
struct Vecs {
    int n;
    double *x, *b, *r, *p, *q;
    double *rh, *vv, *s, *t;   // BiCGSTAB: shadow residual r^, v = A p, s, t = A s
    double *V;           // GMRES basis, column-major, column stride ldv
    long long ldv;
    double *part;        // cooperative partial sums, [slot][block]
    GridBar *bar;
    State *st;
    GmresSmall *gm;
    double rtol;
};
constexpr int PART_SLOTS = LS_MAX_RESTART + 4;

// ---- mixed-precision vectors (workspace) -------------------------------------------
struct MixVecs {
    int n;
    int mode;            // LS_REFINE_FCG or LS_REFINE_IR
    double *x, *b, *r, *q;
    double *P, *W;       // FCG directions and A * directions, column stride ldp
    long long ldp;
    double *dvals;       // p_j . A p_j
    float *rf, *zf, *pf, *qf;
    double *part;
    GridBar *bar;
    State *st;
    double rtol;
};

struct MixedKernels {
    void *mx_init, *in_init, *in_update, *fcg_project, *fcg_update, *mx_check, *ir_start,
        *ir_update;
};
MixedKernels mixed_kernels();

// ---- Krylov launchers (k_krylov.cu) -----------------------------------------------
// ---- Gauss-Seidel triangular solve (k_gs.cu) -----------------------------------------
struct GsArgs {
    int n;
    const double *r;         // b - A x(k), from the residual GEMV
    double *x;               // x(k) -> x(k+1) = x(k) + d
    float2 *delta, *u;       // d, and u_I = T_I^-1 (r_I - sum_{j < I - W} A_Ij d_j), as FP32 pairs
    const CUtensorMap *tmaps;// device: A hi, A lo (n x n), T hi, T lo (nblk*64 x 64), 32 x 64 boxes
    const float *panel;      // the chain's tiles per block, in its read order (gs_panel_kernel)
    unsigned *flagD, *flagU; // per row block: d_I / u_I published (value = sweep number)
    GridBar *bar;            // the final x += d waits for the whole chain
    State *st;
};
struct GsKernels {
    void *tinv, *trsv, *panel;
    int tinv_block, trsv_block, blk, panel_block, panel_tiles_per_block, panel_tile_floats;
    int max_owned;           // row blocks one helper CTA can own
    size_t trsv_smem, panel_smem;
};
GsKernels gs_kernels();
// The four tensor maps of GsArgs::tmaps (maps: 4 x 128 bytes, 64-byte aligned).
bool gs_encode_maps(void *maps, const float *Ahi, const float *Alo, int n, long long ld, const float *Thi,
                    const float *Tlo, int nblk);

// ---- block CG (k_bcg.cu) ------------------------------------------------------------------
constexpr int BCG_MAX_S = 16;
struct BcgSmall {                 // s x s matrices, column-major, leading dimension s
    double rho[BCG_MAX_S * BCG_MAX_S];     // R^T R
    double L[BCG_MAX_S * BCG_MAX_S];       // its Cholesky factor (lower triangle)
    double alpha[BCG_MAX_S * BCG_MAX_S], beta[BCG_MAX_S * BCG_MAX_S];
    double bn[BCG_MAX_S];                  // ||B_j||
    double r2[BCG_MAX_S];                  // ||B_j - A X_j||^2 from the residual GEMVs
    int ok, update_p;
    // deflating form: leading dimension BCG_MAX_S for every small matrix
    double T[BCG_MAX_S * BCG_MAX_S];       // P = W T (the current orthogonalization pass)
    double Lg[BCG_MAX_S * BCG_MAX_S];      // Cholesky factor of gamma = P^T Q (rank x rank)
    double w2[BCG_MAX_S];                  // ||W_j||^2 of the block being orthogonalized
    int rank;                              // orthonormal directions in P (its first columns)
};
struct BcgVecs {
    int n, s;
    long long ld;                 // column stride of the n x s blocks
    double *X, *R, *P, *Q;
    const double *B;
    double *part;                 // [CTA][BCG_MAX_S^2] partial Gram matrices
    double *partb;                // [CTA][BCG_MAX_S^2] a second set (two Gram matrices at once)
    double *part2;                // [CTA][BCG_MAX_S] partial ||B_j||^2
    BcgSmall *sm;
    GridBar *bar;
    State *st;
    double rtol;
};
struct BcgKernels {
    void *init, *step, *check;             // O'Leary's form
    void *dinit, *dstep, *dcheck;          // the deflating form (orthonormal directions of full rank)
    int block;
};
BcgKernels bcg_kernels();

// ---- LU with partial pivoting (k_lu.cu) --------------------------------------------------
struct LuArgs {
    int n;
    double *W;                    // [A | b], n x (n + 1), row-major, leading dimension ld
    long long ld;
    int *ipiv;                    // the row swapped with row k at step k
    double *x;                    // the solution
    double *cand_v;               // [CTA] pivot candidates: |value| and row
    int *cand_i;
    GridBar *bar;
    State *st;
};
struct LuKernels {
    void *factor, *backsolve;     // factor takes (LuArgs, k0, k1): one panel's steps
    void *laswp, *u12, *trail;    // (LuArgs, k0, nb), (LuArgs, k0, nb), (LuArgs, k0)
    int block, nb, tile, u12_block;
};
LuKernels lu_kernels();

// ---- Cholesky (k_chol.cu) --------------------------------------------------------------------
struct CholArgs {
    int n;
    double *W;                    // [A; b^T], (n + 1) x n, row-major, leading dimension ld (lower part used)
    long long ld;
    double *Lp;                   // the current panel's l's, (n + 1) x 32, row-major
    double *y;                    // back substitution: y, overwritten by the updated right sides
    double *x;                    // the solution
    GridBar *bar;
    State *st;                    // status LS_BREAKDOWN (iter = the failing step) on a pivot <= 0
};
struct CholKernels {
    void *panel, *trail, *backsolve, *zero_upper;   // panel and trail take (CholArgs, k0, k1 / nb)
    int block, nb, tile;
};
CholKernels chol_kernels();
size_t chol_workspace_bytes(int n, bool a_on_device);

// ---- self-test of the bounded waits (k_selftest.cu) -------------------------------------------
cudaError_t selftest_launch(int which, GridBar *bar, State *st, cudaStream_t s);

// ---- block GMRES (k_bgmres.cu) -----------------------------------------------------------
constexpr int BGM_MAX_S = 16;
constexpr int BGM_MAX_MS = 256;       // m * s at most
enum : int { BGF_CHOL = 0, BGF_NROT = 1, BGF_LUCKY = 2, BGF_COUNT = 4 };
struct BgmVecs {
    int n, s, m;
    long long ld;                 // column stride of V, W, X, B
    double *V;                    // basis, n x (m+1)s
    double *W;                    // A V_j, n x s
    double *X;
    const double *B;
    double *H;                    // rotated band Hessenberg, (m+1)s x ms, leading dimension (m+1)s
    double *G;                    // rotated right-hand side, (m+1)s x s
    double *Y;                    // ms x s
    double *cs, *sn;              // the cycle's rotations (ms * s at most)
    int *rrow;
    double *Hc;                   // reduced Gram coefficients, (m+1)s x s at most
    double *Lm;                   // s x s Cholesky factor of the last CholQR pass
    double *part;                 // [CTA][part_stride] partial Gram matrices
    long long part_stride;
    double *bn, *r2;              // ||B_c||, ||B_c - A X_c||^2
    int *flags;                   // BGF_*
    int *dead;                    // the dependent columns of the last starting block (s)
    GridBar *bar;
    State *st;
    double rtol;
    int deflate;                  // replace dependent starting columns (else a breakdown)
};
struct BgmKernels {
    void *init, *start, *orth, *finish;
    int block;
};
BgmKernels bgm_kernels();
size_t bgm_orth_smem(int m, int s);
size_t bgm_finish_smem(int m, int s);

// ---- block product Q = A P (k_bgemv.cu) ---------------------------------------------------
struct BgemvArgs {
    int n, s;
    const float *Ph, *Pl;         // P split into FP32 pairs: BCG_MAX_S column panels of ldp floats
    long long ldp;                // a multiple of 256, zero past n
    double *Q;                    // column-major n x s, column stride ldq
    long long ldq;
    State *st;
};
struct BgemvLaunch {
    void *func, *split;           // the product (takes the A descriptor) and the P splitter
    int grid, block, S;           // S: the kernel's column count (s rounded up to a power of two)
    size_t smem;
};
BgemvLaunch bgemv_plan(int s, int num_sms);

struct KrylovKernels {
    void *cg_init, *cg_update, *cg_check;
    void *bs_init, *bs_s, *bs_update, *bs_check;
    void *ja_diag, *ja_init, *ja_next;
    void *gm_init, *gm_start, *gm_arnoldi, *gm_finish;
    int coop_grid;       // blocks of the cooperative vector kernels
    int block;           // threads per block
};
KrylovKernels krylov_kernels(int num_sms);

// ---- fused small-system solvers (k_fused.cu) -------------------------------------------
// One launch runs a whole CG or GMRES(m) solve; CTA c keeps rows
// [c R, c R + R) of A as the FP32 pair in shared memory.  Cluster form: the
// grid is one thread-block cluster (at most FUSED_MAX_CLUSTER CTAs) that
// communicates through distributed shared memory; global form: a cooperative
// grid that communicates through global memory.
constexpr int FUSED_THREADS = 256;
constexpr int FUSED_VEC_REGS = 8;          // vector elements a thread holds: n <= 8 * 256 - 4
constexpr int FUSED_MAX_CLUSTER = 16;
constexpr int FUSED_PART_SLOTS = 2 * LS_MAX_RESTART + 8;
constexpr int FUSED_CG_SLOTS = 8;
struct FusedArgs {
    int n, R, nc;            // size, rows per CTA, row length in shared memory (n rounded up to 4)
    const double *A;         // FP64 A on the device, row-major
    long long lda;
    const double *b;         // device copy of b
    double *x;               // x0 in when x0_given; the solution out
    int x0_given;
    int max_iter;
    double rtol;
    int m, reorth;           // GMRES restart length; 1 = always two Gram-Schmidt passes
    int h_smem;              // GMRES: 1 = the Hessenberg matrix in shared memory, 0 = in H
    double *xch, *xch2;      // global form: n doubles each, the vectors exchanged between CTAs
    double *part;            // global form: partial sums, [slot][CTA], FUSED_PART_SLOTS slots
    double *H;               // GMRES, h_smem = 0: per-CTA (m + 1) x m Hessenberg copies
    unsigned *bar;           // global form: three barrier counters, zero at launch
    State *st;
};
struct FusedKernels {
    void *cg, *gmres;        // global form
    void *cg_cl, *gmres_cl;  // cluster form
};
FusedKernels fused_kernels();
// Dynamic shared memory of a fused launch (R rows per CTA, row length nc,
// restart length m and the Hessenberg matrix's place for GMRES).
inline size_t fused_smem_bytes(bool gmres, int R, int nc, int m, bool h_smem) {
    const size_t Rp = (size_t)((R + 1) & ~1), M = (size_t)m;
    const size_t dbl = gmres ? (M + 1) * Rp + 5 * Rp + 5 * (M + 2) + 4 * (M + 1) +
                                   4 * (M + 2 > Rp ? M + 2 : Rp) + FUSED_PART_SLOTS +
                                   (h_smem ? (M + 1) * M : 0)
                             : (size_t)nc + 6 * Rp + FUSED_CG_SLOTS;
    return dbl * 8 + 16 + (2 * (size_t)R * nc + 2 * (size_t)nc + 2 * Rp) * 4;
}

}  // namespace lsi
