// ls_bgmres.cu -- the host driver of restarted block GMRES (ls_block_gmres_solve):
// workspace, staging of A, B and X, the CUDA graph of the iteration, the result.
//
// Graph: bgm_init, while(outer){ split X, A X into V's first block (block
//        product), bgm_start (R = B - A X, ||R_c||^2, the stop test, V_1 S = R
//        with the dependent columns of R replaced when opts.deflate is set),
//        while(inner){ split V_j, W = A V_j (block product), bgm_orth }, bgm_finish }
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "ls_api_internal.h"

using namespace lsi;

namespace {

struct BgmLayout {
    double *X, *B, *W, *V, *H, *G, *Y, *cs, *sn, *Hc, *Lm, *part, *bn, *r2, *Astage;
    int *rrow, *flags, *dead;
    float *Ahi, *Alo, *Ph, *Pl;
    long long ld, lda_stage, ld32, ldp, part_stride;
    size_t bytes;
};

BgmLayout bgm_layout(void *base, int n, int s, int m, int grid, bool stageA) {
    BgmLayout L{};
    L.ld = (long long)align_up((size_t)std::max(n, 1), 64);
    L.lda_stage = (long long)align_up((size_t)std::max(n, 1), 2);
    L.ld32 = (long long)align_up((size_t)std::max(n, 1), 4);
    L.ldp = (long long)align_up((size_t)std::max(n, 1), 256);
    const long long LH = (long long)(m + 1) * s;
    L.part_stride = LH * s;
    Carver cv(base);
    L.X = cv.take<double>((size_t)L.ld * s);
    L.B = cv.take<double>((size_t)L.ld * s);
    L.W = cv.take<double>((size_t)L.ld * s);
    L.V = cv.take<double>((size_t)L.ld * LH);
    L.H = cv.take<double>((size_t)LH * m * s);
    L.G = cv.take<double>((size_t)LH * s);
    L.Y = cv.take<double>((size_t)m * s * s);
    L.cs = cv.take<double>((size_t)m * s * s);
    L.sn = cv.take<double>((size_t)m * s * s);
    L.rrow = cv.take<int>((size_t)m * s * s);
    L.Hc = cv.take<double>((size_t)LH * s);
    L.Lm = cv.take<double>((size_t)BGM_MAX_S * BGM_MAX_S);
    L.part = cv.take<double>((size_t)grid * L.part_stride);
    L.bn = cv.take<double>(BGM_MAX_S);
    L.r2 = cv.take<double>(BGM_MAX_S);
    L.flags = cv.take<int>(BGF_COUNT);
    L.dead = cv.take<int>(BGM_MAX_S);
    L.Ahi = cv.take<float>((size_t)n * L.ld32);
    L.Alo = cv.take<float>((size_t)n * L.ld32);
    L.Ph = cv.take<float>((size_t)BCG_MAX_S * L.ldp);
    L.Pl = cv.take<float>((size_t)BCG_MAX_S * L.ldp);
    L.Astage = stageA ? cv.take<double>((size_t)n * L.lda_stage) : nullptr;   // last (see ls_api.cu)
    L.bytes = align_up(cv.off, 256);
    return L;
}

int build_bgm_graph(ls_ctx *c, const BgmVecs &v, const BgmLayout &L, int x0_given, const long long *key) {
    const BgmKernels K = bgm_kernels();
    const BgemvLaunch BL = bgemv_plan(v.s, c->num_sms);
    const size_t orth_smem = bgm_orth_smem(v.m, v.s), fin_smem = bgm_finish_smem(v.m, v.s);
    set_smem_limit(K.orth, orth_smem);
    set_smem_limit(K.finish, fin_smem);
    Root R;
    if (!R.create()) return LS_ERR_CUDA;
    cudaGraphConditionalHandle ho, hi;
    if (!R.handle(&ho) || !R.handle(&hi)) {
        R.discard();
        return LS_ERR_CUDA;
    }
    Chain top = R.chain();
    {
        BgmVecs vv = v;
        int x0 = x0_given;
        void *args[] = {&vv, &x0, &ho, &hi};
        top.kernel(K.init, c->K.coop_grid, K.block, 0, args, true);
    }
    Chain outer = top.loop(ho);
    {   // A X into V's first block, one pass over A for all columns
        int nn = v.n, ss = v.s, SS = BL.S;
        const double *Xp = v.X;
        long long ld = v.ld, ldp = L.ldp;
        float *ph = L.Ph, *pl = L.Pl;
        State *stp = v.st;
        const int *kp = nullptr;
        long long kst = 0;
        void *sargs[] = {&nn, &ss, &SS, &Xp, &ld, &ph, &pl, &ldp, &stp, &kp, &kst};
        outer.kernel(BL.split, 4 * c->num_sms, 256, 0, sargs, false);
        BgemvArgs ba{};
        ba.n = v.n;
        ba.s = v.s;
        ba.Ph = L.Ph;
        ba.Pl = L.Pl;
        ba.ldp = L.ldp;
        ba.Q = v.V;
        ba.ldq = v.ld;
        ba.st = v.st;
        const MatDesc *pA = c->dA;
        void *bargs[] = {&pA, &ba};
        outer.kernel(BL.func, BL.grid, BL.block, BL.smem, bargs, false);
    }
    {
        BgmVecs vv = v;
        void *args[] = {&vv, &ho, &hi};
        outer.kernel(K.start, c->K.coop_grid, K.block, 0, args, true);
    }
    Chain inner = outer.loop(hi);
    {
        int nn = v.n, ss = v.s, SS = BL.S;
        const double *Pp = v.V;
        long long ld = v.ld, ldp = L.ldp;
        float *ph = L.Ph, *pl = L.Pl;
        State *stp = v.st;
        const int *kp = &v.st->k;
        long long kst = (long long)v.s * v.ld;
        void *sargs[] = {&nn, &ss, &SS, &Pp, &ld, &ph, &pl, &ldp, &stp, &kp, &kst};
        inner.kernel(BL.split, 4 * c->num_sms, 256, 0, sargs, false);
        BgemvArgs ba{};
        ba.n = v.n;
        ba.s = v.s;
        ba.Ph = L.Ph;
        ba.Pl = L.Pl;
        ba.ldp = L.ldp;
        ba.Q = v.W;
        ba.ldq = v.ld;
        ba.st = v.st;
        const MatDesc *pA = c->dA;
        void *bargs[] = {&pA, &ba};
        inner.kernel(BL.func, BL.grid, BL.block, BL.smem, bargs, false);
        BgmVecs vv = v;
        void *args[] = {&vv, &hi};
        inner.kernel(K.orth, c->K.coop_grid, K.block, orth_smem, args, true);
    }
    {
        BgmVecs vv = v;
        void *args[] = {&vv};
        outer.kernel(K.finish, c->K.coop_grid, K.block, fin_smem, args, true);
    }
    if (top.err != cudaSuccess || inner.err != cudaSuccess || outer.err != cudaSuccess) {
        R.discard();
        return LS_ERR_CUDA;
    }
    return finish_graph(c, c->graph_bgm, R, key);
}

cudaError_t copy_block(ls_ctx *c, double *dst, long long ldd, const double *src, long long lds, int n, int s) {
    return cudaMemcpy2DAsync(dst, ldd * sizeof(double), src, lds * sizeof(double), (size_t)n * sizeof(double), s,
                             cudaMemcpyDefault, c->stream);
}

}  // namespace

size_t lsi::bgm_workspace_bytes(int n, int s, int m, int grid, bool a_on_device) {
    return bgm_layout(nullptr, n, s, m, grid, !a_on_device).bytes;
}

extern "C" int ls_block_gmres_solve(ls_ctx *c, int n, int s, const double *A, int64_t lda, const double *B,
                                    int64_t ldb, double *X, int64_t ldx, const ls_opts *opts, ls_info *info) {
    ls_opts o;
    if (opts) o = *opts;
    else ls_opts_default(&o);
    if (!c || n < 0 || s < 1 || s > BGM_MAX_S || lda < n || ldb < n || ldx < n) return LS_ERR_ARG;
    if (n > 0 && (!A || !B || !X)) return LS_ERR_ARG;
    if (!(o.rtol >= 0.0) || o.max_iter < 0 || o.restart < 1 || o.restart * s > BGM_MAX_MS) return LS_ERR_ARG;
    if (o.precision != LS_F64 || o.f64_matvec) return LS_ERR_UNSUPPORTED;
    if (cudaSetDevice(c->device) != cudaSuccess) return LS_ERR_CUDA;
    if (n == 0) {
        State z{};
        fill_info(info, z, LS_OK, 0.f, 0.0, 0);
        return LS_OK;
    }
    const int m = o.restart;
    const int max_iter = o.max_iter > 0 ? o.max_iter : 10 * n + 10;
    const bool a_dev = is_device_ptr(A);
    const int grid = c->K.coop_grid;
    BgmLayout L = bgm_layout(nullptr, n, s, m, grid, !a_dev);
    int rc = ws_reserve(c, L.bytes);
    if (rc) return rc;
    L = bgm_layout(c->ws, n, s, m, grid, !a_dev);

    const double *Ad;
    long long ldad;
    rc = stage_matrix(c, n, A, lda, L.Astage, L.lda_stage, &Ad, &ldad);
    if (rc) return rc;
    cudaError_t e = copy_block(c, L.B, L.ld, B, ldb, n, s);
    if (e == cudaSuccess && o.x0_given) e = copy_block(c, L.X, L.ld, X, ldx, n, s);
    if (e != cudaSuccess) return map_cuda(e);
    MatDesc *hd = &c->h_desc[0];
    memset(hd, 0, sizeof(MatDesc));
    if (!make_tensor_map_ds(hd, L.Ahi, L.Alo, n, n, L.ld32)) return LS_ERR_UNSUPPORTED;
    rc = upload_desc(c, 0);
    State *hs = c->h_st;
    state_init(hs, max_iter);
    hs->m = m;
    if (!rc) rc = upload_state(c);
    if (rc) return rc;

    BgmVecs v{};
    v.n = n;
    v.s = s;
    v.m = m;
    v.ld = L.ld;
    v.V = L.V;
    v.W = L.W;
    v.X = L.X;
    v.B = L.B;
    v.H = L.H;
    v.G = L.G;
    v.Y = L.Y;
    v.cs = L.cs;
    v.sn = L.sn;
    v.rrow = L.rrow;
    v.Hc = L.Hc;
    v.Lm = L.Lm;
    v.part = L.part;
    v.part_stride = L.part_stride;
    v.bn = L.bn;
    v.r2 = L.r2;
    v.flags = L.flags;
    v.dead = L.dead;
    v.bar = c->bar;
    v.st = c->st;
    v.rtol = o.rtol;
    v.deflate = o.deflate ? 1 : 0;
    long long key[8] = {300 + s + 50 * v.deflate, n, (long long)(uintptr_t)c->ws, m, o.x0_given, L.ld,
                        (long long)(uintptr_t)c->stream, DT_DS};
    if (!c->graph_bgm.matches(key)) {
        rc = build_bgm_graph(c, v, L, o.x0_given, key);
        if (rc) return rc;
    }
    e = cudaEventRecord(c->ev0, c->stream);
    if (e == cudaSuccess) e = split_f64_launch(n, n, Ad, ldad, L.Ahi, L.Alo, L.ld32, c->num_sms, c->stream);
    if (e != cudaSuccess) return map_cuda(e);
    rc = launch_cached(c, c->graph_bgm);
    if (rc) return rc;
    e = cudaEventRecord(c->ev1, c->stream);
    if (e != cudaSuccess) return map_cuda(e);
    rc = read_state(c);
    if (rc) return rc;
    double r2[BGM_MAX_S], bn[BGM_MAX_S];
    e = cudaMemcpyAsync(r2, L.r2, sizeof(double) * s, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bn, L.bn, sizeof(double) * s, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return map_cuda(e);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    const State &st = *hs;
    const int status = status_from_state(st);
    if (status >= 0) {
        e = copy_block(c, X, ldx, L.X, L.ld, n, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return map_cuda(e);
    }
    double worst = 0.0;
    for (int j = 0; j < s; j++) {
        const double r = bn[j] > 0.0 ? std::sqrt(r2[j]) / bn[j] : std::sqrt(r2[j]);
        if (!(r <= worst)) worst = r;
    }
    State sc = st;
    sc.bnorm = 1.0;
    sc.rnorm = worst;
    sc.true_rnorm = worst;
    const double passes = (double)st.iter + st.cycles + 1;   // one pass of A per block product
    c->launches_total += (long long)st.launches;
    fill_info(info, sc, status, ms, passes * (double)n * n * 8.0, (long long)st.launches);
    return status;
}
