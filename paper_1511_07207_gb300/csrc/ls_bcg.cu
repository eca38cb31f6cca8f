// ls_bcg.cu -- the host driver of block CG (ls_block_cg_solve): workspace,
// staging of A, B and X, the CUDA graph of the iteration, and the result.
//
// Graph: [s residual GEMVs if X0 is given] bcg_init,
//        while(outer){ while(inner){ Q = A P, bcg_step },
//                      s residual GEMVs R_j = B_j - A X_j (with ||R_j||^2), bcg_check }
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "ls_api_internal.h"

using namespace lsi;

namespace {

struct BcgLayout {
    double *X, *R, *P, *Q, *B, *part, *partb, *part2, *Astage;
    BcgSmall *sm;
    float *Ahi, *Alo;
    float *Ph, *Pl;      // P split for the block product (pair path)
    long long ld, lda_stage, ld32, ldp;
    size_t bytes;
};

BcgLayout bcg_layout(void *base, int n, int s, int grid, bool stageA, bool split) {
    BcgLayout L{};
    L.ld = (long long)align_up((size_t)std::max(n, 1), 64);
    L.lda_stage = (long long)align_up((size_t)std::max(n, 1), 2);
    L.ld32 = (long long)align_up((size_t)std::max(n, 1), 4);
    Carver cv(base);
    L.X = cv.take<double>((size_t)L.ld * s);
    L.R = cv.take<double>((size_t)L.ld * s);
    L.P = cv.take<double>((size_t)L.ld * s);
    L.Q = cv.take<double>((size_t)L.ld * s);
    L.B = cv.take<double>((size_t)L.ld * s);
    L.part = cv.take<double>((size_t)grid * BCG_MAX_S * BCG_MAX_S);
    L.partb = cv.take<double>((size_t)grid * BCG_MAX_S * BCG_MAX_S);
    L.part2 = cv.take<double>((size_t)grid * BCG_MAX_S);
    L.sm = cv.take<BcgSmall>(1);
    L.Ahi = split ? cv.take<float>((size_t)n * L.ld32) : nullptr;
    L.Alo = split ? cv.take<float>((size_t)n * L.ld32) : nullptr;
    L.ldp = (long long)align_up((size_t)std::max(n, 1), 256);
    L.Ph = split ? cv.take<float>((size_t)BCG_MAX_S * L.ldp) : nullptr;
    L.Pl = split ? cv.take<float>((size_t)BCG_MAX_S * L.ldp) : nullptr;
    L.Astage = stageA ? cv.take<double>((size_t)n * L.lda_stage) : nullptr;   // last (see ls_api.cu)
    L.bytes = align_up(cv.off, 256);
    return L;
}

void resid_nodes(ls_ctx *c, Chain &ch, const GemvLaunch &GL, const BcgVecs &v, const BcgLayout &L) {
    for (int j = 0; j < v.s; j++) {
        GemvArgs a{};
        a.x = v.X + (long long)j * v.ld;
        a.y = v.R + (long long)j * v.ld;
        a.b = v.B + (long long)j * v.ld;
        a.dot_out = &L.sm->r2[j];
        a.st = v.st;
        a.scr = c->scr;
        a.epi = EPI_RESID;
        a.fin = FIN_STORE;
        gemv_node(ch, GL, c->dA, a);
    }
}

int build_bcg_graph(ls_ctx *c, const BcgVecs &v, const BcgLayout &L, const GemvLaunch &GL, int x0_given,
                    int deflate, const long long *key) {
    const BcgKernels K = bcg_kernels();
    void *const k_init = deflate ? K.dinit : K.init, *const k_step = deflate ? K.dstep : K.step;
    void *const k_check = deflate ? K.dcheck : K.check;
    Root R;
    if (!R.create()) return LS_ERR_CUDA;
    cudaGraphConditionalHandle ho, hi;
    if (!R.handle(&ho) || !R.handle(&hi)) {
        R.discard();
        return LS_ERR_CUDA;
    }
    Chain top = R.chain();
    if (x0_given) resid_nodes(c, top, GL, v, L);
    {
        BcgVecs vv = v;
        int x0 = x0_given;
        void *args[] = {&vv, &x0, &ho, &hi};
        top.kernel(k_init, c->K.coop_grid, K.block, 0, args, true);
    }
    Chain outer = top.loop(ho);
    Chain inner = outer.loop(hi);
    if (L.Ph) {
        // Q = A P in one pass over the pair of A (P split first)
        const BgemvLaunch BL = bgemv_plan(v.s, c->num_sms);
        int nn = v.n, ss = v.s, SS = BL.S;
        const double *Pp = v.P;
        long long ld = v.ld, ldp = L.ldp;
        float *ph = L.Ph, *pl = L.Pl;
        State *stp = v.st;
        const int *kp = nullptr;
        long long kst = 0;
        void *sargs[] = {&nn, &ss, &SS, &Pp, &ld, &ph, &pl, &ldp, &stp, &kp, &kst};
        inner.kernel(BL.split, 4 * c->num_sms, 256, 0, sargs, false);
        BgemvArgs ba{};
        ba.n = v.n;
        ba.s = v.s;
        ba.Ph = L.Ph;
        ba.Pl = L.Pl;
        ba.ldp = L.ldp;
        ba.Q = v.Q;
        ba.ldq = v.ld;
        ba.st = v.st;
        const MatDesc *pA = c->dA;
        void *bargs[] = {&pA, &ba};
        inner.kernel(BL.func, BL.grid, BL.block, BL.smem, bargs, false);
    } else {
        for (int j = 0; j < v.s; j++) {   // native FP64 products: one GEMV per column
            GemvArgs a{};
            a.x = v.P + (long long)j * v.ld;
            a.y = v.Q + (long long)j * v.ld;
            a.st = v.st;
            a.scr = c->scr;
            a.epi = EPI_STORE;
            a.fin = FIN_STORE;
            gemv_node(inner, GL, c->dA, a);
        }
    }
    {
        BcgVecs vv = v;
        void *args[] = {&vv, &hi};
        inner.kernel(k_step, c->K.coop_grid, K.block, 0, args, true);
    }
    resid_nodes(c, outer, GL, v, L);
    {
        BcgVecs vv = v;
        void *args[] = {&vv, &ho, &hi};
        outer.kernel(k_check, c->K.coop_grid, K.block, 0, args, true);
    }
    if (top.err != cudaSuccess || inner.err != cudaSuccess || outer.err != cudaSuccess) {
        R.discard();
        return LS_ERR_CUDA;
    }
    return finish_graph(c, c->graph_bcg, R, key);
}

// s columns of n doubles between a caller block (leading dimension ld_user,
// host or device) and a workspace block (leading dimension ld).
cudaError_t copy_block(ls_ctx *c, double *dst, long long ldd, const double *src, long long lds, int n, int s) {
    return cudaMemcpy2DAsync(dst, ldd * sizeof(double), src, lds * sizeof(double), (size_t)n * sizeof(double), s,
                             cudaMemcpyDefault, c->stream);
}

}  // namespace

size_t lsi::bcg_workspace_bytes(int n, int s, int grid, bool a_on_device, bool split) {
    return bcg_layout(nullptr, n, s, grid, !a_on_device, split).bytes;
}

extern "C" int ls_block_cg_solve(ls_ctx *c, int n, int s, const double *A, int64_t lda, const double *B,
                                 int64_t ldb, double *X, int64_t ldx, const ls_opts *opts, ls_info *info) {
    ls_opts o;
    if (opts) o = *opts;
    else ls_opts_default(&o);
    if (!c || n < 0 || s < 1 || s > BCG_MAX_S || lda < n || ldb < n || ldx < n) return LS_ERR_ARG;
    if (n > 0 && (!A || !B || !X)) return LS_ERR_ARG;
    if (!(o.rtol >= 0.0) || o.max_iter < 0) return LS_ERR_ARG;
    if (o.precision != LS_F64) return LS_ERR_UNSUPPORTED;
    if (cudaSetDevice(c->device) != cudaSuccess) return LS_ERR_CUDA;
    if (n == 0) {
        State z{};
        fill_info(info, z, LS_OK, 0.f, 0.0, 0);
        return LS_OK;
    }
    const int max_iter = o.max_iter > 0 ? o.max_iter : 10 * n + 10;
    const bool a_dev = is_device_ptr(A);
    const bool split = o.f64_matvec == 0;
    const int grid = c->K.coop_grid;
    BcgLayout L = bcg_layout(nullptr, n, s, grid, !a_dev, split);
    int rc = ws_reserve(c, L.bytes);
    if (rc) return rc;
    L = bcg_layout(c->ws, n, s, grid, !a_dev, split);

    const double *Ad;
    long long ldad;
    rc = stage_matrix(c, n, A, lda, L.Astage, L.lda_stage, &Ad, &ldad);
    if (rc) return rc;
    cudaError_t e = copy_block(c, L.B, L.ld, B, ldb, n, s);
    if (e == cudaSuccess && o.x0_given) e = copy_block(c, L.X, L.ld, X, ldx, n, s);
    if (e != cudaSuccess) return map_cuda(e);
    MatDesc *hd = &c->h_desc[0];
    memset(hd, 0, sizeof(MatDesc));
    if (split) make_tensor_map_ds(hd, L.Ahi, L.Alo, n, n, L.ld32);
    else make_tensor_map(hd, DT_F64, Ad, n, n, ldad);
    rc = upload_desc(c, 0);
    State *hs = c->h_st;
    state_init(hs, max_iter);
    if (!rc) rc = upload_state(c);
    if (rc) return rc;

    BcgVecs v{};
    v.n = n;
    v.s = s;
    v.ld = L.ld;
    v.X = L.X;
    v.R = L.R;
    v.P = L.P;
    v.Q = L.Q;
    v.B = L.B;
    v.part = L.part;
    v.partb = L.partb;
    v.part2 = L.part2;
    v.sm = L.sm;
    v.bar = c->bar;
    v.st = c->st;
    v.rtol = o.rtol;
    const int dt = split ? DT_DS : DT_F64;
    GemvLaunch GL = gemv_plan(dt, hd->use_tma != 0, EPI_DOT, c->num_sms);
    const int deflate = o.deflate ? 1 : 0;
    long long key[8] = {200 + s + 100 * deflate, n, (long long)(uintptr_t)c->ws, L.ld, o.x0_given, hd->use_tma,
                        (long long)(uintptr_t)c->stream, dt};
    if (!c->graph_bcg.matches(key)) {
        rc = build_bcg_graph(c, v, L, GL, o.x0_given, deflate, key);
        if (rc) return rc;
    }
    e = cudaEventRecord(c->ev0, c->stream);
    if (e == cudaSuccess && split) e = split_f64_launch(n, n, Ad, ldad, L.Ahi, L.Alo, L.ld32, c->num_sms, c->stream);
    if (e != cudaSuccess) return map_cuda(e);
    rc = launch_cached(c, c->graph_bcg);
    if (rc) return rc;
    e = cudaEventRecord(c->ev1, c->stream);
    if (e != cudaSuccess) return map_cuda(e);
    rc = read_state(c);
    if (rc) return rc;
    BcgSmall hsm;
    e = cudaMemcpyAsync(&hsm, L.sm, sizeof(BcgSmall), cudaMemcpyDeviceToHost, c->stream);
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
    // worst true relative residual over the columns (from the last residual GEMVs)
    double worst = 0.0;
    for (int j = 0; j < s; j++) {
        const double r = hsm.bn[j] > 0.0 ? std::sqrt(hsm.r2[j]) / hsm.bn[j] : std::sqrt(hsm.r2[j]);
        if (!(r <= worst)) worst = r;
    }
    State sc = st;
    sc.bnorm = 1.0;
    sc.rnorm = worst;
    sc.true_rnorm = worst;
    const double passes = (double)s * (st.iter + st.cycles + 1 + (o.x0_given ? 1 : 0));
    c->launches_total += (long long)st.launches;
    fill_info(info, sc, status, ms, passes * (double)n * n * 8.0, (long long)st.launches);
    return status;
}
