// ls_mixed.cu -- driver of the mixed-precision CG solve (opts->precision =
// LS_BF16_IR / LS_FP8_IR / LS_F32_IR): quantise A once on the device, then one
// CUDA graph runs the FP64 outer loop (flexible CG or classic refinement)
// around an FP32 inner CG on the stored matrix, with no host round trip.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "ls_api_internal.h"

namespace lsi {

struct MixLayout {
    double *x, *b, *r, *q, *P, *W, *dvals, *Astage;
    float *rf, *zf, *pf, *qf, *scale;
    float *Ahi, *Alo;       // FP32 pair of A for the outer FP64 products (f64_matvec = 0)
    void *Q;
    long long npad, ldp, ldq, lda_stage, ld32;
    int m;
    size_t bytes;
};

static int elt_size(int dtype) { return dtype == DT_BF16 ? 2 : dtype == DT_FP8 ? 1 : 4; }

static MixLayout mix_layout(void *base, int n, int dtype, int m, bool fcg, bool stageA, bool split) {
    MixLayout L{};
    L.npad = (long long)align_up((size_t)std::max(n, 1), 64);
    L.ldp = L.npad;
    L.ldq = (long long)align_up((size_t)std::max(n, 1), 64);
    L.lda_stage = (long long)align_up((size_t)std::max(n, 1), 2);
    L.m = m;
    Carver cv(base);
    L.x = cv.take<double>(L.npad);
    L.b = cv.take<double>(L.npad);
    L.r = cv.take<double>(L.npad);
    L.q = cv.take<double>(L.npad);
    L.P = cv.take<double>(fcg ? (size_t)L.ldp * m : L.npad);
    L.W = cv.take<double>(fcg ? (size_t)L.ldp * m : L.npad);
    L.dvals = cv.take<double>((size_t)m + 1);
    L.rf = cv.take<float>(L.npad);
    L.zf = cv.take<float>(L.npad);
    L.pf = cv.take<float>(L.npad);
    L.qf = cv.take<float>(L.npad);
    L.scale = cv.take<float>(L.npad);
    L.Q = cv.take<unsigned char>((size_t)n * L.ldq * elt_size(dtype));
    L.ld32 = (long long)align_up((size_t)std::max(n, 1), 4);
    L.Ahi = split ? cv.take<float>((size_t)n * L.ld32) : nullptr;
    L.Alo = split ? cv.take<float>((size_t)n * L.ld32) : nullptr;
    // last: no other pointer moves with whether A is staged or borrowed
    L.Astage = stageA ? cv.take<double>((size_t)n * L.lda_stage) : nullptr;
    L.bytes = align_up(cv.off, 256);
    return L;
}

static int storage_dtype(int precision) {
    return precision == LS_BF16_IR ? DT_BF16 : precision == LS_FP8_IR ? DT_FP8 : DT_F32;
}

static int outer_limit(const ls_opts &o) { return o.max_iter > 0 ? o.max_iter : 60; }

size_t mixed_workspace_bytes(int n, const ls_opts *o, bool a_on_device) {
    const int max_outer = outer_limit(*o);
    const int m = std::min(max_outer, LS_MAX_RESTART);
    return mix_layout(nullptr, n, storage_dtype(o->precision), m, o->refine == LS_REFINE_FCG, o->f64_matvec == 0,
                      !a_on_device).bytes;
}

static int build_mixed_graph(ls_ctx *c, const MixVecs &v, const GemvLaunch &L64,
                             const GemvLaunch &Llo, int x0_given, const long long *key) {
    const MixedKernels K = mixed_kernels();
    const int G = c->K.coop_grid, B = c->K.block;
    Root R;
    if (!R.create()) return LS_ERR_CUDA;
    // Every handle must belong to a conditional node of the graph: the
    // refinement loop has no super loop, so it passes its outer handle twice.
    cudaGraphConditionalHandle hs, ho, hi;
    if (!R.handle(&ho) || !R.handle(&hi) || (v.mode == LS_REFINE_FCG && !R.handle(&hs))) {
        R.discard();
        return LS_ERR_CUDA;
    }
    if (v.mode != LS_REFINE_FCG) hs = ho;
    const MatDesc *d64 = c->dA, *dlo = c->dA + 1;
    MixVecs vv = v;
    Chain top = R.chain();
    if (x0_given) {
        GemvArgs a{};
        a.x = v.x; a.y = v.r; a.b = v.b; a.st = v.st; a.scr = c->scr;
        a.epi = EPI_RESID; a.fin = FIN_TRUE_RES;
        gemv_node(top, L64, d64, a);
    }
    {
        int x0 = x0_given;
        void *args[] = {&vv, &x0, &hs, &ho};
        top.kernel(K.mx_init, G, B, 0, args, true);
    }
    // inner FP32 CG body (shared by both outer loops)
    auto inner_body = [&](Chain &in) {
        GemvArgs a{};
        a.x = v.pf; a.y = v.qf; a.z = v.pf; a.st = v.st; a.scr = c->scr;
        a.epi = EPI_DOT; a.fin = FIN_INNER_ALPHA;
        gemv_node(in, Llo, dlo, a);
        void *args[] = {&vv, &hi};
        in.kernel(K.in_update, G, B, 0, args, true);
        return in.err;
    };
    cudaError_t err = cudaSuccess;
    if (v.mode == LS_REFINE_FCG) {
        Chain sup = top.loop(hs);
        Chain out = sup.loop(ho);
        {
            void *args[] = {&vv, &hi};
            out.kernel(K.in_init, G, B, 0, args, true);
        }
        Chain in = out.loop(hi);
        err = inner_body(in);
        {
            void *args[] = {&vv};
            out.kernel(K.fcg_project, G, B, 0, args, true);
            GemvArgs a{};
            a.x = v.P; a.y = v.W; a.kptr = &v.st->nstored; a.kstride = v.ldp; a.kyoff = 0;
            a.z_is_x = 1; a.st = v.st; a.scr = c->scr;
            a.epi = EPI_DOT; a.fin = FIN_FCG_D;
            gemv_node(out, L64, d64, a);
            void *args2[] = {&vv, &ho};
            out.kernel(K.fcg_update, G, B, 0, args2, true);
        }
        {
            GemvArgs a{};
            a.x = v.x; a.y = v.q; a.b = v.b; a.st = v.st; a.scr = c->scr;
            a.epi = EPI_RESID; a.fin = FIN_TRUE_RES;
            gemv_node(sup, L64, d64, a);
            void *args[] = {&vv, &hs, &ho};
            sup.kernel(K.mx_check, G, B, 0, args, false);
        }
        if (top.err || sup.err || out.err || err) err = cudaErrorUnknown;
    } else {
        Chain out = top.loop(ho);
        {
            GemvArgs a{};
            a.x = v.x; a.y = v.r; a.b = v.b; a.st = v.st; a.scr = c->scr;
            a.epi = EPI_RESID; a.fin = FIN_TRUE_RES;
            gemv_node(out, L64, d64, a);
            void *args[] = {&vv, &ho, &hi};
            out.kernel(K.ir_start, G, B, 0, args, true);
        }
        Chain in = out.loop(hi);
        err = inner_body(in);
        {
            void *args[] = {&vv};
            out.kernel(K.ir_update, G, B, 0, args, false);
        }
        if (top.err || out.err || err) err = cudaErrorUnknown;
    }
    if (err != cudaSuccess) {
        R.discard();
        return LS_ERR_CUDA;
    }
    return finish_graph(c, c->graph_mx, R, key);
}

int mixed_cg_solve(ls_ctx *c, int n, const double *A, int64_t lda, const double *b, double *x,
                   const ls_opts *opts, ls_info *info) {
    if (!c || !opts) return LS_ERR_ARG;
    ls_opts o = *opts;
    if (n < 0 || lda < n || (n > 0 && (!A || !b || !x))) return LS_ERR_ARG;
    if (!(o.rtol >= 0.0) || o.max_iter < 0 || o.inner_iters < 0 || !(o.inner_rtol >= 0.0))
        return LS_ERR_ARG;
    if (o.precision != LS_BF16_IR && o.precision != LS_FP8_IR && o.precision != LS_F32_IR)
        return LS_ERR_ARG;
    if (o.refine != LS_REFINE_FCG && o.refine != LS_REFINE_IR) return LS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return LS_ERR_CUDA;
    if (n == 0) {
        State s{};
        fill_info(info, s, LS_OK, 0.f, 0.0, 0);
        return LS_OK;
    }
    const int dtype = storage_dtype(o.precision);
    const int max_outer = outer_limit(o);
    const int m = std::min(max_outer, LS_MAX_RESTART);
    const bool fcg = o.refine == LS_REFINE_FCG;
    const bool a_dev = is_device_ptr(A);
    const bool split = o.f64_matvec == 0;
    MixLayout L = mix_layout(nullptr, n, dtype, m, fcg, !a_dev, split);
    int rc = ws_reserve(c, L.bytes);
    if (rc) return rc;
    L = mix_layout(c->ws, n, dtype, m, fcg, !a_dev, split);

    const double *Ad;
    long long ldad;
    rc = stage_matrix(c, n, A, lda, L.Astage, L.lda_stage, &Ad, &ldad);
    if (!rc) rc = copy_in(c, L.b, b, n);
    if (!rc && o.x0_given) rc = copy_in(c, L.x, x, n);
    if (rc) return rc;

    cudaError_t e = cudaEventRecord(c->ev0, c->stream);
    if (e == cudaSuccess)   // stage A: quantise once per solve
        e = quantize_launch(dtype, n, n, Ad, ldad, L.Q, L.ldq, L.scale, c->num_sms, c->stream);
    if (e == cudaSuccess && split)   // and the FP32 pair for the outer FP64 products
        e = split_f64_launch(n, n, Ad, ldad, L.Ahi, L.Alo, L.ld32, c->num_sms, c->stream);
    if (e != cudaSuccess) return map_cuda(e);

    MatDesc *h64 = &c->h_desc[0], *hlo = &c->h_desc[1];
    memset(h64, 0, sizeof(MatDesc));
    memset(hlo, 0, sizeof(MatDesc));
    if (split) make_tensor_map_ds(h64, L.Ahi, L.Alo, n, n, L.ld32);
    else make_tensor_map(h64, DT_F64, Ad, n, n, ldad);
    make_tensor_map(hlo, dtype, L.Q, n, n, L.ldq);
    hlo->scale = dtype == DT_FP8 ? L.scale : nullptr;
    rc = upload_desc(c, 0);
    if (!rc) rc = upload_desc(c, 1);
    State *hs = c->h_st;
    state_init(hs, 0);
    hs->max_outer = max_outer;
    hs->m = m;
    hs->in_max = o.inner_iters;
    hs->in_tol2 = o.inner_rtol > 0.0 ? (float)(o.inner_rtol * o.inner_rtol) : -1.0f;
    hs->launches = split ? 2 : 1;   // the quantisation (and split) kernels
    if (!rc) rc = upload_state(c);
    if (rc) return rc;

    MixVecs v{};
    v.n = n;
    v.mode = o.refine;
    v.x = L.x; v.b = L.b; v.r = L.r; v.q = L.q; v.P = L.P; v.W = L.W; v.ldp = L.ldp;
    v.dvals = L.dvals;
    v.rf = L.rf; v.zf = L.zf; v.pf = L.pf; v.qf = L.qf;
    v.part = c->part; v.bar = c->bar; v.st = c->st; v.rtol = o.rtol;
    GemvLaunch L64 = gemv_plan(split ? DT_DS : DT_F64, h64->use_tma != 0, EPI_DOT, c->num_sms);
    GemvLaunch Llo = gemv_plan(dtype, hlo->use_tma != 0, EPI_DOT, c->num_sms);
    long long key[8] = {100 + o.refine, n, (long long)(uintptr_t)c->ws, dtype * 2 + (split ? 1 : 0), o.x0_given,
                        h64->use_tma * 2 + hlo->use_tma, (long long)(uintptr_t)c->stream, m};
    if (!c->graph_mx.matches(key)) {
        rc = build_mixed_graph(c, v, L64, Llo, o.x0_given, key);
        if (rc) return rc;
    }
    rc = launch_cached(c, c->graph_mx);
    if (rc) return rc;
    e = cudaEventRecord(c->ev1, c->stream);
    if (e != cudaSuccess) return map_cuda(e);
    rc = read_state(c);
    if (rc) return rc;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    const State &s = *hs;
    const int status = status_from_state(s);
    if (status >= 0) {
        e = cudaMemcpyAsync(x, L.x, n * sizeof(double), cudaMemcpyDefault, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return map_cuda(e);
    }
    // algorithmic bytes of A: quantisation (read FP64, write low precision),
    // FP64 products (outer steps + residual checks + x0), low-precision products
    const double nn = (double)n * n;
    const int esz = elt_size(dtype);
    const double f64_passes = (fcg ? s.outer + s.cycles : s.outer + 1) + (o.x0_given ? 1 : 0);
    const double bytes = nn * (8.0 + esz) + f64_passes * 8.0 * nn + (double)s.iter * esz * nn;
    State sc = s;
    sc.cycles = s.outer;
    c->launches_total += (long long)s.launches;
    fill_info(info, sc, status, ms, bytes, (long long)s.launches);
    return status;
}

}  // namespace lsi
