// ls_lu.cu -- the host driver of the direct method (ls_lu_solve, ls_lu_factor):
// the working matrix [A | b] in the workspace, the elimination by panels
// (per panel: the cooperative panel factorization, the row swaps elsewhere,
// the pivot rows right of the panel, the trailing update), the back
// substitution, the residual check.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "ls_api_internal.h"

using namespace lsi;

namespace {


struct LuLayout {
    double *W, *x, *r, *cand_v, *Astage;
    int *ipiv, *cand_i;
    long long ld, lda_stage;
    size_t bytes;
};

LuLayout lu_layout(void *base, int n, int grid, bool stageA) {
    LuLayout L{};
    L.ld = (long long)align_up((size_t)n + 1, 2);
    L.lda_stage = (long long)align_up((size_t)std::max(n, 1), 2);
    Carver cv(base);
    L.W = cv.take<double>((size_t)std::max(n, 1) * L.ld);
    L.x = cv.take<double>((size_t)std::max(n, 1));
    L.r = cv.take<double>((size_t)std::max(n, 1));
    L.ipiv = cv.take<int>((size_t)std::max(n, 1));
    L.cand_v = cv.take<double>((size_t)grid);
    L.cand_i = cv.take<int>((size_t)grid);
    L.Astage = stageA ? cv.take<double>((size_t)n * L.lda_stage) : nullptr;   // last (see ls_api.cu)
    L.bytes = align_up(cv.off, 256);
    return L;
}

// Stage A and b into [A | b] and run the elimination; on return the state
// holds the status (LS_BREAKDOWN on a zero pivot).
int lu_run(ls_ctx *c, int n, const double *A, long long lda, const double *b, LuLayout &L, LuArgs &a,
           const double **Ad_out, long long *ldad_out, bool solve, float *ms) {
    const double *Ad;
    long long ldad;
    int rc = stage_matrix(c, n, A, lda, L.Astage, L.lda_stage, &Ad, &ldad);
    if (rc) return rc;
    cudaError_t e = cudaMemcpy2DAsync(L.W, L.ld * sizeof(double), Ad, ldad * sizeof(double), (size_t)n * sizeof(double),
                                      n, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(L.W + n, L.ld * sizeof(double), b, sizeof(double), sizeof(double), n, cudaMemcpyDefault,
                              c->stream);
    if (e != cudaSuccess) return map_cuda(e);
    state_init(c->h_st, 0);
    rc = upload_state(c);
    if (rc) return rc;
    a = LuArgs{};
    a.n = n;
    a.W = L.W;
    a.ld = L.ld;
    a.ipiv = L.ipiv;
    a.x = L.x;
    a.cand_v = L.cand_v;
    a.cand_i = L.cand_i;
    a.bar = c->bar;
    a.st = c->st;
    const LuKernels K = lu_kernels();
    e = cudaEventRecord(c->ev0, c->stream);
    for (int k0 = 0; k0 < n && e == cudaSuccess; k0 += K.nb) {
        int kk0 = k0, kk1 = std::min(n, k0 + K.nb), nb = kk1 - kk0;
        void *fargs[] = {&a, &kk0, &kk1};
        e = cudaLaunchCooperativeKernel(K.factor, dim3(c->K.coop_grid), dim3(K.block), fargs, 0, c->stream);
        const int cols_right = n + 1 - kk1, rows_below = n - kk1;
        const int g = std::max(1, std::min((n + 1 + 255) / 256, 4 * c->num_sms));
        void *sargs[] = {&a, &kk0, &nb};
        if (e == cudaSuccess) e = cudaLaunchKernel(K.laswp, dim3(g), dim3(256), sargs, 0, c->stream);
        if (e == cudaSuccess && cols_right > 0) {   // four threads a column
            const int cpb = K.u12_block / 4;
            const int gu = std::max(1, std::min((cols_right + cpb - 1) / cpb, 8 * c->num_sms));
            e = cudaLaunchKernel(K.u12, dim3(gu), dim3(K.u12_block), sargs, 0, c->stream);
        }
        if (e == cudaSuccess && rows_below > 0 && cols_right > 0) {
            dim3 tg((cols_right + K.tile - 1) / K.tile, (rows_below + K.tile - 1) / K.tile);
            void *targs[] = {&a, &kk0};
            e = cudaLaunchKernel(K.trail, tg, dim3(256), targs, 0, c->stream);
        }
    }
    if (e == cudaSuccess && solve) {
        void *args[] = {&a};
        e = cudaLaunchCooperativeKernel(K.backsolve, dim3(c->K.coop_grid), dim3(K.block), args, 0, c->stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(c->ev1, c->stream);
    if (e != cudaSuccess) return map_cuda(e);
    rc = read_state(c);
    if (rc) return rc;
    cudaEventElapsedTime(ms, c->ev0, c->ev1);
    *Ad_out = Ad;
    *ldad_out = ldad;
    return LS_OK;
}

}  // namespace

size_t lsi::lu_workspace_bytes(int n, int grid, bool a_on_device) {
    return lu_layout(nullptr, n, grid, !a_on_device).bytes;
}

extern "C" int ls_lu_solve(ls_ctx *c, int n, const double *A, int64_t lda, const double *b, double *x,
                           const ls_opts *opts, ls_info *info) {
    ls_opts o;
    if (opts) o = *opts;
    else ls_opts_default(&o);
    if (!c || n < 0 || lda < n || (n > 0 && (!A || !b || !x))) return LS_ERR_ARG;
    if (o.precision != LS_F64) return LS_ERR_UNSUPPORTED;
    if (cudaSetDevice(c->device) != cudaSuccess) return LS_ERR_CUDA;
    if (n == 0) {
        State z{};
        fill_info(info, z, LS_OK, 0.f, 0.0, 0);
        return LS_OK;
    }
    const bool a_dev = is_device_ptr(A);
    LuLayout L = lu_layout(nullptr, n, c->K.coop_grid, !a_dev);
    int rc = ws_reserve(c, L.bytes);
    if (rc) return rc;
    L = lu_layout(c->ws, n, c->K.coop_grid, !a_dev);
    LuArgs a;
    const double *Ad;
    long long ldad;
    float ms = 0.f;
    rc = lu_run(c, n, A, lda, b, L, a, &Ad, &ldad, true, &ms);
    if (rc) return rc;
    State st = *c->h_st;
    int status = status_from_state(st);
    if (status == LS_BREAKDOWN || status < 0) {
        c->launches_total += (long long)st.launches;
        fill_info(info, st, status, ms, 0.0, (long long)st.launches);
        return status;
    }
    // the true residual r = b - A x (native FP64 product on A)
    MatDesc *hd = &c->h_desc[1];
    memset(hd, 0, sizeof(MatDesc));
    make_tensor_map(hd, DT_F64, Ad, n, n, ldad);
    rc = upload_desc(c, 1);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(L.r, b, sizeof(double) * n, cudaMemcpyDefault, c->stream);
    GemvLaunch GL = gemv_plan(DT_F64, hd->use_tma != 0, EPI_RESID, c->num_sms);
    GemvArgs ga{};
    ga.x = L.x;
    ga.y = L.r;
    ga.b = L.r;
    ga.st = c->st;
    ga.scr = c->scr;
    ga.epi = EPI_RESID;
    ga.fin = FIN_TRUE_RES;
    if (e == cudaSuccess) e = gemv_launch(GL, c->dA + 1, ga, c->stream);
    double bn2 = 0.0;
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return map_cuda(e);
    rc = read_state(c);
    if (rc) return rc;
    st = *c->h_st;
    {   // ||b|| on the host side of the copy already made: one more small read
        std::vector<double> hb(n);
        e = cudaMemcpyAsync(hb.data(), b, sizeof(double) * n, cudaMemcpyDefault, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return map_cuda(e);
        for (int i = 0; i < n; i++) bn2 += hb[i] * hb[i];
    }
    st.bnorm = std::sqrt(bn2);
    st.rnorm = st.true_rnorm;
    status = std::isfinite(st.true_rnorm) ? LS_OK : LS_ERR_NAN;
    if (status == LS_OK) {
        e = cudaMemcpyAsync(x, L.x, sizeof(double) * n, cudaMemcpyDefault, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return map_cuda(e);
    }
    c->launches_total += (long long)st.launches;
    const double nn = (double)n;
    // one read and one write of the trailing block per panel of LU_NB = 32 columns
    fill_info(info, st, status, ms, 16.0 * nn * nn * nn / (3.0 * 32.0), (long long)st.launches);
    return status;
}

extern "C" int ls_lu_factor(ls_ctx *c, int n, const double *A, int64_t lda, const double *b, double *LU,
                            int64_t ldlu, int *ipiv, double *y) {
    if (!c || n < 0 || lda < n || ldlu < n || (n > 0 && (!A || !b || !LU || !ipiv || !y))) return LS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return LS_ERR_CUDA;
    if (n == 0) return LS_OK;
    const bool a_dev = is_device_ptr(A);
    LuLayout L = lu_layout(nullptr, n, c->K.coop_grid, !a_dev);
    int rc = ws_reserve(c, L.bytes);
    if (rc) return rc;
    L = lu_layout(c->ws, n, c->K.coop_grid, !a_dev);
    LuArgs a;
    const double *Ad;
    long long ldad;
    float ms = 0.f;
    rc = lu_run(c, n, A, lda, b, L, a, &Ad, &ldad, false, &ms);
    if (rc) return rc;
    const State st = *c->h_st;
    cudaError_t e = cudaMemcpy2DAsync(LU, ldlu * sizeof(double), L.W, L.ld * sizeof(double), (size_t)n * sizeof(double),
                                      n, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(y, sizeof(double), L.W + n, L.ld * sizeof(double), sizeof(double), n, cudaMemcpyDefault,
                              c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ipiv, L.ipiv, sizeof(int) * n, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return map_cuda(e);
    c->launches_total += (long long)st.launches;
    return status_from_state(st);
}
