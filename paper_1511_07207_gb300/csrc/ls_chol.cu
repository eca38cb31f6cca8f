// ls_chol.cu -- the host driver of the Cholesky method (ls_chol_solve,
// ls_chol_factor): the working matrix [A; b^T] in the workspace, the
// factorization by panels (per panel: the cooperative panel steps, then the
// trailing lower triangle), the back substitution, the residual check.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ls_api_internal.h"

using namespace lsi;

namespace {

struct CholLayout {
    double *W, *Lp, *y, *x, *r, *Astage;
    long long ld, lda_stage;
    size_t bytes;
};

CholLayout chol_layout(void *base, int n, bool stageA) {
    CholLayout L{};
    L.ld = (long long)align_up((size_t)std::max(n, 1), 2);
    L.lda_stage = (long long)align_up((size_t)std::max(n, 1), 2);
    Carver cv(base);
    L.W = cv.take<double>((size_t)(n + 1) * L.ld);
    L.Lp = cv.take<double>((size_t)(n + 1) * 32);
    L.y = cv.take<double>((size_t)std::max(n, 1));
    L.x = cv.take<double>((size_t)std::max(n, 1));
    L.r = cv.take<double>((size_t)std::max(n, 1));
    L.Astage = stageA ? cv.take<double>((size_t)n * L.lda_stage) : nullptr;   // last (see ls_api.cu)
    L.bytes = align_up(cv.off, 256);
    return L;
}

// Stage A and b into [A; b^T] and factor; on return the state holds the
// status (LS_BREAKDOWN, iter = the step, on a pivot that is not positive).
int chol_run(ls_ctx *c, int n, const double *A, long long lda, const double *b, CholLayout &L, CholArgs &a,
             const double **Ad_out, long long *ldad_out, bool solve, float *ms) {
    const double *Ad;
    long long ldad;
    int rc = stage_matrix(c, n, A, lda, L.Astage, L.lda_stage, &Ad, &ldad);
    if (rc) return rc;
    cudaError_t e = cudaMemcpy2DAsync(L.W, L.ld * sizeof(double), Ad, ldad * sizeof(double), (size_t)n * sizeof(double),
                                      n, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(L.W + (long long)n * L.ld, b, sizeof(double) * n, cudaMemcpyDefault, c->stream);
    if (e != cudaSuccess) return map_cuda(e);
    state_init(c->h_st, 0);
    rc = upload_state(c);
    if (rc) return rc;
    a = CholArgs{};
    a.n = n;
    a.W = L.W;
    a.ld = L.ld;
    a.Lp = L.Lp;
    a.y = L.y;
    a.x = L.x;
    a.bar = c->bar;
    a.st = c->st;
    const CholKernels K = chol_kernels();
    e = cudaEventRecord(c->ev0, c->stream);
    for (int k0 = 0; k0 < n && e == cudaSuccess; k0 += K.nb) {
        int kk0 = k0, kk1 = std::min(n, k0 + K.nb), nb = kk1 - kk0;
        void *pargs[] = {&a, &kk0, &kk1};
        e = cudaLaunchCooperativeKernel(K.panel, dim3(c->K.coop_grid), dim3(K.block), pargs, 0, c->stream);
        const int rows = n + 1 - kk1, cols = n - kk1;   // trailing rows (b's included) and columns
        if (e == cudaSuccess && rows > 0 && cols > 0) {
            dim3 tg((cols + K.tile - 1) / K.tile, (rows + K.tile - 1) / K.tile);
            void *targs[] = {&a, &kk0, &nb};
            e = cudaLaunchKernel(K.trail, tg, dim3(256), targs, 0, c->stream);
        }
    }
    if (e == cudaSuccess && solve) {
        e = cudaMemcpyAsync(L.y, L.W + (long long)n * L.ld, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream);
        void *args[] = {&a};
        if (e == cudaSuccess)
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

size_t lsi::chol_workspace_bytes(int n, bool a_on_device) { return chol_layout(nullptr, n, !a_on_device).bytes; }

extern "C" int ls_chol_solve(ls_ctx *c, int n, const double *A, int64_t lda, const double *b, double *x,
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
    CholLayout L = chol_layout(nullptr, n, !a_dev);
    int rc = ws_reserve(c, L.bytes);
    if (rc) return rc;
    L = chol_layout(c->ws, n, !a_dev);
    CholArgs a;
    const double *Ad;
    long long ldad;
    float ms = 0.f;
    rc = chol_run(c, n, A, lda, b, L, a, &Ad, &ldad, true, &ms);
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
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return map_cuda(e);
    rc = read_state(c);
    if (rc) return rc;
    st = *c->h_st;
    double bn2 = 0.0;
    {
        std::vector<double> hb(n);
        e = cudaMemcpyAsync(hb.data(), b, sizeof(double) * n, cudaMemcpyDefault, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return map_cuda(e);
        for (int i = 0; i < n; i++) bn2 += hb[i] * hb[i];
    }
    st.bnorm = std::sqrt(bn2);
    st.rnorm = st.true_rnorm;
    st.iter = 0;
    status = std::isfinite(st.true_rnorm) ? LS_OK : LS_ERR_NAN;
    if (status == LS_OK) {
        e = cudaMemcpyAsync(x, L.x, sizeof(double) * n, cudaMemcpyDefault, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return map_cuda(e);
    }
    c->launches_total += (long long)st.launches;
    const double nn = (double)n;
    // one read and one write of the trailing lower triangle per panel of 32 columns
    fill_info(info, st, status, ms, 16.0 * nn * nn * nn / (6.0 * 32.0), (long long)st.launches);
    return status;
}

extern "C" int ls_chol_factor(ls_ctx *c, int n, const double *A, int64_t lda, const double *b, double *Lout,
                              int64_t ldl, double *y, int *step) {
    if (!c || n < 0 || lda < n || ldl < n || (n > 0 && (!A || !b || !Lout || !y))) return LS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return LS_ERR_CUDA;
    if (step) *step = -1;
    if (n == 0) return LS_OK;
    const bool a_dev = is_device_ptr(A);
    CholLayout L = chol_layout(nullptr, n, !a_dev);
    int rc = ws_reserve(c, L.bytes);
    if (rc) return rc;
    L = chol_layout(c->ws, n, !a_dev);
    CholArgs a;
    const double *Ad;
    long long ldad;
    float ms = 0.f;
    rc = chol_run(c, n, A, lda, b, L, a, &Ad, &ldad, false, &ms);
    if (rc) return rc;
    const State st = *c->h_st;
    const CholKernels K = chol_kernels();
    void *zargs[] = {&a};
    cudaError_t e = cudaLaunchKernel(K.zero_upper, dim3(std::max(1, std::min(4 * c->num_sms, (n * n + 255) / 256))),
                                     dim3(256), zargs, 0, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(Lout, ldl * sizeof(double), L.W, L.ld * sizeof(double), (size_t)n * sizeof(double), n,
                              cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(y, L.W + (long long)n * L.ld, sizeof(double) * n, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return map_cuda(e);
    c->launches_total += (long long)st.launches + 1;
    const int status = status_from_state(st);
    if (step && status == LS_BREAKDOWN) *step = st.iter;
    return status;
}
