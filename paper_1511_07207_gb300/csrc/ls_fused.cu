// ls_fused.cu -- host side of the fused small-system solvers (k_fused.cu):
// the launch plan, the workspace and the solve.
//
// A CG or GMRES(m) solve in the FP32-pair product mode runs as one
// cooperative kernel when the rows of A fit in the shared memory of the
// co-resident CTAs: G CTAs of R rows each (R <= 32, G at most one per SM),
// each holding 8 R n bytes of A plus its vectors.  On a 152-SM GPU that is n
// up to about 1800.  The default is G = ceil(n / 8) CTAs (8 rows per CTA, a
// row per warp), capped at the SM count; LS_FUSED_CTAS overrides the CTA
// count (for timing other shapes).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "ls_api_internal.h"
#include "ls_internal.h"

namespace lsi {

namespace {
constexpr int FUSED_MAX_ROWS = 32;   // rows per CTA (the per-row loops use one warp)

int env_ctas() {
    const char *s = getenv("LS_FUSED_CTAS");
    return s ? atoi(s) : 0;
}

struct FusedLayout {
    double *x, *b, *xch, *xch2, *part, *H, *Astage;
    unsigned *bar;
    long long lda_stage;
    size_t bytes;
};

FusedLayout fused_layout(void *base, int n, int G, int m, bool gmres, bool stageA) {
    FusedLayout L{};
    const size_t npad = align_up((size_t)std::max(n, 1), 64);
    Carver cv(base);
    L.x = cv.take<double>(npad);
    L.b = cv.take<double>(npad);
    L.xch = cv.take<double>(npad);
    L.xch2 = cv.take<double>(npad);
    L.part = cv.take<double>((size_t)FUSED_PART_SLOTS * G);
    L.H = gmres ? cv.take<double>((size_t)G * (m + 1) * m) : nullptr;
    L.bar = cv.take<unsigned>(64);
    L.lda_stage = (long long)align_up((size_t)std::max(n, 1), 2);
    L.Astage = stageA ? cv.take<double>((size_t)n * L.lda_stage) : nullptr;
    L.bytes = align_up(cv.off, 256);
    return L;
}
}  // namespace

bool fused_plan(const ls_ctx *c, int method, int n, int m, FusedPlan *p) {
    if (n < 1 || (method != LS_METHOD_CG && method != LS_METHOD_GMRES)) return false;
    const bool gmres = method == LS_METHOD_GMRES;
    const FusedKernels K = fused_kernels();
    const void *func = gmres ? K.gmres : K.cg;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, func) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int nc = (n + 3) & ~3;
    const int forced = env_ctas();
    // the default shape, then (if it does not fit) as many CTAs as there are SMs
    const int tries[2] = {forced > 0 ? forced : std::min(c->num_sms, (n + 7) / 8), c->num_sms};
    for (int t = 0; t < 2; t++) {
        const int G0 = std::max(1, std::min(tries[t], c->num_sms));
        const int R = (n + G0 - 1) / G0;
        const int G = (n + R - 1) / R;
        if (R > FUSED_MAX_ROWS) continue;
        const size_t smem = fused_smem_bytes(gmres, R, nc, m);
        if (smem + fa.sharedSizeBytes > (size_t)optin) continue;
        if (set_smem_limit(func, smem) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, FUSED_THREADS, smem) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (per_sm < 1 || G > per_sm * c->num_sms) continue;
        p->G = G;
        p->R = R;
        p->nc = nc;
        p->smem = smem;
        return true;
    }
    return false;
}

size_t fused_workspace_bytes(int n, int G, int m, bool gmres, bool a_on_device) {
    return fused_layout(nullptr, n, G, m, gmres, !a_on_device).bytes;
}

int krylov_fused(ls_ctx *c, int method, int n, const double *A, int64_t lda, const double *b, double *x,
                 const ls_opts &o, const FusedPlan &P, ls_info *info) {
    const bool gmres = method == LS_METHOD_GMRES;
    const int m = o.restart;
    const int max_iter = o.max_iter > 0 ? o.max_iter : 10 * n + 10;
    const bool a_dev = is_device_ptr(A);
    FusedLayout L = fused_layout(nullptr, n, P.G, m, gmres, !a_dev);
    int rc = ws_reserve(c, L.bytes);
    if (rc) return rc;
    L = fused_layout(c->ws, n, P.G, m, gmres, !a_dev);
    const double *Ad;
    long long ldad;
    rc = stage_matrix(c, n, A, lda, L.Astage, L.lda_stage, &Ad, &ldad);
    if (!rc) rc = copy_in(c, L.b, b, n);
    if (!rc && o.x0_given) rc = copy_in(c, L.x, x, n);
    if (rc) return rc;
    State *hs = c->h_st;
    state_init(hs, max_iter);
    hs->m = m;
    hs->reorth = o.reorth;
    rc = upload_state(c);
    if (rc) return rc;
    cudaError_t e = cudaMemsetAsync(L.bar, 0, 64 * sizeof(unsigned), c->stream);
    if (e != cudaSuccess) return map_cuda(e);

    FusedArgs a{};
    a.n = n;
    a.R = P.R;
    a.nc = P.nc;
    a.A = Ad;
    a.lda = ldad;
    a.b = L.b;
    a.x = L.x;
    a.x0_given = o.x0_given;
    a.max_iter = max_iter;
    a.rtol = o.rtol;
    a.m = m;
    a.reorth = o.reorth;
    a.xch = L.xch;
    a.xch2 = L.xch2;
    a.part = L.part;
    a.H = L.H;
    a.bar = L.bar;
    a.st = c->st;
    const FusedKernels K = fused_kernels();
    void *args[] = {&a};
    e = cudaEventRecord(c->ev0, c->stream);
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel(gmres ? K.gmres : K.cg, dim3(P.G), dim3(FUSED_THREADS), args, P.smem,
                                        c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev1, c->stream);
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
    // A streamed from HBM once (the split into shared memory); the products
    // themselves read shared memory
    c->launches_total += (long long)s.launches;
    fill_info(info, s, status, ms, 8.0 * (double)n * n, (long long)s.launches);
    return status;
}

}  // namespace lsi
