// ls_fused.cu -- host side of the fused small-system solvers (k_fused.cu):
// the launch plan, the workspace and the solve.
//
// A CG or GMRES(m) solve in the FP32-pair product mode runs as one kernel
// when the rows of A fit in the shared memory of the CTAs that run it, each
// CTA holding 8 R n bytes of A (R rows) plus its vectors:
//  * cluster form: one thread-block cluster of G = min(16, ceil(n / 8)) CTAs
//    (n up to about 650), which communicate through distributed shared
//    memory and the hardware cluster barrier;
//  * global form: a cooperative grid of G = min(SMs, ceil(n / 8)) CTAs (or
//    one per SM when that is what fits; n up to about 1800 on 152 SMs),
//    which communicate through global memory and a counting grid barrier.
// The cluster form is taken when it fits and the GPU can place such a
// cluster.  LS_FUSED_CTAS forces the global form with that many CTAs (for
// timing and testing other shapes).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "ls_api_internal.h"
#include "ls_internal.h"

namespace lsi {

namespace {
constexpr int FUSED_MAX_ROWS = 64;   // rows per CTA

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

FusedLayout fused_layout(void *base, const FusedPlan &P, int n, int m, bool gmres, bool stageA) {
    FusedLayout L{};
    const size_t npad = align_up((size_t)std::max(n, 1), 64);
    Carver cv(base);
    L.x = cv.take<double>(npad);
    L.b = cv.take<double>(npad);
    L.xch = cv.take<double>(npad);
    L.xch2 = cv.take<double>(npad);
    L.part = cv.take<double>((size_t)FUSED_PART_SLOTS * P.G);
    L.H = gmres && !P.h_smem ? cv.take<double>((size_t)P.G * (m + 1) * m) : nullptr;
    L.bar = cv.take<unsigned>(64);
    L.lda_stage = (long long)align_up((size_t)std::max(n, 1), 2);
    L.Astage = stageA ? cv.take<double>((size_t)n * L.lda_stage) : nullptr;
    L.bytes = align_up(cv.off, 256);
    return L;
}

bool query(cudaError_t e) {
    if (e == cudaSuccess) return true;
    cudaGetLastError();
    return false;
}

// The cluster form for (n, m), if it fits and the GPU can place the cluster.
bool plan_cluster(bool gmres, const void *func, int n, int nc, int m, size_t avail, FusedPlan *p) {
    const int G0 = std::min(FUSED_MAX_CLUSTER, (n + 7) / 8);
    const int R = (n + G0 - 1) / G0;
    const int G = (n + R - 1) / R;
    if (R > FUSED_MAX_ROWS) return false;
    for (int hs = gmres ? 1 : 0; hs >= 0; hs--) {
        const size_t smem = fused_smem_bytes(gmres, R, nc, m, hs != 0);
        if (smem > avail) continue;
        if (!query(set_smem_limit(func, smem))) return false;
        if (G > 8 && !query(cudaFuncSetAttribute(func, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)))
            return false;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = G;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(G);
        cfg.blockDim = dim3(FUSED_THREADS);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (!query(cudaOccupancyMaxActiveClusters(&clusters, func, &cfg)) || clusters < 1) return false;
        p->G = G;
        p->R = R;
        p->nc = nc;
        p->smem = smem;
        p->cluster = true;
        p->h_smem = hs;
        return true;
    }
    return false;
}

// The global form: `want` CTAs, else one per SM.
bool plan_global(const ls_ctx *c, bool gmres, const void *func, int n, int nc, int m, size_t avail, int want,
                 FusedPlan *p) {
    const int tries[2] = {want, c->num_sms};
    for (int t = 0; t < 2; t++) {
        const int G0 = std::max(1, std::min(tries[t], c->num_sms));
        const int R = (n + G0 - 1) / G0;
        const int G = (n + R - 1) / R;
        if (R > FUSED_MAX_ROWS) continue;
        for (int hs = gmres ? 1 : 0; hs >= 0; hs--) {
            const size_t smem = fused_smem_bytes(gmres, R, nc, m, hs != 0);
            if (smem > avail) continue;
            if (!query(set_smem_limit(func, smem))) return false;
            int per_sm = 0;
            if (!query(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, FUSED_THREADS, smem)))
                return false;
            if (per_sm < 1 || G > per_sm * c->num_sms) continue;
            p->G = G;
            p->R = R;
            p->nc = nc;
            p->smem = smem;
            p->cluster = false;
            p->h_smem = hs;
            return true;
        }
    }
    return false;
}
}  // namespace

bool fused_plan(const ls_ctx *c, int method, int n, int m, FusedPlan *p) {
    if (n < 1 || (method != LS_METHOD_CG && method != LS_METHOD_GMRES)) return false;
    const int nc = (n + 3) & ~3;
    if (nc > FUSED_THREADS * FUSED_VEC_REGS) return false;   // the vectors a thread holds
    const bool gmres = method == LS_METHOD_GMRES;
    const FusedKernels K = fused_kernels();
    int optin = 0;
    if (!query(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device))) return false;
    const int forced = env_ctas();
    if (forced <= 0) {
        const void *f = gmres ? K.gmres_cl : K.cg_cl;
        cudaFuncAttributes fa{};
        if (!query(cudaFuncGetAttributes(&fa, f))) return false;
        if ((size_t)optin > fa.sharedSizeBytes && plan_cluster(gmres, f, n, nc, m, optin - fa.sharedSizeBytes, p))
            return true;
    }
    const void *f = gmres ? K.gmres : K.cg;
    cudaFuncAttributes fa{};
    if (!query(cudaFuncGetAttributes(&fa, f)) || (size_t)optin <= fa.sharedSizeBytes) return false;
    const int want = forced > 0 ? forced : std::min(c->num_sms, (n + 7) / 8);
    return plan_global(c, gmres, f, n, nc, m, optin - fa.sharedSizeBytes, want, p);
}

size_t fused_workspace_bytes(const FusedPlan &P, int n, int m, bool gmres, bool a_on_device) {
    return fused_layout(nullptr, P, n, m, gmres, !a_on_device).bytes;
}

int krylov_fused(ls_ctx *c, int method, int n, const double *A, int64_t lda, const double *b, double *x,
                 const ls_opts &o, const FusedPlan &P, ls_info *info) {
    const bool gmres = method == LS_METHOD_GMRES;
    const int m = o.restart;
    const int max_iter = o.max_iter > 0 ? o.max_iter : 10 * n + 10;
    const bool a_dev = is_device_ptr(A);
    FusedLayout L = fused_layout(nullptr, P, n, m, gmres, !a_dev);
    int rc = ws_reserve(c, L.bytes);
    if (rc) return rc;
    L = fused_layout(c->ws, P, n, m, gmres, !a_dev);
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
    cudaError_t e = cudaSuccess;
    if (!P.cluster) e = cudaMemsetAsync(L.bar, 0, 64 * sizeof(unsigned), c->stream);
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
    a.h_smem = P.h_smem;
    a.xch = L.xch;
    a.xch2 = L.xch2;
    a.part = L.part;
    a.H = L.H;
    a.bar = L.bar;
    a.st = c->st;
    const FusedKernels K = fused_kernels();
    void *args[] = {&a};
    e = cudaEventRecord(c->ev0, c->stream);
    if (e == cudaSuccess) {
        if (P.cluster) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = P.G;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(P.G);
            cfg.blockDim = dim3(FUSED_THREADS);
            cfg.dynamicSmemBytes = P.smem;
            cfg.stream = c->stream;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            e = cudaLaunchKernelExC(&cfg, gmres ? K.gmres_cl : K.cg_cl, args);
        } else {
            e = cudaLaunchCooperativeKernel(gmres ? K.gmres : K.cg, dim3(P.G), dim3(FUSED_THREADS), args, P.smem,
                                            c->stream);
        }
    }
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
