// ls_api.cu -- the C ABI (include/ls.h): contexts, workspace, staging of host
// or device buffers, and the device-resident solve drivers.
//
// The paper's host flow (section "Parallel implementation ... using CUDA":
// allocate, copy in, choose the grid, run the kernel, copy out) becomes: copy
// or borrow the inputs once, upload a small state block, launch ONE CUDA
// graph whose while-nodes run the whole iteration on the device (the kernels
// set the loop conditions), and read back the solution and the state.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>

#include "ls_api_internal.h"

using namespace lsi;

// ============================================================================
// small utilities
// ============================================================================
namespace lsi {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int is_device_ptr(const void *p) {
    if (!p) return 0;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int map_cuda(cudaError_t e) { return e == cudaSuccess ? LS_OK : (e == cudaErrorMemoryAllocation ? LS_ERR_NOMEM : LS_ERR_CUDA); }

cudaError_t set_smem_limit(const void *func, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> done;   // (kernel, device) -> limit set
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    auto it = done.find({func, dev});
    if (it != done.end() && it->second >= smem) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) done[{func, dev}] = smem;
    return e;
}


// ---- workspace ----------------------------------------------------------------
int ws_reserve(ls_ctx *c, size_t bytes) {
    if (bytes <= c->ws_bytes) return LS_OK;
    if (c->ws_user) return LS_ERR_NOMEM;
    if (c->ws) cudaFree(c->ws);
    c->ws = nullptr;
    c->ws_bytes = 0;
    c->graph_cg.reset();
    c->graph_gm.reset();
    c->graph_mx.reset();
    c->graph_bs.reset();
    c->graph_ja.reset();
    c->graph_gs.reset();
    c->graph_bcg.reset();
    c->graph_bgm.reset();
    cudaError_t e = cudaMalloc(&c->ws, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return LS_ERR_NOMEM;
    }
    c->ws_bytes = bytes;
    return LS_OK;
}

// ---- graphs ---------------------------------------------------------------------
void GraphCache::reset() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    prog.reset();
    memset(key, 0, sizeof(key));
}

bool GraphCache::matches(const long long *k) const {
    return (exec || prog) && memcmp(key, k, sizeof(key)) == 0;
}

int hostloop_mode() {
    static const int mode = [] {
        const char *e = getenv("LS_HOSTLOOP");
        if (!e) e = getenv("LS_ENGINE_HOSTLOOP");
        return e ? atoi(e) : 0;
    }();
    return mode > 0;
}

int finish_graph(ls_ctx *c, GraphCache &gc, Root &r, const long long *key) {
    (void)c;
    if (r.prog) {
        gc.reset();
        gc.prog = r.prog;
        memcpy(gc.key, key, sizeof(gc.key));
        return LS_OK;
    }
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, r.g, 0);
    if (e != cudaSuccess) {
        r.discard();
        return LS_ERR_CUDA;
    }
    gc.reset();
    gc.graph = r.g;
    gc.exec = ex;
    r.g = nullptr;
    memcpy(gc.key, key, sizeof(gc.key));
    return LS_OK;
}

// Host-loop execution of a recorded program: kernels in order, each while-loop
// re-entered while the device-side condition it reads back is set.
static cudaError_t run_prog(ls_ctx *c, const Prog &p) {
    constexpr long long LOOP_LIMIT = 100000000;   // far above any iteration limit
    for (const ProgOp &op : p.ops) {
        cudaError_t e = cudaSuccess;
        if (op.handle >= 0) {
            for (long long it = 0; it < LOOP_LIMIT; it++) {
                unsigned go = 0;
                e = cudaMemcpyAsync(&go, &c->st->cond[op.handle], sizeof(unsigned),
                                    cudaMemcpyDeviceToHost, c->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
                if (e != cudaSuccess || !go) break;
                e = run_prog(c, *op.body);
                if (e != cudaSuccess) break;
            }
        } else {
            std::vector<void *> args(op.offs.size());
            for (size_t i = 0; i < op.offs.size(); i++)
                args[i] = const_cast<char *>(op.args.data()) + op.offs[i];
            e = op.coop ? cudaLaunchCooperativeKernel(op.func, dim3(op.grid), dim3(op.block),
                                                      args.data(), op.smem, c->stream)
                        : cudaLaunchKernel(op.func, dim3(op.grid), dim3(op.block), args.data(),
                                           op.smem, c->stream);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int launch_cached(ls_ctx *c, GraphCache &gc) {
    if (gc.prog) return map_cuda(run_prog(c, *gc.prog));
    return map_cuda(cudaGraphLaunch(gc.exec, c->stream));
}

// ---- state upload / download -------------------------------------------------------
void state_init(State *h, int max_iter) {
    memset(h, 0, sizeof(State));
    h->max_iter = max_iter;
    h->hostloop = hostloop_mode();
    for (int i = 0; i < LS_COND_SLOTS; i++) h->cond[i] = 1;
}

int upload_state(ls_ctx *c) {
    return map_cuda(cudaMemcpyAsync(c->st, c->h_st, sizeof(State), cudaMemcpyHostToDevice, c->stream));
}

int upload_desc(ls_ctx *c, int which) {
    return map_cuda(cudaMemcpyAsync(c->dA + which, c->h_desc + which, sizeof(MatDesc),
                                    cudaMemcpyHostToDevice, c->stream));
}

int read_state(ls_ctx *c) {
    cudaError_t e = cudaMemcpyAsync(c->h_st, c->st, sizeof(State), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return map_cuda(e);
}

int status_from_state(const State &s) {
    if (s.err & ERRB_TIMEOUT) return LS_ERR_TIMEOUT;
    if (s.err & ERRB_NAN) return LS_ERR_NAN;
    if (s.status == LS_OK || s.status == LS_NOT_CONVERGED || s.status == LS_BREAKDOWN) return s.status;
    return LS_NOT_CONVERGED;
}

// Input staging: copy a vector (host or device) into a device buffer.
int copy_in(ls_ctx *c, double *dst, const double *src, size_t count) {
    if (count == 0) return LS_OK;
    return map_cuda(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDefault, c->stream));
}

// A row-major n x n FP64 matrix: borrow it if it lives on the device,
// otherwise copy it into `stage` with a 16-byte multiple leading dimension.
int stage_matrix(ls_ctx *c, int n, const double *A, long long lda, double *stage,
                 long long lda_stage, const double **outA, long long *outlda) {
    if (is_device_ptr(A)) {
        *outA = A;
        *outlda = lda;
        return LS_OK;
    }
    // a contiguous A (lda equal to the staging pitch) as one plain copy
    cudaError_t e = lda == lda_stage
                        ? cudaMemcpyAsync(stage, A, (size_t)n * lda * sizeof(double), cudaMemcpyHostToDevice, c->stream)
                        : cudaMemcpy2DAsync(stage, lda_stage * sizeof(double), A, lda * sizeof(double),
                                            n * sizeof(double), n, cudaMemcpyHostToDevice, c->stream);
    *outA = stage;
    *outlda = lda_stage;
    return map_cuda(e);
}

}  // namespace lsi

// ============================================================================
// ABI: options, context, workspace
// ============================================================================
extern "C" int ls_opts_default(ls_opts *o) {
    if (!o) return LS_ERR_ARG;
    o->rtol = 1e-10;
    o->max_iter = 0;          // 0 = method default
    o->restart = 30;
    o->precision = LS_F64;
    o->refine = LS_REFINE_FCG;
    o->inner_iters = 25;
    o->inner_rtol = 0.0;
    o->x0_given = 0;
    o->reorth = 0;
    o->f64_matvec = 0;
    o->deflate = 1;
    o->fused = 1;
    return LS_OK;
}

extern "C" const char *ls_strerror(int s) {
    switch (s) {
        case LS_OK: return "converged";
        case LS_NOT_CONVERGED: return "iteration limit reached before the tolerance";
        case LS_BREAKDOWN: return "breakdown (non-positive curvature or zero rotation pivot)";
        case LS_ERR_ARG: return "invalid argument";
        case LS_ERR_NOMEM: return "out of device memory / workspace too small";
        case LS_ERR_CUDA: return "CUDA runtime error";
        case LS_ERR_TIMEOUT: return "an on-device wait timed out";
        case LS_ERR_BUSY: return "server queue full or no capacity";
        case LS_ERR_NAN: return "NaN or Inf in the input or the iteration";
        case LS_ERR_UNSUPPORTED: return "unsupported option combination or device";
        default: return "unknown status";
    }
}

extern "C" int ls_create(ls_ctx **out, int device, void *stream) {
    if (!out) return LS_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return LS_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return LS_ERR_CUDA;
    cudaDeviceProp pr;
    if (cudaGetDeviceProperties(&pr, device) != cudaSuccess) return LS_ERR_CUDA;
    if (!(pr.major == 10 && pr.minor == 3)) return LS_ERR_UNSUPPORTED;
    ls_ctx *c = new (std::nothrow) ls_ctx();
    if (!c) return LS_ERR_NOMEM;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(stream);
    c->num_sms = pr.multiProcessorCount;
    c->K = krylov_kernels(c->num_sms);
    // fixed device block: state, small GMRES state, GEMV scratch, barrier, descriptors, partials
    Carver cv(nullptr);
    cv.take<State>(1);
    cv.take<GmresSmall>(1);
    cv.take<GemvScratch>(1);
    cv.take<GridBar>(1);
    cv.take<MatDesc>(2);
    cv.take<double>((size_t)PART_SLOTS * MAX_GRID);
    size_t fixed = align_up(cv.off, 256);
    if (cudaMalloc(&c->fixed, fixed) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return LS_ERR_NOMEM;
    }
    Carver cf(c->fixed);
    c->st = cf.take<State>(1);
    c->gm = cf.take<GmresSmall>(1);
    c->scr = cf.take<GemvScratch>(1);
    c->bar = cf.take<GridBar>(1);
    c->dA = cf.take<MatDesc>(2);
    c->part = cf.take<double>((size_t)PART_SLOTS * MAX_GRID);
    cudaError_t e = cudaMemsetAsync(c->fixed, 0, fixed, c->stream);
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_st, sizeof(State));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_desc, 2 * sizeof(MatDesc));
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ls_destroy(c);
        return LS_ERR_CUDA;
    }
    *out = c;
    return LS_OK;
}

extern "C" int ls_destroy(ls_ctx *c) {
    if (!c) return LS_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    c->graph_cg.reset();
    c->graph_gm.reset();
    c->graph_mx.reset();
    c->graph_bs.reset();
    c->graph_ja.reset();
    c->graph_gs.reset();
    c->graph_bcg.reset();
    c->graph_bgm.reset();
    extra_destroy(c);
    if (c->ws && !c->ws_user) cudaFree(c->ws);
    if (c->fixed) cudaFree(c->fixed);
    if (c->h_st) cudaFreeHost(c->h_st);
    if (c->h_desc) cudaFreeHost(c->h_desc);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    delete c;
    return LS_OK;
}

extern "C" int ls_set_workspace(ls_ctx *c, void *ptr, size_t bytes) {
    if (!c) return LS_ERR_ARG;
    if (ptr && ((uintptr_t)ptr & 255)) return LS_ERR_ARG;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->ws && !c->ws_user) cudaFree(c->ws);
    c->graph_cg.reset();
    c->graph_gm.reset();
    c->graph_mx.reset();
    c->graph_bs.reset();
    c->graph_ja.reset();
    c->graph_gs.reset();
    c->graph_bcg.reset();
    c->graph_bgm.reset();
    c->ws = static_cast<char *>(ptr);
    c->ws_bytes = ptr ? bytes : 0;
    c->ws_user = ptr != nullptr;
    return LS_OK;
}

extern "C" long long ls_kernel_launches(ls_ctx *c) { return c ? c->launches_total : 0; }

// ============================================================================
// FP64 CG / GMRES
// ============================================================================
namespace lsi {

struct F64Layout {
    double *x, *b, *r, *p, *q, *V, *Astage;
    double *rh, *vv, *s, *t;   // BiCGSTAB
    float *Ahi, *Alo;    // the FP32 pair of A (double-single products)
    float *Thi, *Tlo;    // Gauss-Seidel: inverses of the 64 x 64 diagonal blocks (FP32 pairs)
    unsigned *gflags;    // Gauss-Seidel: 2 x nblk publication flags
    void *gmaps;         // Gauss-Seidel: 4 tensor maps (pair of A, pair of the T_I^-1)
    float *gpanel;       // Gauss-Seidel: the chain CTA's M_{I,w} = T_I^-1 A_{I,I-w}, one contiguous panel
    long long npad, ldv, lda_stage, ld32;
    int nblk;
    size_t bytes;
};

F64Layout f64_layout(void *base, int n, int m, bool gmres, bool stageA, bool split, bool gs) {
    F64Layout L{};
    L.npad = (long long)align_up((size_t)std::max(n, 1), 64);
    L.ldv = L.npad;
    L.lda_stage = (long long)align_up((size_t)std::max(n, 1), 2);
    Carver cv(base);
    L.x = cv.take<double>(L.npad);
    L.b = cv.take<double>(L.npad);
    L.r = cv.take<double>(L.npad);
    L.p = cv.take<double>(L.npad);
    L.q = cv.take<double>(L.npad);
    L.V = gmres ? cv.take<double>((size_t)L.ldv * (m + 1)) : nullptr;
    L.rh = cv.take<double>(L.npad);
    L.vv = cv.take<double>(L.npad);
    L.s = cv.take<double>(L.npad);
    L.t = cv.take<double>(L.npad);
    L.ld32 = (long long)align_up((size_t)std::max(n, 1), 4);
    L.Ahi = split ? cv.take<float>((size_t)n * L.ld32) : nullptr;
    L.Alo = split ? cv.take<float>((size_t)n * L.ld32) : nullptr;
    L.nblk = (std::max(n, 1) + 63) / 64;
    L.Thi = gs ? cv.take<float>((size_t)L.nblk * 64 * 64) : nullptr;
    L.Tlo = gs ? cv.take<float>((size_t)L.nblk * 64 * 64) : nullptr;
    L.gflags = gs ? cv.take<unsigned>((size_t)2 * L.nblk) : nullptr;
    L.gmaps = gs ? static_cast<void *>(cv.take<CUtensorMap>(4)) : nullptr;
    if (gs) {
        const GsKernels G = gs_kernels();
        L.gpanel = cv.take<float>((size_t)L.nblk * G.panel_tiles_per_block * G.panel_tile_floats);
    } else {
        L.gpanel = nullptr;
    }
    // last, so that every pointer a cached graph holds is the same whether
    // A is staged or borrowed
    L.Astage = stageA ? cv.take<double>((size_t)n * L.lda_stage) : nullptr;
    L.bytes = align_up(cv.off, 256);
    return L;
}

int check_common(ls_ctx *c, int n, const double *A, long long lda, const double *b, double *x,
                 const ls_opts *o) {
    if (!c || n < 0 || lda < n || (n > 0 && (!A || !b || !x)) || !o) return LS_ERR_ARG;
    if (!(o->rtol >= 0.0) || o->max_iter < 0) return LS_ERR_ARG;
    return LS_OK;
}

void fill_info(ls_info *info, const State &s, int status, float ms, double bytes, long long launches) {
    if (!info) return;
    info->status = status;
    info->iters = s.iter;
    info->outer_iters = s.cycles;
    info->rel_res = s.bnorm > 0 ? s.rnorm / s.bnorm : 0.0;
    info->true_rel_res = s.bnorm > 0 ? s.true_rnorm / s.bnorm : 0.0;
    info->time_ms = ms;
    info->bytes_moved = bytes;
    info->launches = launches;
}

Vecs make_vecs(ls_ctx *c, const F64Layout &L, int n, double rtol) {
    Vecs v{};
    v.n = n;
    v.x = L.x;
    v.b = L.b;
    v.r = L.r;
    v.p = L.p;
    v.q = L.q;
    v.V = L.V;
    v.ldv = L.ldv;
    v.rh = L.rh;
    v.vv = L.vv;
    v.s = L.s;
    v.t = L.t;
    v.part = c->part;
    v.bar = c->bar;
    v.st = c->st;
    v.gm = c->gm;
    v.rtol = rtol;
    return v;
}

}  // namespace lsi

// Builds: [resid GEMV if x0] cg_init, while(outer){ while(inner){GEMV, update}, resid GEMV, check }
static int build_cg_graph(ls_ctx *c, const Vecs &v, const GemvLaunch &L, int x0_given,
                          const long long *key) {
    Root R;
    if (!R.create()) return LS_ERR_CUDA;
    cudaGraphConditionalHandle ho, hi;
    if (!R.handle(&ho) || !R.handle(&hi)) {
        R.discard();
        return LS_ERR_CUDA;
    }
    Chain top = R.chain();
    const MatDesc *dA = c->dA;
    if (x0_given) {
        GemvArgs a{};
        a.x = v.x; a.y = v.r; a.b = v.b; a.st = v.st; a.scr = c->scr;
        a.epi = EPI_RESID; a.fin = FIN_TRUE_RES;
        gemv_node(top, L, dA, a);
    }
    {
        Vecs vv = v;
        int x0 = x0_given;
        void *args[] = {&vv, &x0, &ho, &hi};
        top.kernel(c->K.cg_init, c->K.coop_grid, c->K.block, 0, args, true);
    }
    Chain outer = top.loop(ho);
    Chain inner = outer.loop(hi);
    {
        GemvArgs a{};
        a.x = v.p; a.y = v.q; a.z = v.p; a.st = v.st; a.scr = c->scr;
        a.epi = EPI_DOT; a.fin = FIN_CG_ALPHA;
        gemv_node(inner, L, dA, a);
        Vecs vv = v;
        void *args[] = {&vv, &hi};
        inner.kernel(c->K.cg_update, c->K.coop_grid, c->K.block, 0, args, true);
    }
    {
        GemvArgs a{};
        a.x = v.x; a.y = v.q; a.b = v.b; a.st = v.st; a.scr = c->scr;
        a.epi = EPI_RESID; a.fin = FIN_TRUE_RES;
        gemv_node(outer, L, dA, a);
        Vecs vv = v;
        void *args[] = {&vv, &ho, &hi};
        outer.kernel(c->K.cg_check, c->K.coop_grid, c->K.block, 0, args, false);
    }
    if (top.err != cudaSuccess || inner.err != cudaSuccess || outer.err != cudaSuccess) {
        R.discard();
        return LS_ERR_CUDA;
    }
    return finish_graph(c, c->graph_cg, R, key);
}

// Builds: [resid GEMV if x0] bs_init, while(outer){ while(inner){GEMV v = A p (r^.v -> alpha),
// bs_s, GEMV t = A s (t.s), bs_update}, resid GEMV, bs_check }
static int build_bicgstab_graph(ls_ctx *c, const Vecs &v, const GemvLaunch &L, int x0_given,
                                const long long *key) {
    Root R;
    if (!R.create()) return LS_ERR_CUDA;
    cudaGraphConditionalHandle ho, hi;
    if (!R.handle(&ho) || !R.handle(&hi)) {
        R.discard();
        return LS_ERR_CUDA;
    }
    Chain top = R.chain();
    const MatDesc *dA = c->dA;
    if (x0_given) {
        GemvArgs a{};
        a.x = v.x; a.y = v.r; a.b = v.b; a.st = v.st; a.scr = c->scr;
        a.epi = EPI_RESID; a.fin = FIN_TRUE_RES;
        gemv_node(top, L, dA, a);
    }
    {
        Vecs vv = v;
        int x0 = x0_given;
        void *args[] = {&vv, &x0, &ho, &hi};
        top.kernel(c->K.bs_init, c->K.coop_grid, c->K.block, 0, args, true);
    }
    Chain outer = top.loop(ho);
    Chain inner = outer.loop(hi);
    {
        GemvArgs a{};
        a.x = v.p; a.y = v.vv; a.z = v.rh; a.st = v.st; a.scr = c->scr;
        a.epi = EPI_DOT; a.fin = FIN_BS_ALPHA;
        gemv_node(inner, L, dA, a);
        Vecs vv = v;
        void *args[] = {&vv, &hi};
        inner.kernel(c->K.bs_s, c->K.coop_grid, c->K.block, 0, args, true);
        GemvArgs a2{};
        a2.x = v.s; a2.y = v.t; a2.z = v.s; a2.st = v.st; a2.scr = c->scr;
        a2.epi = EPI_DOT; a2.fin = FIN_STORE;          // st->dot = t.s
        gemv_node(inner, L, dA, a2);
        void *args2[] = {&vv, &hi};
        inner.kernel(c->K.bs_update, c->K.coop_grid, c->K.block, 0, args2, true);
    }
    {
        GemvArgs a{};
        a.x = v.x; a.y = v.q; a.b = v.b; a.st = v.st; a.scr = c->scr;
        a.epi = EPI_RESID; a.fin = FIN_TRUE_RES;
        gemv_node(outer, L, dA, a);
        Vecs vv = v;
        void *args[] = {&vv, &ho, &hi};
        outer.kernel(c->K.bs_check, c->K.coop_grid, c->K.block, 0, args, true);
    }
    if (top.err != cudaSuccess || inner.err != cudaSuccess || outer.err != cudaSuccess) {
        R.discard();
        return LS_ERR_CUDA;
    }
    return finish_graph(c, c->graph_bs, R, key);
}

// Builds: ja_init, while(loop){ Jacobi GEMV (next iterate, ||b - A x||, stop test), ja_next }
static int build_jacobi_graph(ls_ctx *c, const Vecs &v, const GemvLaunch &L, int x0_given,
                              const long long *key) {
    Root R;
    if (!R.create()) return LS_ERR_CUDA;
    cudaGraphConditionalHandle hl;
    if (!R.handle(&hl)) {
        R.discard();
        return LS_ERR_CUDA;
    }
    Chain top = R.chain();
    {
        Vecs vv = v;
        int x0 = x0_given;
        void *args[] = {&vv, &x0, &hl};
        top.kernel(c->K.ja_init, c->K.coop_grid, c->K.block, 0, args, true);
    }
    Chain loop = top.loop(hl);
    {
        GemvArgs a{};
        a.x = v.x; a.y = v.q; a.b = v.b; a.z = v.p; a.st = v.st; a.scr = c->scr;
        a.epi = EPI_JACOBI; a.fin = FIN_JACOBI;
        gemv_node(loop, L, c->dA, a);
        Vecs vv = v;
        void *args[] = {&vv, &hl};
        loop.kernel(c->K.ja_next, c->K.coop_grid, c->K.block, 0, args, false);
    }
    if (top.err != cudaSuccess || loop.err != cudaSuccess) {
        R.discard();
        return LS_ERR_CUDA;
    }
    return finish_graph(c, c->graph_ja, R, key);
}

// Builds: ja_init, while(loop){ resid GEMV (||b - A x||, stop test), gs_trsv ((D + L) d = r, x += d) }
static int build_gs_graph(ls_ctx *c, const Vecs &v, const F64Layout &L, const GemvLaunch &GL, int x0_given,
                          const long long *key) {
    Root R;
    if (!R.create()) return LS_ERR_CUDA;
    cudaGraphConditionalHandle hl;
    if (!R.handle(&hl)) {
        R.discard();
        return LS_ERR_CUDA;
    }
    Chain top = R.chain();
    {
        Vecs vv = v;
        int x0 = x0_given;
        void *args[] = {&vv, &x0, &hl};
        top.kernel(c->K.ja_init, c->K.coop_grid, c->K.block, 0, args, true);
    }
    Chain loop = top.loop(hl);
    {
        GemvArgs a{};
        a.x = v.x; a.y = v.r; a.b = v.b; a.st = v.st; a.scr = c->scr;
        a.epi = EPI_RESID; a.fin = FIN_JACOBI;
        gemv_node(loop, GL, c->dA, a);
        GsArgs g{};
        g.n = v.n;
        g.r = v.r;
        g.x = v.x;
        g.delta = reinterpret_cast<float2 *>(v.p);   // n FP32 pairs in an n-double vector
        g.u = reinterpret_cast<float2 *>(v.q);
        g.tmaps = static_cast<const CUtensorMap *>(L.gmaps);
        g.panel = L.gpanel;
        g.flagD = L.gflags;
        g.flagU = L.gflags + L.nblk;
        g.bar = v.bar;
        g.st = v.st;
        const GsKernels G = gs_kernels();
        void *args[] = {&g, &hl};
        loop.kernel(G.trsv, c->K.coop_grid, G.trsv_block, G.trsv_smem, args, true);
    }
    if (top.err != cudaSuccess || loop.err != cudaSuccess) {
        R.discard();
        return LS_ERR_CUDA;
    }
    return finish_graph(c, c->graph_gs, R, key);
}

// Builds: gm_init, while(outer){ resid GEMV, gm_start, while(inner){GEMV, arnoldi}, gm_finish }
static int build_gmres_graph(ls_ctx *c, const Vecs &v, const GemvLaunch &L, int x0_given,
                             const long long *key) {
    Root R;
    if (!R.create()) return LS_ERR_CUDA;
    cudaGraphConditionalHandle ho, hi;
    if (!R.handle(&ho) || !R.handle(&hi)) {
        R.discard();
        return LS_ERR_CUDA;
    }
    const MatDesc *dA = c->dA;
    Chain top = R.chain();
    {
        Vecs vv = v;
        int x0 = x0_given;
        void *args[] = {&vv, &x0, &ho};
        top.kernel(c->K.gm_init, c->K.coop_grid, c->K.block, 0, args, true);
    }
    Chain outer = top.loop(ho);
    {
        GemvArgs a{};
        a.x = v.x; a.y = v.q; a.b = v.b; a.st = v.st; a.scr = c->scr;
        a.epi = EPI_RESID; a.fin = FIN_TRUE_RES;
        gemv_node(outer, L, dA, a);
        Vecs vv = v;
        void *args[] = {&vv, &ho, &hi};
        outer.kernel(c->K.gm_start, c->K.coop_grid, c->K.block, 0, args, false);
    }
    Chain inner = outer.loop(hi);
    {
        GemvArgs a{};
        a.x = v.V; a.y = v.V; a.kptr = &v.st->k; a.kstride = v.ldv; a.kyoff = 1;
        a.st = v.st; a.scr = c->scr;
        a.epi = EPI_NRM; a.fin = FIN_WNORM0;
        gemv_node(inner, L, dA, a);
        Vecs vv = v;
        void *args[] = {&vv, &hi};
        inner.kernel(c->K.gm_arnoldi, c->K.coop_grid, c->K.block, 0, args, true);
    }
    {
        Vecs vv = v;
        void *args[] = {&vv};
        outer.kernel(c->K.gm_finish, c->K.coop_grid, c->K.block, 0, args, true);
    }
    if (top.err != cudaSuccess || inner.err != cudaSuccess || outer.err != cudaSuccess) {
        R.discard();
        return LS_ERR_CUDA;
    }
    return finish_graph(c, c->graph_gm, R, key);
}

static int krylov_f64(ls_ctx *c, int method, int n, const double *A, int64_t lda, const double *b,
                      double *x, const ls_opts *opts, ls_info *info) {
    ls_opts o;
    if (opts) o = *opts;
    else ls_opts_default(&o);
    int rc = check_common(c, n, A, lda, b, x, &o);
    if (rc) return rc;
    if (method == LS_METHOD_GMRES && (o.restart < 1 || o.restart > LS_MAX_RESTART)) return LS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return LS_ERR_CUDA;
    if (n == 0) {
        State s{};
        fill_info(info, s, LS_OK, 0.f, 0.0, 0);
        return LS_OK;
    }
    if (o.f64_matvec == 0 && o.fused) {   // small n: the whole solve as one kernel
        FusedPlan P;
        if (fused_plan(c, method, n, o.restart, &P)) return krylov_fused(c, method, n, A, lda, b, x, o, P, info);
    }
    const int m = o.restart;
    const int max_iter = o.max_iter > 0 ? o.max_iter : 10 * n + 10;
    const bool a_dev = is_device_ptr(A);
    const bool split = o.f64_matvec == 0;
    const bool gs = method == LS_METHOD_GAUSS_SEIDEL;
    const bool pair = split || gs;     // the Gauss-Seidel sweep reads the pair whatever the GEMV
    if (gs && (n + 63) / 64 > gs_kernels().max_owned * (c->K.coop_grid - 1)) return LS_ERR_UNSUPPORTED;
    F64Layout L = f64_layout(nullptr, n, m, method == LS_METHOD_GMRES, !a_dev, pair, gs);
    rc = ws_reserve(c, L.bytes);
    if (rc) return rc;
    L = f64_layout(c->ws, n, m, method == LS_METHOD_GMRES, !a_dev, pair, gs);

    // stage inputs
    const double *Ad;
    long long ldad;
    rc = stage_matrix(c, n, A, lda, L.Astage, L.lda_stage, &Ad, &ldad);
    if (!rc) rc = copy_in(c, L.b, b, n);
    if (!rc && o.x0_given) rc = copy_in(c, L.x, x, n);
    if (rc) return rc;
    MatDesc *hd = &c->h_desc[0];
    memset(hd, 0, sizeof(MatDesc));
    if (split) make_tensor_map_ds(hd, L.Ahi, L.Alo, n, n, L.ld32);
    else make_tensor_map(hd, DT_F64, Ad, n, n, ldad);
    rc = upload_desc(c, 0);
    State *hs = c->h_st;
    state_init(hs, max_iter);
    hs->m = m;
    hs->reorth = o.reorth;
    if (!rc) rc = upload_state(c);
    if (rc) return rc;

    Vecs v = make_vecs(c, L, n, o.rtol);
    const int dt = split ? DT_DS : DT_F64;
    GemvLaunch GL = gemv_plan(dt, hd->use_tma != 0, EPI_DOT, c->num_sms);
    long long key[8] = {method, n, (long long)(uintptr_t)c->ws, L.ldv, o.x0_given, hd->use_tma,
                        (long long)(uintptr_t)c->stream, dt};
    GraphCache &gc = method == LS_METHOD_CG         ? c->graph_cg
                     : method == LS_METHOD_BICGSTAB ? c->graph_bs
                     : method == LS_METHOD_JACOBI   ? c->graph_ja
                     : gs                           ? c->graph_gs
                                                    : c->graph_gm;
    if (!gc.matches(key)) {
        rc = method == LS_METHOD_CG         ? build_cg_graph(c, v, GL, o.x0_given, key)
             : method == LS_METHOD_BICGSTAB ? build_bicgstab_graph(c, v, GL, o.x0_given, key)
             : method == LS_METHOD_JACOBI   ? build_jacobi_graph(c, v, GL, o.x0_given, key)
             : gs                           ? build_gs_graph(c, v, L, GL, o.x0_given, key)
                                            : build_gmres_graph(c, v, GL, o.x0_given, key);
        if (rc) return rc;
    }
    cudaError_t e = cudaEventRecord(c->ev0, c->stream);
    if (e == cudaSuccess && method == LS_METHOD_JACOBI) {   // D^-1 into v.p (A may be borrowed per call)
        int nn = n;
        long long la = ldad;
        const double *Ap = Ad;
        double *dv = v.p;
        State *stp = c->st;
        void *args[] = {&nn, &Ap, &la, &dv, &stp};
        const int g = std::min((n + c->K.block - 1) / c->K.block, 4 * c->num_sms);
        e = cudaLaunchKernel(c->K.ja_diag, dim3(g), dim3(c->K.block), args, 0, c->stream);
    }
    if (e == cudaSuccess && gs) {   // flags zeroed; T_I^-1 of the diagonal blocks (A may be borrowed per call)
        alignas(64) CUtensorMap maps[4];
        if (!gs_encode_maps(maps, L.Ahi, L.Alo, n, L.ld32, L.Thi, L.Tlo, L.nblk)) return LS_ERR_UNSUPPORTED;
        e = cudaMemcpyAsync(L.gmaps, maps, sizeof(maps), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);   // maps is on this stack frame
        if (e == cudaSuccess) e = cudaMemsetAsync(L.gflags, 0, sizeof(unsigned) * 2 * L.nblk, c->stream);
        const GsKernels G = gs_kernels();
        int nn = n;
        long long la = ldad;
        const double *Ap = Ad;
        float *th = L.Thi, *tl = L.Tlo;
        State *stp = c->st;
        void *args[] = {&nn, &Ap, &la, &th, &tl, &stp};
        const int g = std::min(L.nblk, 8 * c->num_sms);
        if (e == cudaSuccess) e = cudaLaunchKernel(G.tinv, dim3(g), dim3(G.tinv_block), args, 0, c->stream);
    }
    // the FP32 pair of A: one pass over A, timed as part of the solve
    if (e == cudaSuccess && pair) e = split_f64_launch(n, n, Ad, ldad, L.Ahi, L.Alo, L.ld32, c->num_sms, c->stream);
    if (e == cudaSuccess && gs) {   // the chain's panel, from the pair and the T_I^-1
        const GsKernels G = gs_kernels();
        int nn = n;
        const float *ah = L.Ahi, *al = L.Alo, *th = L.Thi, *tl = L.Tlo;
        long long ld = L.ld32;
        float *pn = L.gpanel;
        State *stp = c->st;
        void *args[] = {&nn, &ah, &al, &ld, &th, &tl, &pn, &stp};
        const int g = std::min(L.nblk * G.panel_tiles_per_block, 8 * c->num_sms);
        e = cudaLaunchKernel(G.panel, dim3(g), dim3(G.panel_block), args, G.panel_smem, c->stream);
    }
    if (e != cudaSuccess) return map_cuda(e);
    rc = launch_cached(c, gc);
    if (rc) return rc;
    e = cudaEventRecord(c->ev1, c->stream);
    if (e != cudaSuccess) return map_cuda(e);
    rc = read_state(c);
    if (rc) return rc;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    const State &s = *hs;
    int status = status_from_state(s);
    // x back to the caller (host or device)
    if (status >= 0) {
        e = cudaMemcpyAsync(x, L.x, n * sizeof(double), cudaMemcpyDefault, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return map_cuda(e);
    }
    // matrix passes: method products + true-residual checks (+ the x0 residual)
    double passes;
    State sc = s;
    if (method == LS_METHOD_JACOBI) {
        passes = s.iter + (s.status == LS_BREAKDOWN ? 1 : 0);
    } else if (gs) {   // a residual GEMV per test, the lower half of A per sweep
        passes = s.status == LS_BREAKDOWN ? 1.0 : s.iter + 0.5 * std::max(s.iter - 1, 0);
    } else if (method == LS_METHOD_CG || method == LS_METHOD_BICGSTAB) {
        passes = s.iter + s.cycles + (o.x0_given ? 1 : 0);
    } else {
        passes = s.total + s.cycles + 1;
        sc.iter = s.total;
        sc.rnorm = s.est;   // the Givens estimate of the last step
    }
    c->launches_total += (long long)s.launches;
    fill_info(info, sc, status, ms, passes * (double)n * n * 8.0, (long long)s.launches);
    return status;
}

extern "C" int ls_cg_solve(ls_ctx *c, int n, const double *A, int64_t lda, const double *b,
                           double *x, const ls_opts *opts, ls_info *info) {
    if (opts && opts->precision != LS_F64) return mixed_cg_solve(c, n, A, lda, b, x, opts, info);
    return krylov_f64(c, LS_METHOD_CG, n, A, lda, b, x, opts, info);
}

extern "C" int ls_gmres_solve(ls_ctx *c, int n, const double *A, int64_t lda, const double *b,
                              double *x, const ls_opts *opts, ls_info *info) {
    if (opts && opts->precision != LS_F64) return LS_ERR_UNSUPPORTED;
    return krylov_f64(c, LS_METHOD_GMRES, n, A, lda, b, x, opts, info);
}

extern "C" int ls_bicgstab_solve(ls_ctx *c, int n, const double *A, int64_t lda, const double *b,
                                 double *x, const ls_opts *opts, ls_info *info) {
    if (opts && opts->precision != LS_F64) return LS_ERR_UNSUPPORTED;
    return krylov_f64(c, LS_METHOD_BICGSTAB, n, A, lda, b, x, opts, info);
}

extern "C" int ls_jacobi_solve(ls_ctx *c, int n, const double *A, int64_t lda, const double *b,
                               double *x, const ls_opts *opts, ls_info *info) {
    if (opts && opts->precision != LS_F64) return LS_ERR_UNSUPPORTED;
    return krylov_f64(c, LS_METHOD_JACOBI, n, A, lda, b, x, opts, info);
}

extern "C" int ls_gauss_seidel_solve(ls_ctx *c, int n, const double *A, int64_t lda, const double *b,
                                     double *x, const ls_opts *opts, ls_info *info) {
    if (opts && opts->precision != LS_F64) return LS_ERR_UNSUPPORTED;
    return krylov_f64(c, LS_METHOD_GAUSS_SEIDEL, n, A, lda, b, x, opts, info);
}

extern "C" int ls_workspace_size(ls_ctx *c, int method, int n, int nrhs, const ls_opts *opts,
                                 int a_on_device, size_t *bytes) {
    if (!c || !bytes || n < 0 || nrhs < 1) return LS_ERR_ARG;
    ls_opts o;
    if (opts) o = *opts;
    else ls_opts_default(&o);
    if (o.precision != LS_F64 && method == LS_METHOD_CG) {
        *bytes = mixed_workspace_bytes(n, &o, a_on_device != 0);
        return LS_OK;
    }
    if (method == LS_METHOD_LU) {
        *bytes = lu_workspace_bytes(n, c->K.coop_grid, a_on_device != 0);
        return LS_OK;
    }
    if (method == LS_METHOD_CHOLESKY) {
        *bytes = chol_workspace_bytes(n, a_on_device != 0);
        return LS_OK;
    }
    if (method == LS_METHOD_BLOCK_GMRES) {
        if (nrhs > BGM_MAX_S || o.restart < 1 || o.restart * nrhs > BGM_MAX_MS) return LS_ERR_ARG;
        *bytes = bgm_workspace_bytes(n, nrhs, o.restart, c->K.coop_grid, a_on_device != 0);
        return LS_OK;
    }
    if (method == LS_METHOD_BLOCK_CG) {
        if (nrhs > BCG_MAX_S) return LS_ERR_ARG;
        *bytes = bcg_workspace_bytes(n, nrhs, c->K.coop_grid, a_on_device != 0, o.f64_matvec == 0);
        return LS_OK;
    }
    const bool gs = method == LS_METHOD_GAUSS_SEIDEL;
    FusedPlan P;
    if ((method == LS_METHOD_CG || method == LS_METHOD_GMRES) && o.f64_matvec == 0 && o.fused &&
        fused_plan(c, method, n, o.restart, &P)) {
        *bytes = fused_workspace_bytes(P, n, o.restart, method == LS_METHOD_GMRES, a_on_device != 0);
        return LS_OK;
    }
    *bytes = f64_layout(nullptr, n, o.restart, method == LS_METHOD_GMRES, !a_on_device, o.f64_matvec == 0 || gs, gs)
                 .bytes;
    return LS_OK;
}

// ============================================================================
// kernel-level entry points
// ============================================================================
// The matrix descriptor of a kernel-level call (LS_F64_PAIR: hi rows, then lo rows).
static void kernel_desc(MatDesc *hd, int dtype, const void *A, int rows, int cols, long long lda) {
    memset(hd, 0, sizeof(MatDesc));
    if (dtype == DT_DS) {
        const float *hi = static_cast<const float *>(A);
        make_tensor_map_ds(hd, hi, hi + (long long)rows * lda, rows, cols, lda);
    } else {
        make_tensor_map(hd, dtype, A, rows, cols, lda);
    }
}

extern "C" int ls_split_f64(ls_ctx *c, int rows, int cols, const double *A, int64_t lda, float *pair,
                            int64_t ldp) {
    if (!c || rows < 0 || cols < 0 || lda < cols || ldp < cols || (ldp & 3)) return LS_ERR_ARG;
    if (rows == 0 || cols == 0) return LS_OK;
    if (!A || !pair) return LS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return LS_ERR_CUDA;
    cudaError_t e = split_f64_launch(rows, cols, A, lda, pair, pair + (long long)rows * ldp, ldp, c->num_sms,
                                     c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) c->launches_total += 1;
    return map_cuda(e);
}

extern "C" int ls_gemv(ls_ctx *c, int dtype, int rows, int cols, const void *A, int64_t lda,
                       const float *scale, const void *x, void *y) {
    if (!c || rows < 0 || cols < 0 || lda < cols || dtype < 0 || dtype > 4) return LS_ERR_ARG;
    if (dtype == DT_DS && (lda & 3)) return LS_ERR_ARG;
    if (rows == 0) return LS_OK;
    if (!A || !x || !y || (dtype == DT_FP8 && !scale)) return LS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return LS_ERR_CUDA;
    MatDesc *hd = &c->h_desc[1];
    kernel_desc(hd, dtype, A, rows, cols, lda);
    hd->scale = scale;
    int rc = upload_desc(c, 1);
    if (rc) return rc;
    state_init(c->h_st, 0);
    rc = upload_state(c);
    if (rc) return rc;
    GemvLaunch L = gemv_plan(dtype, hd->use_tma != 0, EPI_STORE, c->num_sms);
    GemvArgs a{};
    a.x = x;
    a.y = y;
    a.st = c->st;
    a.scr = c->scr;
    a.epi = EPI_STORE;
    a.fin = FIN_STORE;
    cudaError_t e = gemv_launch(L, c->dA + 1, a, c->stream);
    if (e != cudaSuccess) return map_cuda(e);
    rc = read_state(c);
    if (rc) return rc;
    c->launches_total += (long long)c->h_st->launches;
    if (c->h_st->err & ERRB_TIMEOUT) return LS_ERR_TIMEOUT;
    return LS_OK;
}

extern "C" int ls_gemv_timed(ls_ctx *c, int dtype, int rows, int cols, const void *A, int64_t lda,
                             const float *scale, const void *x, void *y, int reps,
                             double *ms_per_launch) {
    if (!c || rows <= 0 || cols <= 0 || lda < cols || dtype < 0 || dtype > 4 || reps < 1 ||
        !ms_per_launch || (dtype == DT_DS && (lda & 3)))
        return LS_ERR_ARG;
    if (!A || !x || !y || (dtype == DT_FP8 && !scale)) return LS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return LS_ERR_CUDA;
    MatDesc *hd = &c->h_desc[1];
    kernel_desc(hd, dtype, A, rows, cols, lda);
    hd->scale = scale;
    int rc = upload_desc(c, 1);
    if (rc) return rc;
    state_init(c->h_st, 0);
    rc = upload_state(c);
    if (rc) return rc;
    GemvLaunch L = gemv_plan(dtype, hd->use_tma != 0, EPI_STORE, c->num_sms);
    GemvArgs a{};
    a.x = x;
    a.y = y;
    a.st = c->st;
    a.scr = c->scr;
    a.epi = EPI_STORE;
    a.fin = FIN_STORE;
    cudaError_t e = gemv_launch(L, c->dA + 1, a, c->stream);   // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(c->ev0, c->stream);
    for (int i = 0; i < reps && e == cudaSuccess; i++) e = gemv_launch(L, c->dA + 1, a, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev1, c->stream);
    if (e != cudaSuccess) return map_cuda(e);
    rc = read_state(c);
    if (rc) return rc;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    *ms_per_launch = ms / reps;
    c->launches_total += (long long)c->h_st->launches;
    if (c->h_st->err & ERRB_TIMEOUT) return LS_ERR_TIMEOUT;
    return LS_OK;
}

extern "C" int ls_quantize(ls_ctx *c, int dtype, int rows, int cols, const double *A, int64_t lda,
                           void *Q, int64_t ldq, float *scale) {
    if (!c || rows < 0 || cols < 0 || lda < cols || ldq < cols) return LS_ERR_ARG;
    if (dtype != DT_BF16 && dtype != DT_FP8 && dtype != DT_F32) return LS_ERR_ARG;
    if (rows == 0) return LS_OK;
    if (!A || !Q || (dtype == DT_FP8 && !scale)) return LS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return LS_ERR_CUDA;
    cudaError_t e = quantize_launch(dtype, rows, cols, A, lda, Q, ldq, scale, c->num_sms, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) c->launches_total += 1;
    return map_cuda(e);
}

extern "C" int ls_selftest_waits(ls_ctx *c, int which) {
    if (!c || which < 0 || which > 1) return LS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return LS_ERR_CUDA;
    GridBar *bar = nullptr;   // a barrier of its own: the context's stays consistent
    cudaError_t e = cudaSuccess;
    if (which == 1) {
        e = cudaMalloc(&bar, 64);
        if (e == cudaSuccess) e = cudaMemsetAsync(bar, 0, 64, c->stream);
    }
    state_init(c->h_st, 0);
    int rc = e == cudaSuccess ? upload_state(c) : map_cuda(e);
    if (!rc) rc = map_cuda(selftest_launch(which, bar, c->st, c->stream));
    if (!rc) rc = read_state(c);
    if (bar) {
        cudaStreamSynchronize(c->stream);
        cudaFree(bar);
    }
    if (rc) return rc;
    return status_from_state(*c->h_st);
}
