// ls_api_internal.h -- the context object and the host-side pieces shared by
// the solver drivers (ls_api.cu, ls_mixed.cu, ls_batch.cu, ls_server.cpp).
#pragma once

#include <cuda_runtime.h>

#include <cstring>
#include <memory>
#include <vector>

#include "ls_device.cuh"
#include "ls_internal.h"

namespace lsi {

struct Prog;

struct GraphCache {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::shared_ptr<Prog> prog;        // host-loop mode
    long long key[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    void reset();
    bool matches(const long long *k) const;
};

class Engine;   // ls_engine_host.h

}  // namespace lsi

struct ls_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    lsi::KrylovKernels K{};
    // fixed device block (allocated by ls_create)
    char *fixed = nullptr;
    lsi::State *st = nullptr;
    lsi::GmresSmall *gm = nullptr;
    lsi::GemvScratch *scr = nullptr;
    lsi::GridBar *bar = nullptr;
    lsi::MatDesc *dA = nullptr;        // [0] solver matrix, [1] kernel-level calls / stored matrix
    double *part = nullptr;
    // pinned host mirrors
    lsi::State *h_st = nullptr;
    lsi::MatDesc *h_desc = nullptr;
    // workspace
    char *ws = nullptr;
    size_t ws_bytes = 0;
    bool ws_user = false;
    // cached executable graphs
    lsi::GraphCache graph_cg, graph_gm, graph_mx, graph_bs, graph_ja, graph_gs, graph_bcg, graph_bgm;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    long long launches_total = 0;
    lsi::Engine *batch = nullptr;
    // set by the tuner while it times a candidate (-1: look the choice up)
    int tune_ks32 = -1, tune_tc = -1;
};

namespace lsi {
size_t align_up(size_t v, size_t a);

// Carves consecutive 256-byte aligned regions out of a base pointer.
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base(static_cast<char *>(b)) {}
    template <class T>
    T *take(size_t count) {
        off = align_up(off, 256);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

// A solver loop recorded for the host instead of a graph (host-loop mode): the
// same kernels with the same arguments, and while-loops whose condition the
// kernels write to State::cond[handle] and the host reads back before every
// pass.  Profilers see each kernel of such a run; graph mode hides the kernels
// inside conditional bodies from them.
struct ProgOp {
    void *func = nullptr;
    int grid = 0, block = 0;
    size_t smem = 0;
    bool coop = false;
    std::vector<char> args;            // parameter bytes at their offsets
    std::vector<size_t> offs;          // parameter offsets
    int handle = -1;                   // >= 0: a while-loop on State::cond[handle]
    std::shared_ptr<struct Prog> body;
};
struct Prog {
    std::vector<ProgOp> ops;
};

// True when LS_HOSTLOOP (or LS_ENGINE_HOSTLOOP) is set to a positive value.
int hostloop_mode();

// Adds nodes one after another to a graph, or ops to a host program.
struct Chain {
    cudaGraph_t g = nullptr;
    Prog *p = nullptr;
    cudaGraphNode_t last = nullptr;
    cudaError_t err = cudaSuccess;
    explicit Chain(cudaGraph_t gr) : g(gr) {}
    explicit Chain(Prog *pr) : p(pr) {}
    Chain() : err(cudaErrorUnknown) {}

    void kernel(void *func, int grid, int block, size_t smem, void **args, bool coop) {
        if (err != cudaSuccess) return;
        if (p) {
            ProgOp op;
            op.func = func; op.grid = grid; op.block = block; op.smem = smem; op.coop = coop;
            for (size_t i = 0;; i++) {
                size_t off = 0, size = 0;
                if (cudaFuncGetParamInfo(func, i, &off, &size) != cudaSuccess) {
                    cudaGetLastError();
                    break;
                }
                if (op.args.size() < off + size) op.args.resize(off + size);
                memcpy(op.args.data() + off, args[i], size);
                op.offs.push_back(off);
            }
            p->ops.push_back(std::move(op));
            return;
        }
        cudaKernelNodeParams kp{};
        kp.func = func;
        kp.gridDim = dim3(grid);
        kp.blockDim = dim3(block);
        kp.sharedMemBytes = (unsigned)smem;
        kp.kernelParams = args;
        cudaGraphNode_t node;
        err = cudaGraphAddKernelNode(&node, g, last ? &last : nullptr, last ? 1 : 0, &kp);
        if (err != cudaSuccess) return;
        if (coop) {
            cudaLaunchAttributeValue v{};
            v.cooperative = 1;
            err = cudaGraphKernelNodeSetAttribute(node, cudaLaunchAttributeCooperative, &v);
        }
        last = node;
    }
    // Appends a while-loop on handle h; returns the chain of its body.
    Chain loop(cudaGraphConditionalHandle h) {
        if (err != cudaSuccess) return Chain();
        if (p) {
            ProgOp op;
            op.handle = (int)h;
            op.body = std::make_shared<Prog>();
            Prog *b = op.body.get();
            p->ops.push_back(std::move(op));
            return Chain(b);
        }
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        err = cudaGraphAddNode(&node, g, last ? &last : nullptr, nullptr, last ? 1 : 0, &np);
        if (err != cudaSuccess) return Chain();
        last = node;
        return Chain(np.conditional.phGraph_out[0]);
    }
};

// The root of a solver loop: a graph, or a host program in host-loop mode.
struct Root {
    cudaGraph_t g = nullptr;
    std::shared_ptr<Prog> prog;
    int handles = 0;
    // Creates the root; returns false on a CUDA error.
    bool create() {
        if (hostloop_mode()) {
            prog = std::make_shared<Prog>();
            return true;
        }
        return cudaGraphCreate(&g, 0) == cudaSuccess;
    }
    // A loop condition: a graph handle (default 1 at every launch), or an
    // index into State::cond (set to 1 by state_init).
    bool handle(cudaGraphConditionalHandle *h) {
        if (prog) {
            if (handles >= LS_COND_SLOTS) return false;
            *h = (cudaGraphConditionalHandle)handles++;
            return true;
        }
        return cudaGraphConditionalHandleCreate(h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    }
    Chain chain() { return prog ? Chain(prog.get()) : Chain(g); }
    void discard() {
        if (g) cudaGraphDestroy(g);
        g = nullptr;
        prog.reset();
        cudaGetLastError();
    }
};

inline void gemv_node(Chain &ch, const GemvLaunch &L, const MatDesc *dA, const GemvArgs &a) {
    // kernelParams must point at storage that outlives the call only until the
    // node is added (the values are copied), so locals are fine.
    const MatDesc *pA = dA;
    GemvArgs aa = a;
    void *args[] = {(void *)&pA, (void *)&aa};
    ch.kernel(L.func, L.grid, L.block, L.smem, args, false);
}

int finish_graph(ls_ctx *c, GraphCache &gc, Root &r, const long long *key);
// Runs a cached solver loop on the context's stream (graph launch or host loop).
int launch_cached(ls_ctx *c, GraphCache &gc);

int is_device_ptr(const void *p);
int map_cuda(cudaError_t e);
int ws_reserve(ls_ctx *c, size_t bytes);
int upload_state(ls_ctx *c);
int upload_desc(ls_ctx *c, int which);
int read_state(ls_ctx *c);
int status_from_state(const State &s);
int copy_in(ls_ctx *c, double *dst, const double *src, size_t count);
void state_init(State *h, int max_iter);
int stage_matrix(ls_ctx *c, int n, const double *A, long long lda, double *stage,
                 long long lda_stage, const double **outA, long long *outlda);
void fill_info(ls_info *info, const State &s, int status, float ms, double bytes, long long launches);
// mixed precision (ls_mixed.cu)
int mixed_cg_solve(ls_ctx *c, int n, const double *A, int64_t lda, const double *b, double *x,
                   const ls_opts *opts, ls_info *info);
size_t mixed_workspace_bytes(int n, const ls_opts *o, bool a_on_device);
// fused small-system solvers (ls_fused.cu): G CTAs of R rows, row length nc
struct FusedPlan {
    int G, R, nc;
    size_t smem;
    bool cluster;        // the grid is one thread-block cluster (else a cooperative grid)
    int h_smem;          // GMRES: the Hessenberg matrix in shared memory
};
// True when a CG / GMRES(m) solve of size n runs as one fused kernel on this
// context's device (A's rows fit in the co-resident CTAs' shared memory).
bool fused_plan(const ls_ctx *c, int method, int n, int m, FusedPlan *p);
size_t fused_workspace_bytes(const FusedPlan &P, int n, int m, bool gmres, bool a_on_device);
int krylov_fused(ls_ctx *c, int method, int n, const double *A, int64_t lda, const double *b, double *x,
                 const ls_opts &o, const FusedPlan &P, ls_info *info);
// block CG workspace (ls_bcg.cu)
size_t bcg_workspace_bytes(int n, int s, int grid, bool a_on_device, bool split);
size_t bgm_workspace_bytes(int n, int s, int m, int grid, bool a_on_device);
size_t lu_workspace_bytes(int n, int grid, bool a_on_device);
// extra resources (batch / server) released by ls_destroy
void extra_destroy(ls_ctx *c);
}  // namespace lsi
