// ls_api_internal.h -- the context object and the host-side pieces shared by
// the solver drivers (ls_api.cu, ls_mixed.cu, ls_batch.cu, ls_server.cpp).
#pragma once

#include <cuda_runtime.h>

#include "ls_device.cuh"
#include "ls_internal.h"

namespace lsi {

struct GraphCache {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
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
    lsi::GraphCache graph_cg, graph_gm, graph_mx;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    long long launches_total = 0;
    lsi::Engine *batch = nullptr;
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

// Adds nodes one after another to a graph.
struct Chain {
    cudaGraph_t g;
    cudaGraphNode_t last = nullptr;
    cudaError_t err = cudaSuccess;
    explicit Chain(cudaGraph_t gr) : g(gr) {}

    void kernel(void *func, int grid, int block, size_t smem, void **args, bool coop) {
        if (err != cudaSuccess) return;
        cudaKernelNodeParams p{};
        p.func = func;
        p.gridDim = dim3(grid);
        p.blockDim = dim3(block);
        p.sharedMemBytes = (unsigned)smem;
        p.kernelParams = args;
        cudaGraphNode_t node;
        err = cudaGraphAddKernelNode(&node, g, last ? &last : nullptr, last ? 1 : 0, &p);
        if (err != cudaSuccess) return;
        if (coop) {
            cudaLaunchAttributeValue v{};
            v.cooperative = 1;
            err = cudaGraphKernelNodeSetAttribute(node, cudaLaunchAttributeCooperative, &v);
        }
        last = node;
    }
    // Appends a while-node on handle h; returns its body graph.
    cudaGraph_t loop(cudaGraphConditionalHandle h) {
        if (err != cudaSuccess) return nullptr;
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        err = cudaGraphAddNode(&node, g, last ? &last : nullptr, nullptr, last ? 1 : 0, &np);
        if (err != cudaSuccess) return nullptr;
        last = node;
        return np.conditional.phGraph_out[0];
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

int finish_graph(ls_ctx *c, GraphCache &gc, cudaGraph_t g, const long long *key);

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
// extra resources (batch / server) released by ls_destroy
void extra_destroy(ls_ctx *c);
}  // namespace lsi
