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

struct BatchResources;   // ls_batch.cu

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
    lsi::BatchResources *batch = nullptr;
};

namespace lsi {
size_t align_up(size_t v, size_t a);
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
