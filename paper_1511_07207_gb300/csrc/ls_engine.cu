// ls_engine.cu -- host side of the batched / served solve engine (ls_engine.h)
// and the ls_batch_solve entry point.
//
// The engine owns the slot and task tables in device memory and one CUDA
// graph: while (any slot active and ticks < limit) { eng_red; eng_prod;
// eng_vec }.  The kernels read the table sizes from a device
// block, so the same graph serves any set of resident slots; the batched
// solver runs it to completion, the server (ls_server.cpp) runs it a few
// ticks at a time between admissions.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ls_api_internal.h"
#include "ls_engine.h"
#include "ls_engine_host.h"

namespace lsi {

// ---- per-slot state initialisation and result collection ---------------------
__global__ void eng_init_state_kernel(SlotState *st, int first, int count) {
    for (int q = blockIdx.x; q < count; q += gridDim.x) {
        SlotState &S = st[first + q];
        int *w = reinterpret_cast<int *>(&S);
        for (size_t e = threadIdx.x; e < sizeof(SlotState) / sizeof(int); e += blockDim.x) w[e] = 0;
        __syncthreads();
        if (threadIdx.x == 0) S.phase = PH_ADMIT;
    }
}

__global__ void eng_collect_kernel(const SlotDesc *desc, const SlotState *st, SlotResult *out,
                                   int first, int count) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x) {
        const SlotState &S = st[first + q];
        const SlotDesc &D = desc[first + q];
        SlotResult r;
        r.status = S.phase == PH_DONE ? S.status : LS_NOT_CONVERGED;
        r.inner = S.inner_total;
        r.outer = S.outer;
        r.done = S.phase == PH_DONE;
        double worst = 0.0;
        for (int j = 0; j < E_MAXS; j++) {
            const double rel = j < D.s && S.bnorm[j] > 0.0 ? S.rn[j] / S.bnorm[j] : 0.0;
            r.colres[j] = rel;
            if (j < D.s) worst = rel > worst || rel != rel ? rel : worst;
        }
        r.rel_res = worst;
        out[q] = r;
    }
}

// ---- buffer sizes ---------------------------------------------------------------
SlotSizes slot_sizes(const ls_ctx *c, int n, int s, int method, int m) {
    SlotSizes z{};
    z.sp = s <= 4 ? 4 : s <= 8 ? 8 : s <= 16 ? 16 : 32;   // the product kernel's widths
    const TuneChoice ch = tune_choice(c, n, s);
    z.ks32 = ch.ks32;
    z.tc = z.sp >= 16 ? ch.tc : 0;
    z.ld32 = a32_ncols(n);
    z.lda_stage = (n + 1) / 2 * 2;
    const size_t nsp = (size_t)n * z.sp;
    z.bytes = 0;
    auto add = [&](size_t b) { z.bytes += align_up(b, 256); };
    const SlotTasks tk = slot_tasks(n, z.sp, z.ks32);
    add((size_t)n * z.ld32 * 4);              // A32
    add((size_t)n * z.ld32 * 4);              // A32lo
    add(nsp * 8); add(nsp * 8); add(nsp * 8); // X, B, R
    add(nsp * 4); add(nsp * 4);               // Xh, Xl
    add(nsp * 4); add(nsp * 4); add(nsp * 4); // Rf, Z, Q
    if (tk.kc32 > 1) add((size_t)tk.kc32 * nsp * 4);                // Yk
    if (tk.kc64 > 1) add((size_t)tk.kc64 * nsp * 8);                // Rk
    add((size_t)(tk.rb32 > 0 ? tk.rb32 : 1) * sizeof(int));         // ticket
    if (method == LS_METHOD_CG) add(2 * nsp * 4);                   // P
    else { add(2 * nsp * 4); add((size_t)(m + 1) * nsp * 4); }      // W, V
    z.stageA = align_up((size_t)n * z.lda_stage * 8, 256);
    z.stageBX = align_up((size_t)n * s * 8, 256);
    return z;
}

void slot_carve(SlotDesc &D, const SlotSizes &z, char *base, int n, int s, int method, int m) {
    Carver cv(base);
    const size_t nsp = (size_t)n * z.sp;
    D.n = n;
    D.s = s;
    D.sp = z.sp;
    D.method = method;
    D.m = m;
    const SlotTasks tk = slot_tasks(n, z.sp, z.ks32);
    D.ks32 = z.ks32;
    D.tc = z.tc;
    D.A32 = cv.take<float>((size_t)n * z.ld32);
    D.A32lo = cv.take<float>((size_t)n * z.ld32);
    D.ld32 = z.ld32;
    D.X = cv.take<double>(nsp);
    D.B = cv.take<double>(nsp);
    D.R = cv.take<double>(nsp);
    D.Xh = cv.take<float>(nsp);
    D.Xl = cv.take<float>(nsp);
    D.Rf = cv.take<float>(nsp);
    D.Z = cv.take<float>(nsp);
    D.Q = cv.take<float>(nsp);
    D.Yk = tk.kc32 > 1 ? cv.take<float>((size_t)tk.kc32 * nsp) : nullptr;
    D.Rk = tk.kc64 > 1 ? cv.take<double>((size_t)tk.kc64 * nsp) : nullptr;
    D.ticket = cv.take<int>(tk.rb32 > 0 ? tk.rb32 : 1);
    D.P = nullptr;
    D.W = nullptr;
    D.V = nullptr;
    if (method == LS_METHOD_CG) {
        D.P = cv.take<float>(2 * nsp);
    } else {
        D.W = cv.take<float>(2 * nsp);
        D.V = cv.take<float>((size_t)(m + 1) * nsp);
    }
}

// ---- the engine ---------------------------------------------------------------------
Engine::~Engine() { release(); }

void Engine::release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (dmem) cudaFree(dmem);
    exec = nullptr;
    graph = nullptr;
    dmem = nullptr;
    cap_slots = cap32 = capb = cap64 = capv = 0;
}

int Engine::reserve(ls_ctx *ctx, int slots, int n32, int nrb, int n64, int nv) {
    c = ctx;
    if (dmem && slots <= cap_slots && n32 <= cap32 && nrb <= capb && n64 <= cap64 && nv <= capv)
        return LS_OK;
    release();
    cap_slots = std::max(slots, 1);
    cap32 = std::max(n32, 1);
    capb = std::max(nrb, 1);
    cap64 = std::max(n64, 1);
    capv = std::max(nv, 1);
    Carver cv(nullptr);
    auto layout = [&](Carver &k) {
        dE = k.take<EngineDev>(1);
        hE.desc = k.take<SlotDesc>(cap_slots);
        hE.st = k.take<SlotState>(cap_slots);
        hE.gm = k.take<SlotGm>(cap_slots);
        hE.t32 = k.take<Task>(cap32);
        hE.t64 = k.take<Task>(cap64);
        hE.tv = k.take<Task>(capv);
        hE.part32 = k.take<double>((size_t)capb * E_PS * 32);
        hE.part64 = k.take<double>((size_t)capb * 32);
        hE.partv = k.take<double>((size_t)capv * 32);
        hE.order = k.take<int>(cap_slots);
        hE.work[0] = k.take<int>((size_t)cap64 + cap32 + capv);
        hE.work[1] = k.take<int>((size_t)cap64 + cap32 + capv);
        hE.wres = cap32;
        hE.wvec = cap32 + cap64;
        hE.active = k.take<int>(A_SIZE);
        hE.launches = k.take<unsigned long long>(1);
        bsrc = k.take<const double *>(cap_slots);
        ldb = k.take<long long>(cap_slots);
        xdst = k.take<double *>((size_t)cap_slots * E_MAXS);
        ldx = k.take<long long>((size_t)cap_slots * E_MAXS);
        fslot = k.take<int>((size_t)cap_slots * E_MAXS);
        fc0 = k.take<int>((size_t)cap_slots * E_MAXS);
        fk = k.take<int>((size_t)cap_slots * E_MAXS);
        results = k.take<SlotResult>(cap_slots);
    };
    layout(cv);
    dbytes = align_up(cv.off, 256);
    if (cudaMalloc(&dmem, dbytes) != cudaSuccess) {
        cudaGetLastError();
        dmem = nullptr;
        cap_slots = 0;
        return LS_ERR_NOMEM;
    }
    Carver real(dmem);
    layout(real);
    if (cudaMemsetAsync(dmem, 0, dbytes, c->stream) != cudaSuccess) return LS_ERR_CUDA;
    K = engine_kernels();
    grid_prod = c->num_sms;                 // one warp-specialised CTA per SM
    grid_vec = 2 * c->num_sms;
    set_smem_limit(K.prod, K.prod_smem);
    return build_graph();
}

int Engine::build_graph() {
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) return LS_ERR_CUDA;
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
        cudaGetLastError();
        return LS_ERR_CUDA;
    }
    Chain top(graph);
    Chain b = top.loop(h);
    if (top.err != cudaSuccess) {
        cudaGetLastError();
        return LS_ERR_CUDA;
    }
    const EngineDev *p = dE;
    {
        void *args[] = {(void *)&p, (void *)&h};
        b.kernel(K.red, cap_slots, K.red_threads, 0, args, false);
    }
    {
        void *args[] = {(void *)&p};
        b.kernel(K.prod, grid_prod, K.prod_threads, K.prod_smem, args, false);
        b.kernel(K.vec, grid_vec, K.vec_threads, 0, args, false);
    }
    if (b.err != cudaSuccess) {
        cudaGetLastError();
        return LS_ERR_CUDA;
    }
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        return LS_ERR_CUDA;
    }
    return LS_OK;
}

// Task tables from the slot sizes.  Packed: each slot's tasks follow the
// previous slot's (the batched solver, whose slot set never changes).  With
// fixed regions sized for max_n rows per slot, a slot's task indices -- and so
// the partial sums it left in the previous tick -- never move when other
// slots are admitted or retired (the server); unused entries have slot = -1.
void Engine::set_tasks(std::vector<SlotDesc> &hd, int fixed_max_n) {
    h32.clear();
    h64.clear();
    hv.clear();
    nb32 = 0;
    const SlotTasks per = slot_tasks(fixed_max_n, 32, E_KS32_MIN);   // the most tasks a slot can have
    const Task none{-1, 0, 0, 0, 0, 0, 0, 0};
    auto region = [&](std::vector<Task> &tab, int q, int per_slot, int &t0) {
        if (fixed_max_n) {
            t0 = q * per_slot;
            tab.resize((size_t)(q + 1) * per_slot, none);
        } else {
            t0 = (int)tab.size();
        }
    };
    auto put = [&](std::vector<Task> &tab, int idx, const Task &t) {
        if (fixed_max_n) tab[idx] = t;
        else tab.push_back(t);
    };
    // packed tables list the costliest slots first (tasks are claimed in
    // table order, so the long ones start early and the short ones fill in)
    std::vector<int> &order = h_order;
    order.resize(hd.size());
    for (int q = 0; q < (int)hd.size(); q++) order[q] = q;
    if (!fixed_max_n)
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return (double)hd[a].n * hd[a].n * hd[a].sp > (double)hd[b].n * hd[b].n * hd[b].sp;
        });
    for (int q : order) {
        SlotDesc &D = hd[q];
        const int n = D.n > 0 ? D.n : 0;
        const SlotTasks tk = slot_tasks(n, D.sp, D.ks32);
        const int ks = D.ks32;
        // FP32 product: row block x K chunk; row blocks own the partial dots
        region(h32, q, per.t32, D.t32);
        D.b32 = fixed_max_n ? q * per.rb32 : nb32;
        D.nb32 = tk.rb32;
        D.n32 = 0;
        for (int b = 0; b < tk.rb32; b++)
            for (int kc = 0; kc < tk.kc32; kc++) {
                const Task t{q, b * E_RB32, std::min(n, (b + 1) * E_RB32), kc * ks,
                             std::min(n, (kc + 1) * ks), kc, D.b32 + b, 0};
                put(h32, D.t32 + D.n32, t);
                D.n32++;
            }
        if (!fixed_max_n) nb32 += tk.rb32;
        // refinement residual: row block x K chunk (the same row blocks)
        region(h64, q, per.t64, D.t64);
        D.n64 = 0;
        const int k64 = ks64(D.sp);
        for (int b = 0; b < tk.rb32; b++)
            for (int kc = 0; kc < tk.kc64; kc++) {
                const Task t{q, b * E_RB32, std::min(n, (b + 1) * E_RB32), kc * k64,
                             std::min(n, (kc + 1) * k64), kc, D.b32 + b, 0};
                put(h64, D.t64 + D.n64, t);
                D.n64++;
            }
        region(hv, q, per.tv, D.tv);
        D.nv = 0;
        const int rv = rbv(D.sp);
        for (int r = 0; r < n; r += rv, D.nv++)
            put(hv, D.tv + D.nv, Task{q, r, std::min(n, r + rv), 0, 0, 0, 0, 0});
    }
    if (fixed_max_n) nb32 = (int)hd.size() * per.rb32;
}

int Engine::upload(const std::vector<SlotDesc> &hd, int tick_limit, bool tables) {
    hE.nslots = (int)hd.size();
    hE.n32 = (int)h32.size();
    hE.n64 = (int)h64.size();
    hE.nv = (int)hv.size();
    hE.tick_limit = tick_limit;
    cudaError_t e = cudaSuccess;
    if (!tables) {   // same slot set: only the loop counters are reset
        e = cudaMemcpyAsync(dE, &hE, sizeof(EngineDev), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(hE.active, 0, A_SIZE * sizeof(int), c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        return map_cuda(e);
    }
    if (!hd.empty())
        e = cudaMemcpyAsync(hE.desc, hd.data(), hd.size() * sizeof(SlotDesc), cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess && !h32.empty())
        e = cudaMemcpyAsync(hE.t32, h32.data(), h32.size() * sizeof(Task), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !h64.empty())
        e = cudaMemcpyAsync(hE.t64, h64.data(), h64.size() * sizeof(Task), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !hv.empty())
        e = cudaMemcpyAsync(hE.tv, hv.data(), hv.size() * sizeof(Task), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !h_order.empty())
        e = cudaMemcpyAsync(hE.order, h_order.data(), h_order.size() * sizeof(int), cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dE, &hE, sizeof(EngineDev), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(hE.active, 0, A_SIZE * sizeof(int), c->stream);
    // the host copies above read pageable memory: make them complete before
    // the host vectors can change
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return map_cuda(e);
}

int Engine::init_slots(int first, int count) {
    if (count <= 0) return LS_OK;
    eng_init_state_kernel<<<std::min(count, 1024), 256, 0, c->stream>>>(hE.st, first, count);
    return map_cuda(cudaGetLastError());
}

int Engine::admit(int first, int count, const std::vector<const double *> &bs,
                  const std::vector<long long> &lb) {
    if (count <= 0) return LS_OK;
    cudaError_t e = cudaMemcpyAsync(bsrc + first, bs.data(), count * sizeof(double *),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ldb + first, lb.data(), count * sizeof(long long), cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return map_cuda(e);
    const EngineDev *p = dE;
    const double *const *bp = bsrc + first;
    const long long *lp = ldb + first;
    void *args[] = {(void *)&p, (void *)&bp, (void *)&lp, (void *)&first, (void *)&count};
    e = cudaLaunchKernel(K.admit, dim3(64, std::min(count, 1024)), dim3(256), args, 0, c->stream);
    return map_cuda(e);
}

int Engine::finish(const std::vector<FinishItem> &items) {
    const int count = (int)items.size();
    if (count <= 0) return LS_OK;
    if (count > cap_slots * E_MAXS) return LS_ERR_ARG;
    std::vector<double *> xs(count);
    std::vector<long long> lx(count);
    std::vector<int> sl(count), c0(count), kk(count);
    for (int i = 0; i < count; i++) {
        xs[i] = items[i].x;
        lx[i] = items[i].ldx;
        sl[i] = items[i].slot;
        c0[i] = items[i].c0;
        kk[i] = items[i].k;
    }
    cudaError_t e = cudaMemcpyAsync(xdst, xs.data(), count * sizeof(double *), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ldx, lx.data(), count * sizeof(long long), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(fslot, sl.data(), count * sizeof(int), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(fc0, c0.data(), count * sizeof(int), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(fk, kk.data(), count * sizeof(int), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return map_cuda(e);
    const EngineDev *p = dE;
    double *const *xp = xdst;
    const long long *lp = ldx;
    const int *sp = fslot, *cp = fc0, *kp = fk;
    void *args[] = {(void *)&p, (void *)&xp, (void *)&lp, (void *)&sp, (void *)&cp, (void *)&kp, (void *)&count};
    e = cudaLaunchKernel(K.finish, dim3(64, std::min(count, 1024)), dim3(256), args, 0, c->stream);
    return map_cuda(e);
}

int Engine::collect(int first, int count, std::vector<SlotResult> &out) {
    out.resize(count);
    if (count <= 0) return LS_OK;
    eng_collect_kernel<<<(count + 127) / 128, 128, 0, c->stream>>>(hE.desc, hE.st, results + first,
                                                                   first, count);
    int err = 0;
    cudaError_t e = cudaMemcpyAsync(out.data(), results + first, count * sizeof(SlotResult),
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&err, hE.active + A_ERR, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && err) return LS_ERR_TIMEOUT;
    return map_cuda(e);
}

// LS_HOSTLOOP=1 (or LS_ENGINE_HOSTLOOP=1) runs the same kernels from a host
// loop instead of the graph's while-node (the loop condition is read back every
// tick), which lets profilers see each kernel; the value 2 also times every
// kernel with CUDA events and prints the totals to stderr.
int Engine::run() {
    const char *env = getenv("LS_HOSTLOOP");
    if (!env) env = getenv("LS_ENGINE_HOSTLOOP");
    const int mode = env ? atoi(env) : 0;
    if (mode <= 0) return map_cuda(cudaGraphLaunch(exec, c->stream));
    hE.host_loop = 1;
    cudaError_t e = cudaMemcpyAsync(dE, &hE, sizeof(EngineDev), cudaMemcpyHostToDevice, c->stream);
    cudaGraphConditionalHandle none = 0;
    const EngineDev *p = dE;
    void *args_red[] = {(void *)&p, (void *)&none};
    void *args[] = {(void *)&p};
    cudaEvent_t ev[4];
    for (int i = 0; i < 4; i++) cudaEventCreate(&ev[i]);
    double tot[3] = {0, 0, 0};
    long long ticks = 0;
    int go = 1;
    while (e == cudaSuccess && go) {
        if (mode == 2) cudaEventRecord(ev[0], c->stream);
        e = cudaLaunchKernel(K.red, dim3(cap_slots), dim3(K.red_threads), args_red, 0, c->stream);
        if (mode == 2) cudaEventRecord(ev[1], c->stream);
        if (e == cudaSuccess)
            e = cudaLaunchKernel(K.prod, dim3(grid_prod), dim3(K.prod_threads), args, K.prod_smem, c->stream);
        if (mode == 2) cudaEventRecord(ev[2], c->stream);
        if (e == cudaSuccess)
            e = cudaLaunchKernel(K.vec, dim3(grid_vec), dim3(K.vec_threads), args, 0, c->stream);
        if (mode == 2) cudaEventRecord(ev[3], c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&go, hE.active + 4, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (mode == 2 && e == cudaSuccess)
            for (int i = 0; i < 3; i++) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
                tot[i] += ms;
            }
        ticks++;
    }
    for (int i = 0; i < 4; i++) cudaEventDestroy(ev[i]);
    if (mode == 2)
        fprintf(stderr, "engine ticks %lld  red %.3f ms  prod %.3f ms  vec %.3f ms\n", ticks, tot[0],
                tot[1], tot[2]);
    hE.host_loop = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(dE, &hE, sizeof(EngineDev), cudaMemcpyHostToDevice, c->stream);
    return map_cuda(e);
}

unsigned long long Engine::launches() {
    unsigned long long v = 0;
    cudaMemcpyAsync(&v, hE.launches, sizeof(v), cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    return v;
}

void extra_destroy(ls_ctx *c) {
    delete c->batch;
    c->batch = nullptr;
}

}  // namespace lsi

using namespace lsi;

// ============================================================================
// ls_batch_solve
// ============================================================================
extern "C" int ls_batch_solve(ls_ctx *c, int count, const ls_system *sys, ls_info *infos) {
    if (!c || count < 0 || (count > 0 && !sys)) return LS_ERR_ARG;
    if (count == 0) return LS_OK;
    for (int q = 0; q < count; q++) {
        const ls_system &S = sys[q];
        bool bad = S.n < 1 || S.n > LS_BATCH_MAX_N || S.nrhs < 1 || S.nrhs > LS_BATCH_MAX_RHS;
        bad = bad || S.lda < S.n || S.ldb < S.n || S.ldx < S.n || !S.A || !S.B || !S.X;
        bad = bad || (S.method != LS_METHOD_CG && S.method != LS_METHOD_GMRES);
        bad = bad || (S.method == LS_METHOD_GMRES && (S.opts.restart < 1 || S.opts.restart > E_MAXM));
        bad = bad || !(S.opts.rtol >= 0.0) || S.opts.max_iter < 0;
        if (bad) {   // name the offending system; nothing is solved
            if (infos) {
                memset(&infos[q], 0, sizeof(ls_info));
                infos[q].status = LS_ERR_ARG;
            }
            return LS_ERR_ARG;
        }
    }
    if (cudaSetDevice(c->device) != cudaSuccess) return LS_ERR_CUDA;

    // sizes and workspace
    std::vector<SlotSizes> z(count);
    std::vector<int> a_dev(count), b_dev(count), x_dev(count);
    size_t total = 0;
    int n32 = 0, nb32 = 0, n64 = 0, nv = 0;
    for (int q = 0; q < count; q++) {
        const ls_system &S = sys[q];
        z[q] = slot_sizes(c, S.n, S.nrhs, S.method, S.opts.restart);
        a_dev[q] = is_device_ptr(S.A);
        b_dev[q] = is_device_ptr(S.B);
        x_dev[q] = is_device_ptr(S.X);
        total += z[q].bytes + (a_dev[q] ? 0 : z[q].stageA) + (b_dev[q] ? 0 : z[q].stageBX) +
                 (x_dev[q] ? 0 : z[q].stageBX);
        const SlotTasks tk = slot_tasks(S.n, z[q].sp, z[q].ks32);
        n32 += tk.t32;
        nb32 += tk.rb32;
        n64 += tk.t64;
        nv += tk.tv;
    }
    int rc = ws_reserve(c, total);
    if (rc) return rc;
    if (!c->batch) c->batch = new (std::nothrow) Engine();
    if (!c->batch) return LS_ERR_NOMEM;
    Engine &E = *c->batch;
    rc = E.reserve(c, count, n32, nb32, n64, nv);
    if (rc) return rc;

    // carve, stage, describe
    std::vector<SlotDesc> hd(count);
    std::vector<const double *> bsrc(count);
    std::vector<long long> ldb(count), ldx(count);
    std::vector<double *> xdst(count), xstage(count, nullptr);
    char *p = c->ws;
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < count && e == cudaSuccess; q++) {
        const ls_system &S = sys[q];
        SlotDesc &D = hd[q];
        memset(&D, 0, sizeof(D));
        slot_carve(D, z[q], p, S.n, S.nrhs, S.method, S.opts.restart);
        p += z[q].bytes;
        D.inner_iters = S.method == LS_METHOD_CG ? (S.opts.inner_iters > 0 ? 4 * S.opts.inner_iters : 100)
                                                 : S.opts.restart;
        D.max_outer = S.opts.max_iter > 0 ? S.opts.max_iter : 20;
        D.inner_tol = S.opts.inner_rtol > 0.0 ? (float)S.opts.inner_rtol : 1e-6f;
        D.rtol = S.opts.rtol;
        if (a_dev[q]) {
            D.A64 = S.A;
            D.lda64 = S.lda;
        } else {
            double *st = reinterpret_cast<double *>(p);
            p += z[q].stageA;
            e = cudaMemcpy2DAsync(st, z[q].lda_stage * 8, S.A, S.lda * 8, S.n * 8, S.n,
                                  cudaMemcpyHostToDevice, c->stream);
            D.A64 = st;
            D.lda64 = z[q].lda_stage;
        }
        if (b_dev[q]) {
            bsrc[q] = S.B;
            ldb[q] = S.ldb;
        } else {
            double *st = reinterpret_cast<double *>(p);
            p += z[q].stageBX;
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(st, (size_t)S.n * 8, S.B, S.ldb * 8, S.n * 8, S.nrhs,
                                      cudaMemcpyHostToDevice, c->stream);
            bsrc[q] = st;
            ldb[q] = S.n;
        }
        if (x_dev[q]) {
            xdst[q] = S.X;
            ldx[q] = S.ldx;
        } else {
            xstage[q] = reinterpret_cast<double *>(p);
            p += z[q].stageBX;
            xdst[q] = xstage[q];
            ldx[q] = S.n;
        }
    }
    if (e != cudaSuccess) return map_cuda(e);
    E.set_tasks(hd, 0);
    rc = E.upload(hd, INT_MAX, true);
    if (!rc) rc = E.init_slots(0, count);
    if (!rc) rc = E.admit(0, count, bsrc, ldb);
    if (rc) return rc;
    const unsigned long long l0 = E.launches();
    e = cudaEventRecord(c->ev0, c->stream);
    if (e == cudaSuccess) rc = E.run();
    if (e == cudaSuccess && !rc) e = cudaEventRecord(c->ev1, c->stream);
    if (e != cudaSuccess || rc) return rc ? rc : map_cuda(e);
    std::vector<FinishItem> items(count);
    for (int q = 0; q < count; q++) items[q] = FinishItem{q, 0, sys[q].nrhs, xdst[q], ldx[q]};
    rc = E.finish(items);
    std::vector<SlotResult> res;
    if (!rc) rc = E.collect(0, count, res);
    if (rc) return rc;
    for (int q = 0; q < count && e == cudaSuccess; q++) {
        if (!xstage[q]) continue;
        const ls_system &S = sys[q];
        e = cudaMemcpy2DAsync(S.X, S.ldx * 8, xstage[q], (size_t)S.n * 8, S.n * 8, S.nrhs,
                              cudaMemcpyDeviceToHost, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return map_cuda(e);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    const long long launched = (long long)(E.launches() - l0) + 2;   // + admit, finish
    c->launches_total += launched + 2;                               // + init, collect
    int worst = LS_OK;
    for (int q = 0; q < count; q++) {
        const SlotResult &r = res[q];
        int st = r.status;
        if (st < 0 && worst >= 0) worst = st;
        else if (worst >= 0 && st > worst) worst = st;
        if (infos) {
            ls_info &I = infos[q];
            const double nn = (double)sys[q].n * sys[q].n;
            I.status = st;
            I.iters = r.inner;
            I.outer_iters = r.outer;
            I.rel_res = r.rel_res;
            I.true_rel_res = r.rel_res;
            I.time_ms = ms;
            I.bytes_moved = nn * (8.0 + 4.0) + (double)r.outer * 8.0 * nn + (double)r.inner * 4.0 * nn;
            I.launches = launched;
        }
    }
    return worst;
}
