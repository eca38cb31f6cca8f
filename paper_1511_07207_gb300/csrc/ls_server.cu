// ls_server.cu -- continuous-batching solve server (ls_server_* in ls.h).
//
// One scheduler thread per server owns a CUDA stream, a device memory pool of
// hbm_budget_bytes and an engine (ls_engine.h) with max_slots slots.  Its
// loop: admit queued requests while a slot is free and the request's device
// bytes fit in the pool (first fit, in arrival order); run the engine for
// step_iters ticks over every resident request; retire the requests that
// finished (write X, post the info, free the slot and its memory).  Requests
// that arrive while others are on the GPU join at the next step, and their
// work overlaps with the resident ones inside the same engine launches.
// With merge_rhs, queued requests that share their matrix (the same device
// A, lda, n, method and options) are admitted together as the right-hand-side
// columns of one slot (up to 32), so A is streamed once per step for all of
// them; every column still follows its own iteration.
// submit and poll only touch the host-side queue and result table, under a
// mutex, so any thread may call them.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "ls_api_internal.h"
#include "ls_engine.h"
#include "ls_engine_host.h"

using namespace lsi;
using Clock = std::chrono::steady_clock;

namespace {

// First-fit allocator over one device buffer; 256-byte granules.
class Pool {
public:
    char *base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;   // offset -> length

    int init(size_t bytes) {
        size = bytes / 256 * 256;
        if (cudaMalloc(&base, size) != cudaSuccess) {
            cudaGetLastError();
            base = nullptr;
            return LS_ERR_NOMEM;
        }
        free_.clear();
        free_[0] = size;
        return LS_OK;
    }
    void release() {
        if (base) cudaFree(base);
        base = nullptr;
    }
    char *alloc(size_t bytes) {
        bytes = align_up(bytes, 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                return base + off;
            }
        }
        return nullptr;
    }
    void free(char *p, size_t bytes) {
        bytes = align_up(bytes, 256);
        size_t off = (size_t)(p - base);
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + bytes == nx->first) {   // merge with the next block
            bytes += nx->second;
            free_.erase(nx);
        }
        auto pv = free_.lower_bound(off);
        if (pv != free_.begin()) {
            --pv;
            if (pv->first + pv->second == off) {                 // merge with the previous one
                off = pv->first;
                bytes += pv->second;
                free_.erase(pv);
            }
        }
        free_[off] = bytes;
    }
};

struct Request {
    uint64_t ticket;
    ls_system sys;                      // A borrowed if on the device; B always copied
    std::vector<double> hostA;          // copy of a host A (row-major, ld n)
    std::vector<double> hostB;          // copy of B (column-major, ld n)
    bool a_dev = false, x_dev = false;
    Clock::time_point t_submit;
    size_t bytes = 0;
    SlotSizes z{};
};

struct Member {
    Request req;
    int c0 = 0;                         // first column of the slot
    double *xstage = nullptr;           // device staging of a host X
};

struct Resident {
    std::vector<Member> m;              // requests sharing the slot (columns c0 ..)
    char *mem = nullptr;
    size_t bytes = 0;
    SlotSizes z{};
    int s = 0;                          // columns in use
    bool a_stage = false;               // A copied from the host (single member)
};

// Requests that may share a slot: the same device-resident A and options.
bool same_problem(const Request &a, const Request &b) {
    const ls_system &x = a.sys, &y = b.sys;
    return a.a_dev && b.a_dev && x.A == y.A && x.lda == y.lda && x.n == y.n && x.method == y.method &&
           x.opts.rtol == y.opts.rtol && x.opts.restart == y.opts.restart &&
           x.opts.inner_iters == y.opts.inner_iters && x.opts.inner_rtol == y.opts.inner_rtol &&
           x.opts.max_iter == y.opts.max_iter;
}

// Device bytes of a slot of s columns for the problem of `rq` (engine buffers,
// A's copy when it is on the host, B's staging, X's staging when any member's
// X is on the host).
size_t slot_bytes(const ls_ctx *c, const Request &rq, int s, bool any_host_x, SlotSizes *zo) {
    const ls_system &S = rq.sys;
    const SlotSizes z = slot_sizes(c, S.n, s, S.method, S.opts.restart);
    if (zo) *zo = z;
    return z.bytes + (rq.a_dev ? 0 : z.stageA) + z.stageBX + (any_host_x ? z.stageBX : 0);
}

}  // namespace

struct ls_server {
    ls_ctx *ctx = nullptr;
    ls_server_cfg cfg{};
    ls_ctx shadow;                      // the scheduler's own stream and events
    Pool pool;
    Engine eng;
    std::vector<SlotDesc> hd;           // slot table (n = 0: free)
    std::vector<int> used;
    std::vector<Resident> res;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, ls_info> done;
    std::unordered_set<uint64_t> pending;          // queued or resident tickets
    std::atomic<bool> stop{false};
    std::atomic<uint64_t> next_ticket{1};
    std::thread thr;
    int thread_err = LS_OK;
    int n_resident = 0;
    bool tables_dirty = true;

    void run();
    int admit_slot(std::vector<Request> &members, int slot);
    void retire(int slot, const SlotResult &r);
};

namespace {
constexpr int SERVER_MAX_N = LS_BATCH_MAX_N;
}

int ls_server::admit_slot(std::vector<Request> &members, int slot) {
    const Request &r0 = members[0];
    const ls_system S = r0.sys;         // a copy: the members are moved into the slot below
    int ncol = 0;
    bool any_host_x = false;
    for (const Request &q : members) {
        ncol += q.sys.nrhs;
        any_host_x = any_host_x || !q.x_dev;
    }
    Resident &R = res[slot];
    R.bytes = slot_bytes(&shadow, r0, ncol, any_host_x, &R.z);
    char *mem = pool.alloc(R.bytes);
    if (!mem) return LS_ERR_NOMEM;
    R.mem = mem;
    R.s = ncol;
    R.a_stage = !r0.a_dev;
    SlotDesc &D = hd[slot];
    memset(&D, 0, sizeof(D));
    slot_carve(D, R.z, mem, S.n, ncol, S.method, S.opts.restart);
    char *p = mem + R.z.bytes;
    D.inner_iters = S.method == LS_METHOD_CG ? (S.opts.inner_iters > 0 ? 4 * S.opts.inner_iters : 100)
                                             : S.opts.restart;
    D.max_outer = S.opts.max_iter > 0 ? S.opts.max_iter : 20;
    D.inner_tol = S.opts.inner_rtol > 0.0 ? (float)S.opts.inner_rtol : 1e-6f;
    D.rtol = S.opts.rtol;
    cudaStream_t st = shadow.stream;
    cudaError_t e = cudaSuccess;
    if (r0.a_dev) {
        D.A64 = S.A;
        D.lda64 = S.lda;
    } else {
        double *a = reinterpret_cast<double *>(p);
        p += R.z.stageA;
        e = cudaMemcpy2DAsync(a, R.z.lda_stage * 8, r0.hostA.data(), (size_t)S.n * 8, (size_t)S.n * 8,
                              S.n, cudaMemcpyHostToDevice, st);
        D.A64 = a;
        D.lda64 = R.z.lda_stage;
    }
    // B staging: the members' columns side by side (column-major, ld n)
    double *bstage = reinterpret_cast<double *>(p);
    p += R.z.stageBX;
    double *xstage = any_host_x ? reinterpret_cast<double *>(p) : nullptr;
    R.m.clear();
    int c0 = 0;
    for (Request &q : members) {
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(bstage + (size_t)c0 * S.n, q.hostB.data(), (size_t)S.n * q.sys.nrhs * 8,
                                cudaMemcpyHostToDevice, st);
        Member mb;
        mb.c0 = c0;
        mb.xstage = q.x_dev ? nullptr : xstage + (size_t)c0 * S.n;
        c0 += q.sys.nrhs;
        mb.req = std::move(q);
        R.m.push_back(std::move(mb));
    }
    used[slot] = 1;
    n_resident++;
    if (e != cudaSuccess) return map_cuda(e);
    return LS_OK;
}

void ls_server::retire(int slot, const SlotResult &r) {
    Resident &R = res[slot];
    std::vector<std::pair<uint64_t, ls_info>> out;
    for (const Member &mb : R.m) {
        const ls_system &S = mb.req.sys;
        ls_info info{};
        info.status = r.status;
        info.iters = r.inner;
        info.outer_iters = r.outer;
        double worst = 0.0;
        for (int j = mb.c0; j < mb.c0 + S.nrhs && j < E_MAXS; j++)
            worst = r.colres[j] > worst || r.colres[j] != r.colres[j] ? r.colres[j] : worst;
        info.rel_res = worst;
        info.true_rel_res = worst;
        info.time_ms = std::chrono::duration<double, std::milli>(Clock::now() - mb.req.t_submit).count();
        const double nn = (double)S.n * S.n;
        info.bytes_moved = (nn * 12.0 + r.outer * 8.0 * nn + r.inner * 4.0 * nn) / (double)R.m.size();
        out.emplace_back(mb.req.ticket, info);
    }
    pool.free(R.mem, R.bytes);
    R.mem = nullptr;
    R.m.clear();
    memset(&hd[slot], 0, sizeof(SlotDesc));
    used[slot] = 0;
    n_resident--;
    std::lock_guard<std::mutex> lk(mu);
    for (auto &o : out) {
        done[o.first] = o.second;
        pending.erase(o.first);
    }
}

void ls_server::run() {
    cudaSetDevice(ctx->device);
    const int cap = cfg.max_slots;
    std::vector<SlotResult> results;
    while (true) {
        // ---- admission (arrival order, first fit in the pool) ----
        std::vector<int> admitted;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (queue.empty() && n_resident == 0) {
                if (stop) break;
                cv.wait_for(lk, std::chrono::milliseconds(50));
                if (queue.empty()) continue;
            }
            if (stop) break;
            while (!queue.empty()) {
                int slot = -1;
                for (int q = 0; q < cap; q++)
                    if (!used[q]) { slot = q; break; }
                if (slot < 0) break;
                Request &rq = queue.front();
                if (rq.bytes > pool.size) {                 // can never fit (checked at submit too)
                    ls_info info{};
                    info.status = LS_ERR_NOMEM;
                    done[rq.ticket] = info;
                    pending.erase(rq.ticket);
                    queue.pop_front();
                    continue;
                }
                // the requests that share the head's matrix (bounded scan)
                std::vector<size_t> pick(1, 0);
                int ncol = rq.sys.nrhs;
                bool any_host_x = !rq.x_dev;
                if (cfg.merge_rhs && rq.a_dev) {
                    for (size_t i = 1; i < queue.size() && i < 4096 && ncol < LS_BATCH_MAX_RHS; i++) {
                        const Request &o = queue[i];
                        if (ncol + o.sys.nrhs > LS_BATCH_MAX_RHS || !same_problem(rq, o)) continue;
                        const bool hx = any_host_x || !o.x_dev;
                        if (slot_bytes(&shadow, rq, ncol + o.sys.nrhs, hx, nullptr) > pool.size) break;
                        pick.push_back(i);
                        ncol += o.sys.nrhs;
                        any_host_x = hx;
                    }
                }
                std::vector<Request> members;
                members.reserve(pick.size());
                for (size_t i : pick) members.push_back(std::move(queue[i]));
                for (size_t k = pick.size(); k-- > 0;) queue.erase(queue.begin() + (long)pick[k]);
                lk.unlock();
                int rc = admit_slot(members, slot);
                if (rc == LS_ERR_NOMEM && members.size() > 1) {
                    // not enough free memory for the merged slot: admit the head
                    // alone, requeue the others at the front
                    lk.lock();
                    for (size_t k = members.size(); k-- > 1;) queue.push_front(std::move(members[k]));
                    members.resize(1);
                    lk.unlock();
                    rc = admit_slot(members, slot);
                }
                lk.lock();
                if (rc == LS_ERR_NOMEM) {                   // wait for memory to free up
                    for (size_t k = members.size(); k-- > 0;) queue.push_front(std::move(members[k]));
                    break;
                }
                if (rc != LS_OK) {
                    for (const Member &mb : res[slot].m) {
                        ls_info info{};
                        info.status = rc;
                        done[mb.req.ticket] = info;
                        pending.erase(mb.req.ticket);
                    }
                    pool.free(res[slot].mem, res[slot].bytes);
                    res[slot].m.clear();
                    memset(&hd[slot], 0, sizeof(SlotDesc));
                    used[slot] = 0;
                    n_resident--;
                    continue;
                }
                admitted.push_back(slot);
            }
        }
        if (n_resident == 0) continue;
        // ---- publish the slot table (fixed task regions per slot, so the
        //      partial sums of resident slots keep their indices) ----
        const bool changed = !admitted.empty() || tables_dirty;
        if (changed) eng.set_tasks(hd, SERVER_MAX_N);
        int rc = eng.upload(hd, std::max(cfg.step_iters, 1), changed);
        tables_dirty = false;
        for (int s : admitted) {
            if (!rc) rc = eng.init_slots(s, 1);
            std::vector<const double *> bs(1, nullptr);
            std::vector<long long> lb(1, hd[s].n);
            // B was staged right after the slot's engine buffers and A's copy
            char *p = res[s].mem + res[s].z.bytes + (res[s].a_stage ? res[s].z.stageA : 0);
            bs[0] = reinterpret_cast<const double *>(p);
            if (!rc) rc = eng.admit(s, 1, bs, lb);
        }
        // ---- one step: step_iters ticks over every resident slot ----
        if (!rc) rc = eng.run();
        if (!rc) rc = eng.collect(0, cap, results);
        if (rc) {
            thread_err = rc;
            break;
        }
        std::vector<FinishItem> items;
        std::vector<int> fin;
        for (int s = 0; s < cap; s++) {
            if (!used[s] || !results[s].done) continue;
            for (const Member &mb : res[s].m) {
                const ls_system &S = mb.req.sys;
                items.push_back(FinishItem{s, mb.c0, S.nrhs, mb.xstage ? mb.xstage : S.X,
                                           mb.xstage ? (long long)S.n : S.ldx});
            }
            fin.push_back(s);
        }
        if (!items.empty()) {
            rc = eng.finish(items);
            for (int s : fin)
                for (const Member &mb : res[s].m) {
                    const ls_system &S = mb.req.sys;
                    if (!rc && mb.xstage)
                        rc = map_cuda(cudaMemcpy2DAsync(S.X, S.ldx * 8, mb.xstage, (size_t)S.n * 8,
                                                        (size_t)S.n * 8, S.nrhs, cudaMemcpyDeviceToHost,
                                                        shadow.stream));
                }
            if (!rc) rc = map_cuda(cudaStreamSynchronize(shadow.stream));
            for (int s : fin) {
                SlotResult r = results[s];
                if (rc) r.status = rc;
                retire(s, r);
            }
            tables_dirty = true;
        }
    }
    // cancel whatever is left (resident or queued)
    std::lock_guard<std::mutex> lk(mu);
    for (int s = 0; s < cap; s++) {
        if (!used[s]) continue;
        for (const Member &mb : res[s].m) {
            ls_info info{};
            info.status = thread_err ? thread_err : LS_NOT_CONVERGED;
            done[mb.req.ticket] = info;
            pending.erase(mb.req.ticket);
        }
        pool.free(res[s].mem, res[s].bytes);
        res[s].m.clear();
        used[s] = 0;
    }
    n_resident = 0;
    for (auto &rq : queue) {
        ls_info info{};
        info.status = LS_NOT_CONVERGED;
        done[rq.ticket] = info;
        pending.erase(rq.ticket);
    }
    queue.clear();
}

extern "C" int ls_server_start(ls_ctx *c, const ls_server_cfg *cfg, ls_server **out) {
    if (!c || !cfg || !out) return LS_ERR_ARG;
    *out = nullptr;
    if (cfg->max_slots < 1 || cfg->max_slots > 4096 || cfg->step_iters < 1 || cfg->queue_capacity < 1 ||
        cfg->hbm_budget_bytes < 4096)
        return LS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return LS_ERR_CUDA;
    ls_server *s = new (std::nothrow) ls_server();
    if (!s) return LS_ERR_NOMEM;
    s->ctx = c;
    s->cfg = *cfg;
    // the scheduler works on its own stream; the shadow context carries it
    s->shadow.device = c->device;
    s->shadow.num_sms = c->num_sms;
    s->shadow.K = c->K;
    if (cudaStreamCreateWithFlags(&s->shadow.stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return LS_ERR_CUDA;
    }
    int rc = s->pool.init(cfg->hbm_budget_bytes);
    const int cap = cfg->max_slots;
    const SlotTasks per = slot_tasks(SERVER_MAX_N, 32, E_KS32_MIN);   // the most tasks a slot can have
    if (!rc) rc = s->eng.reserve(&s->shadow, cap, cap * per.t32, cap * per.rb32, cap * per.t64, cap * per.tv);
    if (rc) {
        s->eng.release();
        s->pool.release();
        cudaStreamDestroy(s->shadow.stream);
        delete s;
        return rc;
    }
    s->hd.assign(cap, SlotDesc{});
    s->used.assign(cap, 0);
    s->res.resize(cap);
    s->thr = std::thread([s] { s->run(); });
    *out = s;
    return LS_OK;
}

extern "C" int ls_server_submit(ls_server *s, const ls_system *req, uint64_t *ticket) {
    if (!s || !req || !ticket) return LS_ERR_ARG;
    const ls_system &S = *req;
    if (S.n < 1 || S.n > SERVER_MAX_N || S.nrhs < 1 || S.nrhs > LS_BATCH_MAX_RHS || S.lda < S.n ||
        S.ldb < S.n || S.ldx < S.n || !S.A || !S.B || !S.X)
        return LS_ERR_ARG;
    if (S.method != LS_METHOD_CG && S.method != LS_METHOD_GMRES) return LS_ERR_ARG;
    if (S.method == LS_METHOD_GMRES && (S.opts.restart < 1 || S.opts.restart > E_MAXM)) return LS_ERR_ARG;
    if (!(S.opts.rtol >= 0.0) || S.opts.max_iter < 0) return LS_ERR_ARG;
    if (s->stop) return LS_ERR_BUSY;
    Request rq;
    rq.sys = S;
    rq.t_submit = Clock::now();
    cudaSetDevice(s->ctx->device);
    rq.a_dev = is_device_ptr(S.A) != 0;
    rq.x_dev = is_device_ptr(S.X) != 0;
    rq.bytes = slot_bytes(&s->shadow, rq, S.nrhs, !rq.x_dev, &rq.z);
    if (rq.bytes > s->pool.size) return LS_ERR_NOMEM;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if ((int)s->queue.size() >= s->cfg.queue_capacity) return LS_ERR_BUSY;
    }
    // deep copies: B always; A only when it lives in host memory
    rq.hostB.resize((size_t)S.n * S.nrhs);
    cudaError_t e = cudaMemcpy2D(rq.hostB.data(), (size_t)S.n * 8, S.B, S.ldb * 8, (size_t)S.n * 8, S.nrhs,
                                 cudaMemcpyDefault);
    if (e == cudaSuccess && !rq.a_dev) {
        rq.hostA.resize((size_t)S.n * S.n);
        e = cudaMemcpy2D(rq.hostA.data(), (size_t)S.n * 8, S.A, S.lda * 8, (size_t)S.n * 8, S.n,
                         cudaMemcpyDefault);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return LS_ERR_CUDA;
    }
    rq.sys.B = nullptr;                 // the copy is used from now on
    {
        std::lock_guard<std::mutex> lk(s->mu);
        rq.ticket = s->next_ticket++;
        *ticket = rq.ticket;
        s->pending.insert(rq.ticket);
        s->queue.push_back(std::move(rq));
    }
    s->cv.notify_one();
    return LS_OK;
}

extern "C" int ls_server_poll(ls_server *s, uint64_t ticket, int *done, ls_info *info) {
    if (!s || !done) return LS_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->done.find(ticket);
    if (it != s->done.end()) {
        *done = 1;
        if (info) *info = it->second;
        s->done.erase(it);
        return LS_OK;
    }
    if (!s->pending.count(ticket)) return LS_ERR_ARG;   // unknown, or already collected
    *done = 0;
    return LS_OK;
}

extern "C" int ls_server_stop(ls_server *s) {
    if (!s) return LS_ERR_ARG;
    s->stop = true;
    s->cv.notify_all();
    if (s->thr.joinable()) s->thr.join();
    cudaSetDevice(s->ctx->device);
    cudaStreamSynchronize(s->shadow.stream);
    s->eng.release();
    s->pool.release();
    cudaStreamDestroy(s->shadow.stream);
    const int err = s->thread_err;
    delete s;
    return err;
}
