// ls_tune.cu -- the tile-shape autotuner of the batched engine.
//
// Each slot of the batched / served engine (one dense system with s <= 32
// right-hand sides, padded to sp in {4, 8, 16, 32} columns) streams A in
// product tasks of 256 rows x ks32 columns and forms its inner block products
// either on the tensor cores (sp = 16, 32) or on the FP32 pipe.  Which is
// fastest depends on n (how many tasks a slot offers, how much split-K
// fix-up they need), on sp and on the GPU.  ls_autotune times every candidate
// (ks32 in {256, 512, 1024}; tensor cores or FP32 pipe) on synthetic batches
// of each size bucket [2^b, 2^(b+1)) and sp, and keeps the fastest in a JSON
// cache keyed by (bucket, sp, precision of the inner products, SM count).
// The engine looks a slot's choice up when it sizes the slot, so a slot's
// arithmetic depends only on its own n and s, never on the other slots.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "ls_api_internal.h"
#include "ls_engine.h"
#include "ls_engine_host.h"

namespace lsi {
namespace {

constexpr int BUCKET_MIN = 6, BUCKET_MAX = 13;   // n from 64 to LS_BATCH_MAX_N
constexpr int TUNE_REPS = 5;                     // timed runs per candidate (best of)
constexpr double TUNE_MARGIN = 0.03;             // a candidate must beat the default by 3 %

struct Table {
    std::mutex mu;
    bool loaded = false;                 // a file was read (or the tuner ran) in this process
    int sms = 0;                         // SM count the entries were timed on
    std::map<std::pair<int, int>, TuneChoice> entries;   // (bucket, sp) -> choice
};
Table &table() {
    static Table t;
    return t;
}

int bucket_of(int n) {
    int b = 0;
    while ((2 << b) <= n) b++;           // 2^b <= n < 2^(b+1)
    return std::min(std::max(b, BUCKET_MIN), BUCKET_MAX);
}

int sp_of(int s) { return s <= 4 ? 4 : s <= 8 ? 8 : s <= 16 ? 16 : 32; }

TuneChoice default_choice(int sp) { return TuneChoice{E_KS32, sp >= 16 ? 1 : 0}; }

// ---- a small reader for the cache format written by save_file ----------------------
// {"format": "ls-tune-1", "sms": 152, "precision": "fp32", "entries": [
//   {"bucket": 10, "sp": 32, "ks32": 512, "tc": 1, "ms": 1.25}, ...]}
bool find_int(const std::string &obj, const char *key, long *v) {
    const std::string k = std::string("\"") + key + "\"";
    size_t p = obj.find(k);
    if (p == std::string::npos) return false;
    p = obj.find(':', p + k.size());
    if (p == std::string::npos) return false;
    const char *c = obj.c_str() + p + 1;
    char *end = nullptr;
    const long x = strtol(c, &end, 10);
    if (end == c) return false;
    *v = x;
    return true;
}

int parse(const std::string &text, int *sms, std::map<std::pair<int, int>, TuneChoice> *out) {
    if (text.find("\"ls-tune-1\"") == std::string::npos) return LS_ERR_ARG;
    const size_t ep = text.find("\"entries\"");
    long v = 0;
    if (ep == std::string::npos || !find_int(text.substr(0, ep), "sms", &v) || v <= 0) return LS_ERR_ARG;
    *sms = (int)v;
    size_t p = text.find('[', ep);
    if (p == std::string::npos) return LS_ERR_ARG;
    const size_t close = text.find(']', p);
    if (close == std::string::npos) return LS_ERR_ARG;
    for (;;) {
        const size_t a = text.find('{', p);
        if (a == std::string::npos || a > close) break;
        const size_t b = text.find('}', a);
        if (b == std::string::npos || b > close) return LS_ERR_ARG;
        const std::string obj = text.substr(a, b - a + 1);
        long bucket, sp, ks, tc;
        if (!find_int(obj, "bucket", &bucket) || !find_int(obj, "sp", &sp) || !find_int(obj, "ks32", &ks) ||
            !find_int(obj, "tc", &tc))
            return LS_ERR_ARG;
        if (bucket < BUCKET_MIN || bucket > BUCKET_MAX || (sp != 4 && sp != 8 && sp != 16 && sp != 32) ||
            ks < E_KS32_MIN || ks > 4096 || ks % E_KC32 != 0 || (tc != 0 && tc != 1) || (tc && sp < 16))
            return LS_ERR_ARG;
        (*out)[{(int)bucket, (int)sp}] = TuneChoice{(int)ks, (int)tc};
        p = b + 1;
    }
    return LS_OK;
}

int load_file(const char *path) {
    FILE *f = fopen(path, "rb");
    if (!f) return LS_ERR_ARG;
    std::string text;
    char buf[4096];
    size_t k;
    while ((k = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, k);
    fclose(f);
    int sms = 0;
    std::map<std::pair<int, int>, TuneChoice> e;
    const int rc = parse(text, &sms, &e);
    if (rc) return rc;
    Table &t = table();
    std::lock_guard<std::mutex> lk(t.mu);
    t.entries = std::move(e);
    t.sms = sms;
    t.loaded = true;
    return LS_OK;
}

int save_file(const char *path, const std::map<std::pair<int, int>, std::pair<TuneChoice, double>> &rows,
              int sms) {
    FILE *f = fopen(path, "wb");
    if (!f) return LS_ERR_ARG;
    fprintf(f, "{\"format\": \"ls-tune-1\", \"sms\": %d, \"precision\": \"fp32\", \"entries\": [", sms);
    bool first = true;
    for (const auto &r : rows) {
        fprintf(f, "%s\n  {\"bucket\": %d, \"sp\": %d, \"ks32\": %d, \"tc\": %d, \"ms\": %.4f}", first ? "" : ",",
                r.first.first, r.first.second, r.second.first.ks32, r.second.first.tc, r.second.second);
        first = false;
    }
    fprintf(f, "\n]}\n");
    return fclose(f) == 0 ? LS_OK : LS_ERR_ARG;
}

// LS_ENGINE_TC=0..3 overrides the product form (bit 0: sp = 16, bit 1: sp = 32).
int env_tc(int sp, int tc) {
    const char *env = getenv("LS_ENGINE_TC");
    if (!(env && env[0] >= '0' && env[0] <= '3' && env[1] == 0)) return tc;
    const int bits = env[0] - '0';
    return sp == 16 ? (bits & 1) : sp == 32 ? ((bits >> 1) & 1) : 0;
}

}  // namespace

TuneChoice tune_choice(const ls_ctx *c, int n, int s) {
    const int sp = sp_of(s);
    TuneChoice ch = default_choice(sp);
    if (c && c->tune_ks32 > 0) {         // the tuner is timing a candidate
        ch.ks32 = c->tune_ks32;
        ch.tc = sp >= 16 ? c->tune_tc : 0;
        return ch;
    }
    Table &t = table();
    {
        std::lock_guard<std::mutex> lk(t.mu);
        if (!t.loaded) {                 // first lookup: the cache named by LS_TUNE_CACHE, if any
            t.loaded = true;
            const char *path = getenv("LS_TUNE_CACHE");
            if (path && *path) {
                t.mu.unlock();
                load_file(path);         // a missing or malformed file leaves the defaults
                t.mu.lock();
            }
        }
        if (c && t.sms == c->num_sms) {
            auto it = t.entries.find({bucket_of(n), sp});
            if (it != t.entries.end()) ch = it->second;
        }
    }
    ch.tc = env_tc(sp, ch.tc);
    return ch;
}

// Synthetic systems for the timings: A = 2 I + E, E symmetric with entries
// uniform in [-1/(2n), 1/(2n)] (eigenvalues within 2 +- 0.6/sqrt(n): the
// inner CG never breaks down), and B uniform in [-1, 1].
__device__ __forceinline__ double tune_hash(unsigned long long x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return (double)(x >> 11) * (1.0 / 9007199254740992.0);   // [0, 1)
}
__global__ void tune_fill_kernel(double *A, int n, unsigned seed) {
    const long long total = (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        const int lo = min(i, j), hi = max(i, j);
        const double r = tune_hash(((unsigned long long)seed << 40) ^ ((unsigned long long)lo << 20) ^ hi);
        A[e] = (i == j ? 2.0 : 0.0) + (r - 0.5) / n;
    }
}
__global__ void tune_rhs_kernel(double *B, long long count, unsigned seed) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
         e += (long long)gridDim.x * blockDim.x)
        B[e] = 2.0 * tune_hash(((unsigned long long)seed << 40) ^ (unsigned long long)e) - 1.0;
}

}  // namespace lsi

using namespace lsi;

extern "C" int ls_tune_load(const char *path) {
    if (!path) return LS_ERR_ARG;
    return load_file(path);
}

extern "C" int ls_tune_reset(void) {
    Table &t = table();
    std::lock_guard<std::mutex> lk(t.mu);
    t.entries.clear();
    t.sms = 0;
    t.loaded = true;                     // defaults; LS_TUNE_CACHE is not read again
    return LS_OK;
}

extern "C" int ls_tune_lookup(int n, int nrhs, int num_sms, int *ks32, int *tc) {
    if (n < 1 || nrhs < 1 || nrhs > LS_BATCH_MAX_RHS || num_sms < 1 || !ks32 || !tc) return LS_ERR_ARG;
    ls_ctx probe;                        // only num_sms is read
    probe.num_sms = num_sms;
    const TuneChoice ch = tune_choice(&probe, n, nrhs);
    *ks32 = ch.ks32;
    *tc = ch.tc;
    return LS_OK;
}

extern "C" int ls_autotune(ls_ctx *c, const char *path, int flags) {
    if (!c) return LS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return LS_ERR_CUDA;
    const bool quick = (flags & LS_TUNE_QUICK) != 0;
    const int bmin = quick ? 9 : BUCKET_MIN, bmax = quick ? 10 : BUCKET_MAX;
    std::map<std::pair<int, int>, std::pair<TuneChoice, double>> best;
    int rc = LS_OK;
    for (int b = bmin; b <= bmax && rc == LS_OK; b++) {
        const int n = std::min(LS_BATCH_MAX_N, 3 << (b - 1));            // 1.5 x 2^b
        const int tasks = ((n + E_RB32 - 1) / E_RB32) * ((n + E_KS32 - 1) / E_KS32);
        const int count = std::min(64, std::max(2, (4 * c->num_sms + tasks - 1) / tasks));
        double *A = nullptr, *Bm = nullptr, *X = nullptr;
        const size_t an = (size_t)n * n, bn = (size_t)n * LS_BATCH_MAX_RHS;
        cudaError_t e = cudaMalloc(&A, count * an * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&Bm, count * bn * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&X, count * bn * sizeof(double));
        for (int q = 0; q < count && e == cudaSuccess; q++) {
            tune_fill_kernel<<<2 * c->num_sms, 256, 0, c->stream>>>(A + q * an, n, 1000u * b + q);
            tune_rhs_kernel<<<2 * c->num_sms, 256, 0, c->stream>>>(Bm + q * bn, (long long)bn, 7000u * b + q);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = map_cuda(e);
        const int sps[4] = {4, 8, 16, 32};
        for (int si = 0; si < 4 && rc == LS_OK; si++) {
            const int sp = sps[si];
            if (quick && sp < 16) continue;
            std::vector<ls_system> sys(count);
            for (int q = 0; q < count; q++) {
                ls_system &S = sys[q];
                memset(&S, 0, sizeof(S));
                S.method = LS_METHOD_CG;
                S.n = n;
                S.nrhs = sp;
                S.A = A + q * an;
                S.lda = n;
                S.B = Bm + q * bn;
                S.ldb = n;
                S.X = X + q * bn;
                S.ldx = n;
                ls_opts_default(&S.opts);
                S.opts.rtol = 0.0;               // the same work for every candidate: one
                S.opts.max_iter = 1;             // refinement step of 32 inner iterations
                S.opts.inner_iters = 8;
                S.opts.inner_rtol = 1e-20;
            }
            std::vector<ls_info> info(count);
            double best_ms = 1e300, default_ms = 1e300;
            const TuneChoice def = default_choice(sp);
            TuneChoice best_ch = def;
            int last_kc = -1;
            for (int ks : {256, 512, 1024}) {
                const int kc = (n + ks - 1) / ks;
                if (kc == last_kc) continue;     // the same tasks as the previous width
                last_kc = kc;
                for (int tc = 0; tc <= (sp >= 16 ? 1 : 0) && rc == LS_OK; tc++) {
                    c->tune_ks32 = ks;
                    c->tune_tc = tc;
                    double ms = 1e300;
                    for (int rep = 0; rep < TUNE_REPS + 1 && rc == LS_OK; rep++) {   // the first warms up
                        const int st = ls_batch_solve(c, count, sys.data(), info.data());
                        if (st < 0) rc = st;
                        else if (rep > 0) ms = std::min(ms, info[0].time_ms);
                    }
                    c->tune_ks32 = -1;
                    c->tune_tc = -1;
                    if (rc != LS_OK) break;
                    if (ks == def.ks32 && tc == def.tc) default_ms = ms;
                    if (ms < best_ms) {
                        best_ms = ms;
                        best_ch = TuneChoice{ks, tc};
                    }
                }
            }
            // keep the default unless a candidate is clearly faster (timings of
            // a few milliseconds carry some percent of noise)
            if (best_ms > (1.0 - TUNE_MARGIN) * default_ms) {
                best_ch = def;
                best_ms = default_ms;
            }
            if (rc == LS_OK) best[{b, sp}] = {best_ch, best_ms};
        }
        cudaFree(A);
        cudaFree(Bm);
        cudaFree(X);
    }
    c->tune_ks32 = -1;
    c->tune_tc = -1;
    if (rc) return rc;
    {
        Table &t = table();
        std::lock_guard<std::mutex> lk(t.mu);
        if (t.sms != c->num_sms) t.entries.clear();
        for (const auto &r : best) t.entries[r.first] = r.second.first;
        t.sms = c->num_sms;
        t.loaded = true;
    }
    return path ? save_file(path, best, c->num_sms) : LS_OK;
}
