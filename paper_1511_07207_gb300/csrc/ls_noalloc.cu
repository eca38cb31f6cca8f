// ls_noalloc.cu -- y = A x for callers that cannot allocate device memory.
//
// ls_gemv needs a context, and creating one allocates the context's device
// block.  Some callers cannot do that: a process whose device memory is
// already fully reserved by a framework's caching allocator or a memory pool
// (a direct cudaMalloc would fail or fragment the pool), or a latency-bound
// loop that must not pay for cudaMalloc / cudaFree, which can synchronise the
// whole device.  ls_gemv_noalloc runs the same matrix-vector kernel with all
// of its scratch -- the matrix descriptor (TMA map), the small state block,
// the completion ticket, the per-CTA partial dot products and the partial
// row sums of row tiles shared between CTAs -- in one file-scope static
// device array of fixed size, which every GPU that loads this library holds
// until the process exits.  The caller passes only A, x and y.
#include <cuda_runtime.h>

#include <cstddef>
#include <cstring>
#include <mutex>

#include "ls_device.cuh"
#include "ls_internal.h"

using namespace lsi;

namespace {

// The static array is laid out as [MatDesc (512 B slot) | State | GemvScratch head + the
// partial sums of at most NOALLOC_MAX_CTAS CTAs].
constexpr size_t OFF_DESC = 0;
constexpr size_t OFF_STATE = 512;
constexpr size_t OFF_SCRATCH = OFF_STATE + ((sizeof(State) + 255) / 256) * 256;
constexpr size_t SCRATCH_HEAD = offsetof(GemvScratch, fix);
constexpr size_t NOALLOC_BYTES =
    OFF_SCRATCH + SCRATCH_HEAD + (size_t)LS_NOALLOC_MAX_CTAS * 2 * GEMV_MAX_TR * sizeof(double);
static_assert(sizeof(MatDesc) <= OFF_STATE, "descriptor slot");
static_assert(LS_NOALLOC_MAX_CTAS <= MAX_GRID, "scratch head holds MAX_GRID dots");
static_assert(NOALLOC_BYTES <= LS_NOALLOC_SCRATCH_BYTES, "static scratch too small");

__device__ __align__(256) unsigned char g_noalloc_scratch[LS_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char *g_dev_ptr[MAX_DEVICES] = {};
int g_sms[MAX_DEVICES] = {};

// Device address of the static array on the current device (looked up once
// per device; host code cannot use the symbol itself as an address).
int scratch_for_current_device(unsigned char **p, int *sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LS_ERR_CUDA;
    if (dev < 0 || dev >= MAX_DEVICES) return LS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
        void *addr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
        if (e != cudaSuccess || !addr) {
            cudaGetLastError();
            return LS_ERR_CUDA;
        }
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return LS_ERR_CUDA;
        }
        g_dev_ptr[dev] = static_cast<unsigned char *>(addr);
        g_sms[dev] = n;
    }
    *p = g_dev_ptr[dev];
    *sms = g_sms[dev];
    return LS_OK;
}

}  // namespace

extern "C" int ls_gemv_noalloc(int dtype, int rows, int cols, const void *A, int64_t lda,
                               const float *scale, const void *x, void *y, void *stream) {
    if (rows < 0 || cols < 0 || lda < cols || dtype < 0 || dtype > 4) return LS_ERR_ARG;
    if (dtype == DT_DS && (lda & 3)) return LS_ERR_ARG;
    if (rows == 0) return LS_OK;
    if (!A || !x || !y || (dtype == DT_FP8 && !scale)) return LS_ERR_ARG;
    unsigned char *base = nullptr;
    int sms = 0;
    int rc = scratch_for_current_device(&base, &sms);
    if (rc) return rc;
    GemvLaunch L = gemv_plan(dtype, true, EPI_STORE, sms);
    if (L.grid > LS_NOALLOC_MAX_CTAS) return LS_ERR_UNSUPPORTED;   // partial sums would not fit

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MatDesc hd;
    memset(&hd, 0, sizeof(hd));
    if (dtype == DT_DS) {   // the FP32 pair: hi rows, then lo rows, both with leading dimension lda
        const float *hi = static_cast<const float *>(A);
        make_tensor_map_ds(&hd, hi, hi + (long long)rows * lda, rows, cols, lda);
    } else {
        make_tensor_map(&hd, dtype, A, rows, cols, lda);
    }
    hd.scale = scale;
    L = gemv_plan(dtype, hd.use_tma != 0, EPI_STORE, sms);
    MatDesc *dA = reinterpret_cast<MatDesc *>(base + OFF_DESC);
    State *st = reinterpret_cast<State *>(base + OFF_STATE);
    GemvScratch *scr = reinterpret_cast<GemvScratch *>(base + OFF_SCRATCH);

    // The array keeps whatever the previous call left: rewrite the descriptor
    // and clear the state block and the completion ticket, which must start
    // at zero.  The partial sums are always written before they are read.
    cudaError_t e = cudaMemcpyAsync(dA, &hd, sizeof(MatDesc), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, sizeof(State), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(scr, 0, SCRATCH_HEAD, s);
    GemvArgs a{};
    a.x = x;
    a.y = y;
    a.st = st;
    a.scr = scr;
    a.epi = EPI_STORE;
    a.fin = FIN_STORE;
    if (e == cudaSuccess) e = gemv_launch(L, dA, a, s);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &st->err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return LS_ERR_CUDA;
    }
    return (err & ERRB_TIMEOUT) ? LS_ERR_TIMEOUT : LS_OK;
}
