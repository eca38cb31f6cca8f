// k_selftest.cu -- self-test of the bounded on-device waits: an mbarrier
// that nothing completes and a grid barrier that one CTA never reaches.
// Each wait gives up after WAIT_LIMIT_NS, records ERRB_TIMEOUT in the state
// and returns, so the host reads LS_ERR_TIMEOUT and the context stays usable.
#include <cuda_runtime.h>

#include "ls_device.cuh"
#include "ls_internal.h"

namespace lsi {

__global__ void selftest_mbar_kernel(State *st) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(&bar, 0)) set_err(st, ERRB_TIMEOUT);   // nothing arrives
}

// Launched with 2 CTAs: CTA 1 leaves at once, CTA 0 waits for it at the barrier.
__global__ void selftest_grid_kernel(GridBar *bar, State *st) {
    if (blockIdx.x != 0) return;
    grid_sync(bar, st);            // gives up after the limit and sets ERRB_TIMEOUT itself
}

cudaError_t selftest_launch(int which, GridBar *bar, State *st, cudaStream_t s) {
    if (which == 0) selftest_mbar_kernel<<<1, 32, 0, s>>>(st);
    else selftest_grid_kernel<<<2, 32, 0, s>>>(bar, st);
    return cudaGetLastError();
}

}  // namespace lsi
