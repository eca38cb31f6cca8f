// ls_device.cuh -- device helpers: mbarrier / TMA wrappers (inline PTX),
// bounded waits, deterministic reductions and a bounded grid barrier.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ls_internal.h"

namespace lsi {

// Every on-device wait gives up after this long (ns of %globaltimer), sets an
// error bit and returns, so no kernel can hang the GPU.
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;   // 2 s

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Sets a solver loop condition: through the graph handle, or into
// State::cond[h] when the loop runs from the host.
__device__ __forceinline__ void set_cond(State *st, cudaGraphConditionalHandle h, unsigned v) {
    if (*(volatile int *)&st->hostloop)
        ((volatile unsigned *)st->cond)[h & (LS_COND_SLOTS - 1)] = v;
    else
        cudaGraphSetConditional(h, v);
}

// ---- mbarrier ------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for phase `parity` of the barrier to complete; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    unsigned long long t0 = gtimer();
    while (!mbar_try_wait(bar, parity)) {
        if (gtimer() - t0 > WAIT_LIMIT_NS) return false;
    }
    return true;
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- TMA -----------------------------------------------------------------------
// The tensor map lives in global memory (written by the host between
// launches); acquire it for the async proxy before the first use.
__device__ __forceinline__ void tmap_acquire(const void *tmap) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap) : "memory");
}
__device__ __forceinline__ void tma_load_2d(void *smem_dst, const void *tmap, int x, int y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(smem_dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Contiguous copy global -> shared (both 16-byte aligned, bytes a multiple of
// 16), completion counted on the mbarrier.
__device__ __forceinline__ void bulk_load_1d(void *smem_dst, const void *gsrc, unsigned bytes,
                                             uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(smem_dst)),
        "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---- named barriers (a subset of the block's warps) ------------------------------------
__device__ __forceinline__ void named_bar(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
// Barrier that also returns the OR of `pred` over the participating threads.
__device__ __forceinline__ bool named_bar_or(int id, int nthreads, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

// ---- reductions ---------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; every thread gets the result.  `red` needs
// blockDim.x / 32 entries.  Fixed order, so deterministic.
template <class T>
__device__ __forceinline__ T block_sum(T v, T *red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    T s = 0;
    for (int i = 0; i < nw; i++) s += red[i];
    return s;
}

// ---- launch counting -----------------------------------------------------------------
__device__ __forceinline__ void count_launch(State *st) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&st->launches, 1ull);
}

__device__ __forceinline__ void set_err(State *st, int bits) { atomicOr(&st->err, bits); }

// ---- bounded grid barrier (cooperative launches only) ---------------------------------
struct GridBar {
    unsigned count;
    unsigned gen;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// atomicAdd with acquire-release ordering at GPU scope: publishes the
// writes that precede it (the CTA's, through a barrier) and, for the thread
// that sees the final count, makes the others' writes visible.
__device__ __forceinline__ int atom_add_acq_rel(int *p, int v) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// All blocks of the grid meet here.  Returns false (and sets ERRB_TIMEOUT)
// if the others did not arrive within WAIT_LIMIT_NS.
__device__ __forceinline__ bool grid_sync(GridBar *b, State *st) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned g = ld_acquire_u32(&b->gen);
        __threadfence();
        unsigned arrived = atomicAdd(&b->count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&b->count, 0u);
            __threadfence();
            st_release_u32(&b->gen, g + 1);
        } else {
            unsigned long long t0 = gtimer();
            unsigned ns = 32;
            while (ld_acquire_u32(&b->gen) == g) {
                __nanosleep(ns);
                if (ns < 256) ns <<= 1;
                if (gtimer() - t0 > WAIT_LIMIT_NS) {
                    set_err(st, ERRB_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// ---- grid-stride ranges --------------------------------------------------------------
// Balanced contiguous range [lo, hi) of 0..n for block `b` of `nb`.
__device__ __forceinline__ void block_range(long long n, int b, int nb, long long &lo,
                                            long long &hi) {
    lo = n * b / nb;
    hi = n * (b + 1) / nb;
}

}  // namespace lsi
