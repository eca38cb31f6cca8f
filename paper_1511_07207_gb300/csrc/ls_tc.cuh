// ls_tc.cuh -- 5th-generation tensor-core helpers (tcgen05, sm_103a), inline PTX.
//
// Used by the block products, the only dense contractions on the solver path:
// Y = A P with P a block of s right-hand-side directions.  One elected thread
// issues tcgen05.mma with both operands in shared memory (K-major, 128-byte
// swizzle, the layout a 2-D TMA copy with CU_TENSOR_MAP_SWIZZLE_128B writes);
// the accumulator lives in tensor memory (TMEM) and is read back with
// tcgen05.ld after a tcgen05.commit has arrived on an mbarrier.
//
// Shared-memory matrix descriptor (64 bits):
//   [0,14)  start address >> 4      [16,30) leading-dimension byte offset >> 4
//   [32,46) stride byte offset >> 4 [46,48) descriptor version (1)
//   [49,52) base offset (0: atoms 1024-byte aligned)  [61,64) swizzle (2 = 128 B)
// K-major, 128-byte swizzle: each row of the tile is 128 bytes of K (32 FP32
// values), rows in groups of 8 (1024 bytes, stride 1024); the 16-byte chunk j
// of row r sits at chunk position j ^ (r & 7).  Stepping along K inside the
// 128-byte row moves the start address by the step's bytes.
//
// Instruction descriptor of kind::tf32 (32 bits):
//   [4,6) accumulator format (1 = FP32), [7,10) A format, [10,13) B format
//   (2 = TF32), bit 15/16 A/B major-ness (0 = K-major), [17,23) N >> 3,
//   [24,29) M >> 4.
// The tensor core reads a TF32 operand from an FP32 word and keeps its sign,
// exponent and top 10 fraction bits.
#pragma once

#include <stdint.h>

#include "ls_device.cuh"

namespace lsi {

__device__ __forceinline__ uint64_t tc_desc_sw128(uint32_t smem_addr) {
    uint64_t d = 0;
    d |= (uint64_t)((smem_addr >> 4) & 0x3FFFu);
    d |= (uint64_t)(16u >> 4) << 16;         // leading byte offset (unused with this swizzle)
    d |= (uint64_t)(1024u >> 4) << 32;       // stride between 8-row groups
    d |= (uint64_t)1 << 46;                  // descriptor version
    d |= (uint64_t)2 << 61;                  // 128-byte swizzle
    return d;
}

__host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---- tensor memory allocation (one whole warp) ----------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t *slot_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// ---- ordering between thread barriers and tensor-core operations -------------------------
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy writes to shared memory become visible to the tensor core
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// D (+)= A B, A and B in shared memory, D in tensor memory (one thread).
__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                            bool accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}

// The mbarrier receives one arrival once every tcgen05.mma issued so far by
// this thread has completed.
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// Lane (warp quarter * 32 + lane), 16 consecutive 32-bit columns from col.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
        "%13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// The part of an FP32 value a TF32 operand keeps (low 13 fraction bits
// cleared).
__device__ __forceinline__ float tf32_head(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// x rounded to the nearest TF32 value (ties away from zero), as an FP32 word
// whose low 13 fraction bits are zero, so the tensor core reads it exactly.
// Integer operations on the bit pattern: adding half a TF32 unit to the
// magnitude and clearing the dropped bits rounds it; infinities stay
// infinities, values that round past the largest finite one become infinite.
__device__ __forceinline__ float tf32_rn(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

}  // namespace lsi
