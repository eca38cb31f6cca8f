// ls_ds.cuh -- double-single ("FP32 pair") arithmetic on the FP32 pipe.
//
// An FP64 matrix is kept as the pair hi = fp32(a), lo = fp32(a - hi) (about
// 48 significant bits) and every product a x is formed from the pair and the
// split of x with error-free transformations: Knuth's two-sum for additions
// and the FMA-based two-product for the leading product.  The accumulator
// (hi, lo) carries about 48 bits; the result is returned in FP64.  Used by
// the GEMV (k_gemv.cu) and by the fused small-system solvers (k_fused.cu).
#pragma once

#include <cuda_runtime.h>

namespace lsi {

// Double-single accumulator (hi, lo): hi + lo carries about 48 bits.
struct DSV {
    float h, l;
};
// (hi, lo) + (hi, lo): the high parts by two-sum (Knuth), every rounding
// error into lo.  The intrinsics keep the compiler from contracting or
// reassociating the error-free steps.
__device__ __forceinline__ DSV operator+(DSV a, DSV b) {
    const float s = __fadd_rn(a.h, b.h);
    const float bv = __fsub_rn(s, a.h);
    const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bv)), __fsub_rn(b.h, bv));
    return DSV{s, __fadd_rn(e, __fadd_rn(a.l, b.l))};
}
__device__ __forceinline__ DSV &operator+=(DSV &a, DSV b) { return a = a + b; }
__device__ __forceinline__ double to_double(DSV v) { return (double)v.h + (double)v.l; }
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ float to_double(float v) { return v; }
__device__ __forceinline__ float shfl_xor_v(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_xor_v(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ DSV shfl_xor_v(DSV v, int o) {
    return DSV{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
}
// acc += a x for a = ah + al, x = xh + xl: ah xh = p + e exactly (FMA gives
// the product error), the cross terms ah xl + al xh and e go to lo with the
// two-sum error of hi + p (al xl, below 2^-48 |a x|, is dropped).
__device__ __forceinline__ void ds_fma(float ah, float al, DSV x, DSV &acc) {
    const float p = __fmul_rn(ah, x.h);
    const float pe = fmaf(ah, x.h, -p);
    const float t = fmaf(al, x.h, fmaf(ah, x.l, pe));
    const float sh = __fadd_rn(acc.h, p);
    const float bv = __fsub_rn(sh, acc.h);
    const float er = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(sh, bv)), __fsub_rn(p, bv));
    acc.h = sh;
    acc.l = __fadd_rn(acc.l, __fadd_rn(t, er));
}
// An FP64 vector element as the (hi, lo) pair that multiplies the matrix.
__device__ __forceinline__ DSV ds_split(double v) {
    const float h = __double2float_rn(v);
    return DSV{h, __double2float_rn(v - (double)h)};
}

}  // namespace lsi
