// split_pair.h -- one FP64 value as the FP32 pair (hi, lo) of the solvers'
// storage: hi = fp32(v), lo = fp32(v - hi), each rounded to nearest, ties to
// even.  Host and device share this code (the host side is what the CPU test
// of the bit manipulation compiles).
//
// On this GPU the FP64 pipe runs at 1/64 of the FP32 rate, and the plain form
// (a double-to-float conversion, a float-to-double conversion, a subtraction
// and another conversion: four FP64-pipe instructions per element) bounds the
// split of A at about a third of HBM bandwidth.  For v = 0 and for binary
// exponents E in [-74, 126] the pair is formed instead from the bit pattern
// with 32-bit integer operations:
//   v = (-1)^s 2^E (1 + f 2^-52).  hi keeps the top 23 bits of f, rounded on
//   the 29 bits R below them: up when R > 2^28, or R = 2^28 and the kept bits
//   are odd (a carry out of the fraction raises the exponent field, which the
//   packed layout does by itself).
//   v - hi = (-1)^s (R - up 2^29) 2^(E-52) exactly, |R - up 2^29| <= 2^28, so
//   lo is that integer rounded to FP32 (an integer-to-float conversion, to
//   nearest even) times the power of two 2^(E-52): the product is exact
//   because E - 52 >= -126 keeps it a normal number.  A zero difference gives
//   +0, as the subtraction does.
// Other values (the residual in the subnormal range, |v| >= 2^127 where hi
// may overflow, subnormal v, infinities, NaN) take the plain form.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define LS_SPLIT_FN __host__ __device__ __forceinline__
#else
#define LS_SPLIT_FN inline
#endif

namespace lsi {

LS_SPLIT_FN float split_bits_to_float(uint32_t b) {
    float f;
    memcpy(&f, &b, 4);
    return f;
}

LS_SPLIT_FN uint32_t split_float_to_bits(float f) {
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
}

// The plain form: the conversions and the subtraction, each rounded to nearest.
LS_SPLIT_FN void split_pair_plain(double v, float &h, float &l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

#if defined(__CUDACC__)
// The plain form, out of line on the device: a call is a real branch, so the
// common path below never issues the plain form's FP64 instructions (an
// instruction whose predicate is off still takes an issue slot of its pipe,
// and the FP64 pipe runs at 1/64 of the FP32 rate).
static __device__ __noinline__ float2 split_pair_plain_call(double v) {
    float2 r;
    split_pair_plain(v, r.x, r.y);
    return r;
}
#endif

LS_SPLIT_FN void split_pair(double v, float &h, float &l) {
    uint64_t u;
    memcpy(&u, &v, 8);
    const uint32_t hw = (uint32_t)(u >> 32), lw = (uint32_t)u;
    const uint32_t s = hw & 0x80000000u;
    const int e = (int)((hw >> 20) & 0x7FFu);   // biased exponent: E = e - 1023
    if (((hw & 0x7FFFFFFFu) | lw) == 0u) {       // +0 or -0
        h = split_bits_to_float(s);
        l = 0.0f;
        return;
    }
    if (e < 1023 - 74 || e > 1023 + 126) {
#if defined(__CUDA_ARCH__)
        const float2 r = split_pair_plain_call(v);
        h = r.x;
        l = r.y;
#else
        split_pair_plain(v, h, l);
#endif
        return;
    }
    const uint32_t keep = ((hw & 0xFFFFFu) << 3) | (lw >> 29);   // top 23 bits of f
    const uint32_t R = lw & 0x1FFFFFFFu;                          // the 29 bits below them
    const uint32_t up = (R > 0x10000000u || (R == 0x10000000u && (keep & 1u))) ? 1u : 0u;
    h = split_bits_to_float((s | ((uint32_t)(e - 1023 + 127) << 23) | keep) + up);
    const int D = (int)R - (up ? 0x20000000 : 0);
    if (D == 0) {
        l = 0.0f;
        return;
    }
    const float scale = split_bits_to_float((uint32_t)(e - 1023 - 52 + 127) << 23);   // 2^(E-52)
#if defined(__CUDA_ARCH__)
    const float mag = __fmul_rn(__int2float_rn(D), scale);
#else
    const float mag = (float)D * scale;   // the host's default rounding: to nearest, ties to even
#endif
    l = split_bits_to_float(split_float_to_bits(mag) ^ s);
}

}  // namespace lsi
