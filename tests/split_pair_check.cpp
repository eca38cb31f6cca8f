// Host check of the bit-pattern FP32-pair split: split_pair must give the
// same bits as the plain conversions (split_pair_plain) for every input class.
// Prints "checked N mismatches M"; exit status 1 on a mismatch.
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>

#include "split_pair.h"

static uint64_t rng_state = 0x9E3779B97F4A7C15ull;
static uint64_t next_u64() {   // xorshift64*
    rng_state ^= rng_state >> 12;
    rng_state ^= rng_state << 25;
    rng_state ^= rng_state >> 27;
    return rng_state * 0x2545F4914F6CDD1Dull;
}
static double from_bits(uint64_t b) {
    double d;
    memcpy(&d, &b, 8);
    return d;
}
static double make(uint64_t sign, int E, uint64_t frac) {   // (-1)^sign 2^E (1 + frac 2^-52)
    return from_bits((sign << 63) | ((uint64_t)(E + 1023) << 52) | (frac & ((1ull << 52) - 1)));
}

static long long checked = 0, bad = 0;
static void check(double v) {
    float h1, l1, h2, l2;
    lsi::split_pair(v, h1, l1);
    lsi::split_pair_plain(v, h2, l2);
    checked++;
    const bool hn = std::isnan(h1) && std::isnan(h2), ln = std::isnan(l1) && std::isnan(l2);
    uint32_t a, b, c, d;
    memcpy(&a, &h1, 4);
    memcpy(&b, &h2, 4);
    memcpy(&c, &l1, 4);
    memcpy(&d, &l2, 4);
    if ((!hn && a != b) || (!ln && c != d)) {
        if (bad < 10)
            printf("mismatch v=%a: hi %08x vs %08x, lo %08x vs %08x\n", v, (unsigned)a, (unsigned)b, (unsigned)c,
                   (unsigned)d);
        bad++;
    }
}

int main() {
    // every bit pattern class: random 64-bit words
    for (int i = 0; i < 2000000; i++) check(from_bits(next_u64()));
    // the fast range and its borders, random fractions
    for (int E = -80; E <= 130; E++)
        for (int i = 0; i < 20000; i++) check(make(next_u64() & 1, E, next_u64()));
    // rounding cases on the 29 low bits: R = 0, 1, 2^28 - 1, 2^28 (ties), 2^28 + 1, 2^29 - 1,
    // kept bits even, odd, and all ones (carry into the exponent)
    const uint64_t Rs[] = {0, 1, (1u << 28) - 1, 1u << 28, (1u << 28) + 1, (1u << 29) - 1};
    const uint64_t keeps[] = {0, 1, 2, 3, 0x7FFFFE, 0x7FFFFF, 0x2AAAAA, 0x555555};
    for (int E = -80; E <= 130; E++)
        for (uint64_t k : keeps)
            for (uint64_t R : Rs)
                for (uint64_t sg = 0; sg < 2; sg++) check(make(sg, E, (k << 29) | R));
    // zeros, subnormals, infinities, NaN, extremes
    const double specials[] = {0.0, -0.0, 5e-324, -5e-324, 2.2250738585072009e-308, 2.2250738585072014e-308,
                               1e-300, -1e-300, 1e300, -1e300, 3.4028234663852886e38, 3.4028235677973366e38,
                               -3.4028235677973366e38, 1.7976931348623157e308, INFINITY, -INFINITY, NAN, 1.0,
                               -1.0, 0.1, 1.0 / 3.0, 1e-23, 1e-22, 1e-16};
    for (double v : specials) check(v);
    printf("checked %lld mismatches %lld\n", checked, bad);
    return bad ? 1 : 0;
}
