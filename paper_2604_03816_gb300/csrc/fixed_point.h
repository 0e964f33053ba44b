// Exact fixed-point digit arithmetic of the complex128 tensor-core path (integer ops
// only; host and device).
//
// A row of doubles with largest biased exponent field E (zero and subnormals counted as
// 1) satisfies |x| < 2^e with e = E - 1022.  Each x becomes the integer
//     X = round(x 2^(53 - e)),  |X| < 2^53,
// written with six balanced base-512 digits
//     X = d0 2^45 + d1 2^36 + d2 2^27 + d3 2^18 + d4 2^9 + d5,
//     d0 in [-256, 256], d1..d5 in [-256, 255],
// so x 2^(8 - e) = d0 + d1 2^-9 + ... + d5 2^-45 to within 2^-46.  Every digit is an
// integer of at most 9 bits plus sign and so exact in FP16.  The digits come from the
// unsigned fields of Y = X + OFFSET, OFFSET = 256 (2^0 + 2^9 + ... + 2^45).
//
// A dot product of two such digit vectors, accumulated level by level (level s = all
// digit pairs with i + j = s), is put back together as a 64-bit integer Z and then turned
// into the nearest double of Z 2^p with integer operations (assemble), so that neither
// the split nor the recombination touches the FP64 pipe.
#pragma once

#include <math.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define FXP_HD __host__ __device__ __forceinline__
#else
#define FXP_HD inline
#endif

namespace fxp {

constexpr int DIGITS = 6;
constexpr int DBITS = 9;
constexpr uint64_t OFFSET = 256ull * ((1ull << 0) + (1ull << 9) + (1ull << 18) + (1ull << 27) +
                                      (1ull << 36) + (1ull << 45));
FXP_HD uint32_t exp_field(uint64_t bits) {
    const uint32_t e = (uint32_t)(bits >> 52) & 0x7FFu;
    return e ? e : 1u;
}

// X = x 2^(53 - e) rounded to nearest (ties away from zero), e = emax - 1022, for a
// finite x whose exponent field is at most emax.  Shifts of 54 or more give 0 (the
// magnitude is below 2^53 and the added half below 2^62), so the shift is clamped to 63.
FXP_HD int64_t to_fixed(uint64_t bits, uint32_t emax) {
    const uint32_t ef = (uint32_t)(bits >> 52) & 0x7FFu;
    uint64_t m = (bits & 0xFFFFFFFFFFFFFull) | (ef ? (1ull << 52) : 0ull);
    uint32_t sh = emax - (ef ? ef : 1u);
    sh = sh > 63u ? 63u : sh;
    m = (m + ((1ull << sh) >> 1)) >> sh;
    return (bits >> 63) ? -(int64_t)m : (int64_t)m;
}

// Unsigned field i (0 = most significant) of Y = X + OFFSET; the digit is field - 256.
FXP_HD uint32_t field(uint64_t y, int i) {
    return i == 0 ? (uint32_t)(y >> 45) : (uint32_t)(y >> (9 * (5 - i))) & 511u;
}

// The six digits d0..d5 of X (most significant first).
FXP_HD void digits(int64_t x, int (&d)[DIGITS]) {
    const uint64_t y = (uint64_t)x + OFFSET;
    for (int i = 0; i < DIGITS; ++i) d[i] = (int)field(y, i) - 256;
}

FXP_HD uint64_t bits_of(double x) {
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    __builtin_memcpy(&b, &x, 8);
    return b;
#endif
}

// Results outside the normal range: conversion and scaling in FP64 (rare).
#if defined(__CUDACC__)
__host__ __device__ __noinline__
#else
__attribute__((noinline)) inline
#endif
double assemble_slow(int64_t z, int p) {
    return ldexp((double)z, p);
}

// ---------------------------------------------------------------------------------------
// The kernel's forms of the same arithmetic, on 32-bit words (fewer instructions than
// generic 64-bit code).  Each has a test against the reference forms above.

// Digit-pair words: (field of re) in bits 0..9 and (field of im) in bits 16..25, each
// ORed into the FP16 pattern 0x6800, which then reads 2048 + 2 u; the kernel turns it
// into the digit u - 256 with one exact half2 multiply-add (x 0.5 - 1280).
constexpr uint32_t PAIR_BIAS = 0x68006800u;

FXP_HD uint32_t funnel_r(uint32_t lo, uint32_t hi, uint32_t sh) {   // (hi:lo) >> sh, sh < 32
#if defined(__CUDA_ARCH__)
    return __funnelshift_r(lo, hi, sh);
#else
    return sh ? (lo >> sh) | (hi << (32u - sh)) : lo;
#endif
}

FXP_HD uint32_t funnel_l(uint32_t lo, uint32_t hi, uint32_t sh) {   // high word of (hi:lo) << sh, sh < 32
#if defined(__CUDA_ARCH__)
    return __funnelshift_l(lo, hi, sh);
#else
    return sh ? (hi << sh) | (lo >> (32u - sh)) : hi;
#endif
}

FXP_HD uint32_t byte_perm(uint32_t x, uint32_t y, uint32_t sel) {
#if defined(__CUDA_ARCH__)
    return __byte_perm(x, y, sel);
#else
    const uint64_t v = ((uint64_t)y << 32) | x;
    uint32_t r = 0;
    for (int i = 0; i < 4; ++i) r |= (uint32_t)((v >> (8 * ((sel >> (4 * i)) & 7u))) & 0xFFu) << (8 * i);
    return r;
#endif
}

// Y' = 2 X + 1 + 2 OFFSET in words (yh:yl), so that Y' >> 1 = X + OFFSET, for one double
// (hi:lo words) on the grid of emax.  With M2 = 2 x 2^(53 - e) as a 54-bit magnitude and
// s the sign mask, X' = (M2 ^ s) >> sh (arithmetic) is floor(2 v) for v >= 0 and
// floor(2 v - 2^-sh) for v < 0 (v = x 2^(53 - e)); then floor((X' + 1) / 2) is v rounded
// to nearest with ties away from zero -- to_fixed() -- with no variable rounding constant,
// and shifts of 55 or more give X' in {0, -1}, i.e. X = 0, by themselves.
FXP_HD void offset_fixed(uint32_t hi, uint32_t lo, uint32_t emax, uint32_t &yh, uint32_t &yl) {
    const uint32_t ef = (hi >> 20) & 0x7FFu;
    const uint32_t mh = (hi & 0xFFFFFu) | (ef ? 0x100000u : 0u);
    uint32_t sh = emax - (ef ? ef : 1u);
    sh = sh > 63u ? 63u : sh;
    const uint32_t sg = (uint32_t)((int32_t)hi >> 31);
    const uint32_t ah = funnel_l(lo, mh, 1) ^ sg, al = (lo << 1) ^ sg;
    uint32_t xh, xl;
    if (sh < 32u) {
        xl = funnel_r(al, ah, sh);
        xh = (uint32_t)((int32_t)ah >> sh);
    } else {
        xl = (uint32_t)((int32_t)ah >> (sh - 32u));
        xh = (uint32_t)((int32_t)ah >> 31);
    }
    const uint64_t y = ((((uint64_t)xh) << 32) | xl) + (2ull * OFFSET + 1ull);
    yl = (uint32_t)y;
    yh = (uint32_t)(y >> 32);
}

// The six digit-pair words (most significant first) of the amplitude (re, im) from the
// Y' words of both parts: fields of Y' at bits 46 (ten bits), 37, 28, 19, 10 and 1.  A
// byte permute puts the two parts' 16-bit windows side by side, one shift and one
// mask-and-bias finish each word.
FXP_HD void digit_pair_words(uint32_t rh, uint32_t rl, uint32_t ih, uint32_t il, uint32_t (&w)[DIGITS]) {
    const uint32_t M9 = 0x01FF01FFu, M10 = 0x03FF03FFu;
    w[0] = ((byte_perm(rh, ih, 0x6521u) >> 6) & M10) | PAIR_BIAS;     // Y' bits 46..55
    w[1] = ((byte_perm(rh, ih, 0x5410u) >> 5) & M9) | PAIR_BIAS;      // 37..45
    w[2] = ((byte_perm(funnel_r(rl, rh, 24), funnel_r(il, ih, 24), 0x5410u) >> 4) & M9) | PAIR_BIAS;  // 28..36
    w[3] = ((byte_perm(rl, il, 0x7632u) >> 3) & M9) | PAIR_BIAS;      // 19..27
    w[4] = ((byte_perm(rl, il, 0x6521u) >> 2) & M9) | PAIR_BIAS;      // 10..18
    w[5] = ((byte_perm(rl, il, 0x5410u) >> 1) & M9) | PAIR_BIAS;      // 1..9
}

FXP_HD int clz32(uint32_t x) {
#if defined(__CUDA_ARCH__)
    return __clz((int)x);
#else
    return x ? __builtin_clz(x) : 32;
#endif
}

// An integer-valued float with |v| <= 2^22 as an int32: v + 1.5 2^23 is exact and its bit
// pattern is 0x4B400000 + v (FP32 steps by 1 on [2^23, 2^24]).
FXP_HD int32_t small_float_to_int(float v) {
    const float t = v + 12582912.0f;
    uint32_t b;
#if defined(__CUDA_ARCH__)
    b = __float_as_uint(t);
#else
    __builtin_memcpy(&b, &t, 4);
#endif
    return (int32_t)(b - 0x4B400000u);
}

// assemble() on 32-bit words: |Z| normalised to bit 63 with one funnel shift, rounded at
// bit 11, the exponent added to the high word.  |Z| < 2^32 (results 2^-20 and more below
// the row's scale, or zero) and results outside the normal range take the slow path.
FXP_HD double assemble_words(int64_t z, int p) {
    const uint32_t zh = (uint32_t)((uint64_t)z >> 32), zl = (uint32_t)z;
    const uint32_t sg = (uint32_t)((int32_t)zh >> 31);
    const uint64_t mag = ((((uint64_t)(zh ^ sg)) << 32) | (zl ^ sg)) + (uint64_t)(sg & 1u);
    const uint32_t mh = (uint32_t)(mag >> 32), ml = (uint32_t)mag;
    const int lz = clz32(mh);
    const int be = 63 - lz + p + 1023;
    if (mh == 0u || (unsigned)(be - 1) >= 2046u) return z == 0 ? 0.0 : assemble_slow(z, p);
    const uint32_t nh = funnel_l(ml, mh, (uint32_t)lz), nl = ml << lz;
    const uint32_t ql = funnel_r(nl, nh, 11), qh = nh >> 11;
    const uint32_t rest = nl & 0x7FFu;
    const uint32_t inc = (uint32_t)(rest > 0x400u) | ((uint32_t)(rest == 0x400u) & ql);
    const uint64_t q = ((((uint64_t)qh) << 32) | ql) + inc;
    const uint32_t hi = ((uint32_t)(q >> 32) + ((uint32_t)(be - 1) << 20)) | (sg & 0x80000000u);
    const uint64_t bits = (((uint64_t)hi) << 32) | (uint32_t)q;
    double out;
#if defined(__CUDA_ARCH__)
    out = __longlong_as_double((long long)bits);
#else
    __builtin_memcpy(&out, &bits, 8);
#endif
    return out;
}

// Z = i0 2^40 + i1 2^31 + i2 2^22 + i3 2^13 + i45 (the five level accumulators as
// integers) and the nearest double of Z 2^p.
FXP_HD double combine_words(int32_t i0, int32_t i1, int32_t i2, int32_t i3, int32_t i45, int p) {
    const int64_t z = (int64_t)i45 + (int64_t)i3 * (1ll << 13) + (int64_t)i2 * (1ll << 22) +
                      (int64_t)i1 * (1ll << 31) + (int64_t)i0 * (1ll << 40);
    return assemble_words(z, p);
}

// Nearest double to Z 2^p (ties to even), by integer operations while the result is a
// normal number.  Z is normalised so that its top bit is bit 63; bits 62..11 are the
// stored significand, bit 10 the rounding bit, bits 9..0 the sticky bits; adding the
// rounded 53-bit significand to (exponent - 1) << 52 carries into the exponent by itself.
FXP_HD double assemble(int64_t z, int p) {
    const uint64_t sgn = (uint64_t)z & (1ull << 63);
    const uint64_t mag = z < 0 ? 0ull - (uint64_t)z : (uint64_t)z;
#if defined(__CUDA_ARCH__)
    int lz = __clzll((long long)mag);
#else
    int lz = mag ? __builtin_clzll(mag) : 64;
#endif
    lz = lz > 63 ? 63 : lz;
    const int be = 63 - lz + p + 1023;               // biased exponent before rounding
    if ((unsigned)(be - 1) >= 2046u) return assemble_slow(z, p);
    const uint64_t m = mag << lz;
    uint64_t q = m >> 11;
    const uint64_t rest = m & 0x7FFull;
    q += (uint64_t)((rest > 0x400ull) | ((rest == 0x400ull) & (q & 1ull)));
    const uint64_t bits = sgn | (((uint64_t)(be - 1) << 52) + q);
    double out;
#if defined(__CUDA_ARCH__)
    out = __longlong_as_double((long long)bits);
#else
    __builtin_memcpy(&out, &bits, 8);
#endif
    return z == 0 ? 0.0 : out;
}

}  // namespace fxp
