// Conversions between binary32 and binary64 done with integer operations on
// the IEEE 754 encodings.
//
// The ELBM collision is bound by the FP64 pipe, which also executes the
// FP32 <-> FP64 conversion instructions; the integer pipes beside it are
// nearly idle.  These helpers move that work there.
// Encodings: binary32 = 1 sign bit, 8 exponent bits biased by 127, 23
// fraction bits; binary64 = 1, 11 biased by 1023, 52.  Each function
// states its domain and how its result relates to the conversion
// instruction it replaces.
//
// The header also compiles as plain C++ (no CUDA), so that host tests can
// check these functions against the C conversions.
#pragma once
#include <cstdint>
#include <cstring>
#if defined(__CUDACC__)
#define LBM_BITS_FN __host__ __device__ __forceinline__
#else
#define LBM_BITS_FN inline
#endif

namespace lbm {

LBM_BITS_FN uint32_t f32_bits(float v)
{
#if defined(__CUDA_ARCH__)
    return __float_as_uint(v);
#else
    uint32_t b;
    std::memcpy(&b, &v, 4);
    return b;
#endif
}

LBM_BITS_FN float f32_from_bits(uint32_t b)
{
#if defined(__CUDA_ARCH__)
    return __uint_as_float(b);
#else
    float v;
    std::memcpy(&v, &b, 4);
    return v;
#endif
}

LBM_BITS_FN uint64_t f64_bits(double v)
{
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(v);
#else
    uint64_t b;
    std::memcpy(&b, &v, 8);
    return b;
#endif
}

LBM_BITS_FN double f64_from_words(uint32_t hi, uint32_t lo)
{
#if defined(__CUDA_ARCH__)
    return __hiloint2double((int)hi, (int)lo);
#else
    const uint64_t b = ((uint64_t)hi << 32) | lo;
    double v;
    std::memcpy(&v, &b, 8);
    return v;
#endif
}

// (double)v, exactly, for every v.  A normal v (biased exponent 1..254)
// keeps its sign and fraction: the exponent is rebiased by 1023 - 127 = 896
// and the 23 fraction bits become the top of the 52, 20 in the high word and
// the low 3 at the top of the low word.  Infinities and NaN (exponent 255)
// take exponent 2047 the same way.  A subnormal v is first scaled by 2^64 in
// FP32 (exact: the product is normal) and its exponent then lowered by 64;
// a zero keeps its sign.
LBM_BITS_FN double widen(float v)
{
    const uint32_t b = f32_bits(v);
    const uint32_t mag = b & 0x7FFFFFFFu;
    const uint32_t e = mag >> 23;
    const uint32_t ms = f32_bits(v * 18446744073709551616.0f) & 0x7FFFFFFFu;
    const uint32_t m = e == 0u ? ms : mag;
    const uint32_t bias = e == 0u ? 832u : (e == 255u ? 1792u : 896u);
    const uint32_t hi = mag == 0u ? 0u : (m >> 3) + (bias << 20);
    return f64_from_words((b & 0x80000000u) | hi, m << 29);
}

// (double)v for a normal v (biased exponent 1..254) only, as widen does it.
LBM_BITS_FN double widen_normal(float v)
{
    const uint32_t b = f32_bits(v);
    return f64_from_words((b & 0x80000000u) | (((b & 0x7FFFFFFFu) >> 3) + (896u << 20)), b << 29);
}

// x truncated toward zero to 24 significant bits, as binary32: the high 23
// fraction bits are kept.  |x| below 2^-126 gives +-0 and |x| at or above
// 2^128 gives +-infinity (NaN: +-infinity as well).  Within the normal
// range the result is within one unit in the last place of (float)x.
LBM_BITS_FN float narrow_trunc(double x)
{
    const uint64_t b = f64_bits(x);
    const uint32_t hi = (uint32_t)(b >> 32);
    const uint32_t sign = hi & 0x80000000u;
    const uint32_t e = (hi >> 20) & 0x7FFu;
    const uint32_t mag = (uint32_t)((b & 0x7FFFFFFFFFFFFFFFull) >> 29) - (896u << 23);
    const uint32_t r = e < 897u ? 0u : (e > 1150u ? 0x7F800000u : mag);
    return f32_from_bits(sign | r);
}

// (float)x, rounded to nearest with ties to even, for every x (the value
// of the conversion instruction; NaN gives a NaN).  For a normal result the
// 52-bit fraction is rounded at bit 29: adding 2^28 - 1 plus the lowest kept
// bit and dropping 29 bits, where a carry steps the exponent (up to
// infinity, which is then the correctly rounded result); the exponent is
// rebiased by -896.  For a subnormal result (|x| < 2^-126) the significand
// 2^52 + fraction is shifted right by 926 - e (e the biased exponent) and
// rounded the same way by its remainder; below 2^-150 that is zero.
LBM_BITS_FN float narrow(double x)
{
    const uint64_t b = f64_bits(x);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const uint64_t mag = b & 0x7FFFFFFFFFFFFFFFull;
    const uint32_t e = (uint32_t)(mag >> 52);
    const uint32_t rn = (uint32_t)((mag + 0x0FFFFFFFull + ((mag >> 29) & 1u)) >> 29) - (896u << 23);
    const uint32_t sh = e >= 873u ? 926u - e : 54u;       // 30..53 for subnormal results
    const uint32_t s = sh > 53u ? 53u : sh;
    const uint64_t sig = (mag & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const uint64_t q = sig >> s;
    const uint64_t rem = sig & ((1ull << s) - 1u);
    const uint64_t half = 1ull << (s - 1u);
    const uint32_t rs = (uint32_t)q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u);
    const uint32_t sub = (sh > 53u || e == 0u) ? 0u : rs;
    const bool nan = e == 2047u && (mag & 0xFFFFFFFFFFFFFull) != 0u;
    const uint32_t r = e >= 897u ? (e >= 1151u ? (nan ? 0x7FC00000u : 0x7F800000u) : rn) : sub;
    return f32_from_bits(sign | r);
}

}  // namespace lbm
