// sph_bits.h -- exact IEEE 754 format conversions in integer arithmetic.
//
// GB300 runs FP64 at 1/64 of the FP32 rate, and a conversion to or from
// FP64 occupies the FP64 pipe like an FMA.  Kernels bound by that pipe (the
// bucket kernel) convert with these instead: integer shifts and adds on the
// ALU pipe, with results bit-identical to the hardware conversions
// (float -> double exact; double -> float rounded to nearest, ties to even,
// with subnormals, infinities and NaN; int times a power of two -> double
// exact).  Plain C++ with a host/device qualifier, so that a host test can
// check them against the host's own conversions.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define SPH_HD __host__ __device__ __forceinline__
#else
#define SPH_HD inline
#endif

namespace sph {
namespace bits {

SPH_HD uint32_t f_bits(float f)
{
#if defined(__CUDA_ARCH__)
    return __float_as_uint(f);
#else
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
#endif
}
SPH_HD float f_from(uint32_t u)
{
#if defined(__CUDA_ARCH__)
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}
SPH_HD uint64_t d_bits(double d)
{
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(d);
#else
    uint64_t u;
    memcpy(&u, &d, 8);
    return u;
#endif
}
SPH_HD double d_from(uint64_t u)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)u);
#else
    double d;
    memcpy(&d, &u, 8);
    return d;
#endif
}
// index of the highest set bit of x != 0
SPH_HD int top_bit(uint32_t x)
{
#if defined(__CUDA_ARCH__)
    return 31 - __clz(x);
#else
    return 31 - __builtin_clz(x);
#endif
}

// float -> double (exact)
SPH_HD double f2d(float f)
{
    const uint32_t u = f_bits(f);
    const uint64_t s = (uint64_t)(u >> 31) << 63;
    const uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    if (e == 0xffu)  // infinity or NaN (payload kept, quiet bit included)
        return d_from(s | (0x7ffull << 52) | ((uint64_t)m << 29));
    if (e != 0u) return d_from(s | ((uint64_t)(e + 896u) << 52) | ((uint64_t)m << 29));
    if (m == 0u) return d_from(s);  // signed zero
    // subnormal: m 2^-149 = 1.f 2^(p - 149), p the top bit of m
    const int p = top_bit(m);
    const uint64_t frac = (uint64_t)(m ^ (1u << p)) << (52 - p);
    return d_from(s | ((uint64_t)(p + 874) << 52) | frac);
}

// double -> float, rounded to nearest with ties to even (the IEEE default
// and the hardware's cvt.rn); a NaN gives a quiet NaN of the same sign
SPH_HD float d2f(double d)
{
    const uint64_t u = d_bits(d);
    const uint32_t s = (uint32_t)(u >> 63) << 31;
    const int E = (int)((u >> 52) & 0x7ffu);
    const uint64_t mant = u & 0xfffffffffffffull;
    if (E == 0x7ff) return f_from(s | 0x7f800000u | (mant ? 0x400000u | (uint32_t)(mant >> 29) : 0u));
    const int e = E - 896;  // biased float exponent
    if (e >= 0xff) return f_from(s | 0x7f800000u);  // |d| >= 2^128: infinity
    if (e >= 1) {
        // a carry out of the fraction raises the exponent (to infinity at the top)
        uint32_t f = ((uint32_t)e << 23) | (uint32_t)(mant >> 29);
        const uint32_t rem = (uint32_t)mant & 0x1fffffffu;
        f += (rem > 0x10000000u || (rem == 0x10000000u && (f & 1u))) ? 1u : 0u;
        return f_from(s | f);
    }
    // subnormal or zero result: sig 2^(E - 1075) in units of 2^-149 is
    // sig 2^-sh with sh = 926 - E >= 30
    if (E == 0) return f_from(s);  // below 2^-1022
    const int sh = 926 - E;
    if (sh >= 64) return f_from(s);
    const uint64_t sig = mant | (1ull << 52);
    const uint64_t q = sig >> sh, rem = sig & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    const uint64_t up = (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;
    return f_from(s | (uint32_t)(q + up));  // q + up = 2^23 is the smallest normal
}

// (double)v * q, exact, for q a positive normal power of two whose product
// with v stays normal (a grid index times the grid spacing)
SPH_HD double i2d_pow2(int v, double q)
{
    if (v == 0) return 0.0;
    const uint64_t s = v < 0 ? 1ull << 63 : 0ull;
    const uint32_t a = v < 0 ? 0u - (uint32_t)v : (uint32_t)v;
    const int p = top_bit(a);
    const uint64_t frac = (uint64_t)(a ^ (1u << p)) << (52 - p);
    const uint64_t Eq = (d_bits(q) >> 52) & 0x7ffu;
    return d_from(s | ((Eq + (uint64_t)p) << 52) | frac);
}

}  // namespace bits
}  // namespace sph
