// Conversions between IEEE 754 binary64 and binary32 in 32-bit integer
// arithmetic.  On GB300 a hardware conversion between double and float
// issues on the FP64 pipe, which runs at 1/64 of the FP32 rate; the k = 1
// set-up kernels are bound by that pipe, and about half of their FP64-pipe
// instructions are such conversions.  These routines do the same conversions
// on the integer ALU pipe.
//
// f64_to_f32_rn: the correctly rounded narrowing of IEEE 754-2008 (rounding
// attribute roundTiesToEven, Section 4.3.1): the result is the float nearest
// to x, ties to the one with an even significand; magnitudes that round
// beyond the largest finite float give infinity (Section 7.4), results below
// the normal range are the correctly rounded subnormals (gradual underflow),
// infinities keep their sign and a NaN gives a quiet NaN.
// f32_to_f64: the exact widening (every float is a double).
// Both are checked bit for bit against the GPU's own conversions in
// tests/test_gpu_convert.py.
#pragma once

#include <cuda_runtime.h>

namespace emin {

__device__ __forceinline__ float f64_to_f32_rn(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
    const unsigned sign = hi & 0x80000000u;
    const int E = (int)((hi >> 20) & 0x7ffu);  // biased exponent (bias 1023)
    const int fe = E - 896;                    // biased float exponent (bias 127)
    if (fe >= 1 && fe <= 254) {
        // normal range: keep the top 23 of the 52 fraction bits, round the
        // other 29 to nearest, ties to even; a carry out of the fraction
        // moves into the exponent (and from exponent 254 to infinity)
        const unsigned keep = ((hi & 0xfffffu) << 3) | (lo >> 29);
        const unsigned rem = lo & 0x1fffffffu;
        const unsigned up = (rem > 0x10000000u) || (rem == 0x10000000u && (keep & 1u));
        return __uint_as_float(sign | (((unsigned)fe << 23) + keep + up));
    }
    if (E == 0x7ff) {
        const bool nan = ((hi & 0xfffffu) | lo) != 0u;
        return __uint_as_float(sign | (nan ? 0x7fc00000u : 0x7f800000u));
    }
    if (fe > 254) return __uint_as_float(sign | 0x7f800000u);  // beyond the float range
    // below the normal range: the value is S 2^(E - 1075) with the 53-bit
    // significand S (E >= 1); in units of the smallest subnormal 2^-149 that
    // is S >> (sh) with sh = 926 - E >= 30; zero and double subnormals
    // (E = 0) lie far below half of 2^-149
    if (E == 0) return __uint_as_float(sign);
    const int sh = 926 - E;
    if (sh > 54) return __uint_as_float(sign);  // below half the smallest subnormal
    const unsigned long long S = (u & 0xfffffffffffffull) | 0x10000000000000ull;
    const unsigned long long keep = S >> sh;
    const unsigned long long rem = S & ((1ull << sh) - 1ull);
    const unsigned long long half = 1ull << (sh - 1);
    const unsigned long long up = (rem > half) || (rem == half && (keep & 1ull));
    // a carry into bit 23 gives the smallest normal float, as it should
    return __uint_as_float(sign | (unsigned)(keep + up));
}

__device__ __forceinline__ double f32_to_f64(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned sign = b & 0x80000000u;
    const unsigned fe = (b >> 23) & 0xffu, fm = b & 0x7fffffu;
    unsigned hi, lo;
    if (fe >= 1u && fe <= 254u) {
        hi = sign | ((fe + 896u) << 20) | (fm >> 3);
        lo = fm << 29;
    } else if (fe == 255u) {
        hi = sign | 0x7ff00000u | (fm >> 3) | (fm ? 0x80000u : 0u);  // NaN stays quiet
        lo = fm << 29;
    } else if (fm == 0u) {
        hi = sign;
        lo = 0u;
    } else {
        // float subnormal fm 2^-149: leading bit p (0..22) becomes the
        // implicit bit of a normal double with exponent p - 149
        const int p = 31 - __clz(fm);
        const unsigned long long m = ((unsigned long long)fm << (52 - p)) & 0xfffffffffffffull;
        hi = sign | ((unsigned)(p + 874) << 20) | (unsigned)(m >> 32);
        lo = (unsigned)m;
    }
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

// a value of the iteration type as a double (exact for both types)
__device__ __forceinline__ double as_f64(float f) { return f32_to_f64(f); }
__device__ __forceinline__ double as_f64(double d) { return d; }

}  // namespace emin
