// df32.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo of
// two fp32 numbers (|lo| <= ulp(hi) / 2), about 48 significant bits.  Products
// are made error-free with fma, sums with Knuth's TwoSum.  FP64 issues at
// about 1/64 of the fp32 rate on this part, so a double-float multiply-add
// (about 12 fp32 operations) is several times faster than an FP64 one.
//
// Every operation whose rounding error is captured is written with the
// explicit _rn intrinsics, which the compiler never contracts into an fma.
#pragma once

#include <cstdint>

namespace vpx {

struct df32 {
    float hi, lo;
};

__host__ __device__ inline df32 df_split(double x) {
    const float h = (float)x;
    return df32{h, (float)(x - (double)h)};
}

__device__ inline double df_value(df32 a) { return (double)a.hi + (double)a.lo; }

// x * 2^e as a double, by moving the fp32 fields into the binary64 format;
// fp32 subnormals (far below any value they are added to here) become 0
__device__ inline double f32_scaled_to_f64(float x, int e) {
    const uint32_t b = __float_as_uint(x);
    const int ex = (int)((b >> 23) & 0xffu);
    if (ex == 0) return 0.0;
    const int be = ex - 127 + 1023 + e;
    if (be < 1 || be > 2046) return ldexp((double)x, e);
    const uint64_t bits = ((uint64_t)(b >> 31) << 63) | ((uint64_t)be << 52) | ((uint64_t)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
}

// (hi + lo) 2^e as a double: integer operations and one FP64 add
__device__ inline double df_to_f64_scaled(df32 a, int e) {
    return f32_scaled_to_f64(a.hi, e) + f32_scaled_to_f64(a.lo, e);
}

// x as hi + lo (|x - hi - lo| <= 2^-47 |x|) from the bit pattern, without FP64
// arithmetic: hi keeps the leading 24 significant bits (truncated), lo the
// next 29 rounded to fp32.  Exponents outside [-70, 100] take the FP64 route.
__device__ inline df32 df_split_bits(double x) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0) return df32{0.f, 0.f};   // zero or subnormal (below 2^-1022)
    const int e = ex - 1023;
    if (e < -70 || e > 100) return df_split(x);
    const uint32_t sign = (uint32_t)(b >> 63) << 31;
    const uint64_t m = b & 0xfffffffffffffull;
    const float hi = __uint_as_float(sign | ((uint32_t)(e + 127) << 23) | (uint32_t)(m >> 29));
    const uint32_t r = (uint32_t)(m & 0x1fffffffu);
    if (r == 0) return df32{hi, 0.f};
    // r 2^(e-52): convert the 29-bit integer, then move its exponent
    const uint32_t fb = __float_as_uint(__uint2float_rn(r));
    return df32{hi, __uint_as_float(sign | (fb + ((uint32_t)(e - 52) << 23)))};
}

// exact sum s + e = a + b (TwoSum)
__device__ inline void df_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// acc += a * b, without renormalising acc (call df_norm at the end of a sum)
__device__ inline void df_mac(df32 &acc, df32 a, df32 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    float s, t;
    df_two_sum(acc.hi, p, s, t);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, e));
}

__device__ inline df32 df_norm(df32 a) {
    const float s = __fadd_rn(a.hi, a.lo);
    return df32{s, __fsub_rn(a.lo, __fsub_rn(s, a.hi))};
}

__device__ inline df32 df_add(df32 a, df32 b) {
    float s, t;
    df_two_sum(a.hi, b.hi, s, t);
    return df_norm(df32{s, __fadd_rn(t, __fadd_rn(a.lo, b.lo))});
}

// sum over the 32 lanes of a warp
__device__ inline df32 df_warp_sum(df32 a) {
    a = df_norm(a);
    for (int o = 16; o; o >>= 1) {
        df32 b;
        b.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
        b.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
        a = df_add(a, b);
    }
    return a;
}

}  // namespace vpx
