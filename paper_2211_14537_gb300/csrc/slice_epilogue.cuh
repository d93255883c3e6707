// slice_epilogue.cuh -- the epilogue shared by both engines of the exact-slice
// table GEMM (gemm.cu: mma.sync, gemm_tc.cu: tcgen05).
//
// An output of the sliced GEMM is held as S fp32 order sums acc_d (each exact,
// an integer), worth  sum_d acc_d 2^{-7d} * 2^{e_row} * scale_p * 2^{e_vec - 14}.
// FP64 issues at about 2 operations per clock per SM on this part, 1/64 of the
// fp32 rate, so the epilogue keeps every step it can in fp32 and integer
// arithmetic:
//   1. recombine the orders into a double-float (hi, lo) with TwoSum in fp32
//      (hi + lo carries about 48 bits; both lie on the grid 2^{-7(S-1)}, so
//      neither is subnormal unless zero);
//   2. multiply by the pair scale held as a double-float mantissa (ph + pl in
//      [0.5, 1)) with an integer exponent, error-free product by fma;
//   3. build the two fp64 halves by writing the fp32 sign, exponent + the row
//      and pair exponents, and mantissa into an IEEE binary64 bit pattern
//      (integer operations only), then one fp64 add.
// Relative error per output is below 2^-46 of that output's own magnitude.
#pragma once

#include <cstdint>

namespace vpx {

struct SliceScale {
    float hi, lo;   // mantissa of the pair scale, hi + lo in [0.5, 1)
    int e;          // its exponent, including the vector's exponent and 2^-14
};

__device__ inline SliceScale slice_pair_scale(double scale, int extra_e) {
    SliceScale s;
    int e = 0;
    const double m = frexp(scale, &e);
    s.hi = (float)m;
    s.lo = (float)(m - (double)s.hi);
    s.e = e + extra_e;
    return s;
}

// x * 2^e as a double, by moving the fp32 fields into the binary64 format;
// fp32 subnormals (only from cancellation far below the grid) become 0.
__device__ inline double f32_scaled_to_f64(float x, int e) {
    const uint32_t b = __float_as_uint(x);
    const int ex = (int)((b >> 23) & 0xffu);
    if (ex == 0) return 0.0;
    const int be = ex - 127 + 1023 + e;
    if (be < 1 || be > 2046) return ldexp((double)x, e);
    const uint64_t bits = ((uint64_t)(b >> 31) << 63) | ((uint64_t)be << 52) | ((uint64_t)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
}

// acc[0] is the most significant order.  Returns the exact sum as hi + lo.
template <int S>
__device__ inline void slice_recombine(const float (&acc)[S], float &hi, float &lo) {
    hi = acc[S - 1];
    lo = 0.f;
#pragma unroll
    for (int d = S - 2; d >= 0; --d) {
        hi *= 0x1p-7f;
        lo *= 0x1p-7f;
        const float b = acc[d];
        const float sm = hi + b, bb = sm - hi;
        const float er = (hi - (sm - bb)) + (b - bb);
        hi = sm;
        lo += er;
        const float s2 = hi + lo;
        lo = lo - (s2 - hi);
        hi = s2;
    }
}

__device__ inline double slice_output(float hi, float lo, const SliceScale &ps, int row_e) {
    const float p = hi * ps.hi;
    float q = fmaf(hi, ps.hi, -p);
    q = fmaf(hi, ps.lo, q);
    q = fmaf(lo, ps.hi, q);
    const int E = row_e + ps.e;
    return f32_scaled_to_f64(p, E) + f32_scaled_to_f64(q, E);
}

}  // namespace vpx
