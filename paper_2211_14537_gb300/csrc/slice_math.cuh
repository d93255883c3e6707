// slice_math.cuh -- device arithmetic of the exact-slice table GEMM shared by
// its engines (gemm.cu, gemm_frag.cu: mma.sync; gemm_tc.cu: tcgen05): splitting
// an FP64 vector into bf16 integer slices, and the epilogue.
//
// Slicing.  e = exponent of max|v| (frexp convention); every element becomes the
// integer N = round(v 2^{7S-e}) (|N| <= 2^42 for S = 6 stored slices), split
// into balanced base-128 digits from the bottom: the lower S-1 digits in
// [-64, 63], the top digit (the remainder) in [-128, 128].  Integer arithmetic
// on the bit pattern only, apart from the exact digit -> bf16 conversion.
//
// Epilogue.
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

#include <cuda_bf16.h>

#include <cstdint>

#include "df32.cuh"   // f32_scaled_to_f64
#include "gemm.cuh"   // kSlicesS (slices stored per operand), kSliceBitsB (bits per slice)

namespace vpx {

// exponent e of the largest |x| over a warp's elements, given each lane's
// max |bit pattern| (|x| compares as its bit pattern): max|x| in [2^{e-1}, 2^e)
__device__ inline int slice_warp_expo(uint64_t mb) {
    for (int o = 16; o; o >>= 1) {
        const uint64_t t = (uint64_t)__shfl_xor_sync(0xffffffffu, (long long)mb, o);
        mb = t > mb ? t : mb;
    }
    if (mb == 0) return 0;
    const int bex = (int)(mb >> 52);
    if (bex != 0) return bex - 1022;
    int e = 0;
    frexp(__longlong_as_double((long long)mb), &e);   // subnormal maximum
    return e;
}

__device__ inline uint64_t slice_abs_bits(double x) {
    return (uint64_t)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// N = round(x 2^{7S-e}) for S = kSlicesS
__device__ inline int64_t slice_fixed_point(double x, int e) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0) return 0;   // zero or subnormal: below the last slice for any normal max
    const uint64_t m = (b & 0xfffffffffffffull) | (1ull << 52);
    const int sh = 1075 - ex - kSlicesS * kSliceBitsB + e;   // x 2^{7S-e} = m 2^{-sh}, sh >= 11
    if (sh >= 64) return 0;
    const int64_t n = (int64_t)((m + (1ull << (sh - 1))) >> sh);
    return (b >> 63) ? -n : n;
}

// digits of N, most significant first, as bf16 bit patterns
__device__ inline void slice_digits(int64_t n, uint16_t (&d)[kSlicesS]) {
#pragma unroll
    for (int k = kSlicesS - 1; k > 0; --k) {
        const int64_t up = (n + 64) >> 7;
        d[k] = __bfloat16_as_ushort(__float2bfloat16_rn((float)(n - up * 128)));
        n = up;
    }
    d[0] = __bfloat16_as_ushort(__float2bfloat16_rn((float)n));
}

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
    const float p = __fmul_rn(hi, ps.hi);   // kept a rounded product: q below is its exact error
    float q = fmaf(hi, ps.hi, -p);
    q = fmaf(hi, ps.lo, q);
    q = fmaf(lo, ps.hi, q);
    const int E = row_e + ps.e;
    return f32_scaled_to_f64(p, E) + f32_scaled_to_f64(q, E);
}

}  // namespace vpx
