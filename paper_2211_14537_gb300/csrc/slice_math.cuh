// slice_math.cuh -- device arithmetic of the exact-slice table GEMM shared by
// its engines (gemm_frag.cu: mma.sync; gemm_ws.cu: tcgen05): splitting
// an FP64 vector into bf16 integer slices, and the epilogue.
//
// Slicing.  e = one more than the exponent of max|v| (frexp convention), so
// that max|v| < 2^(e-1); every element becomes the integer
// N = round(v 2^{8S-e}) (|N| < 2^39 for S = 5 slices), split into
// balanced base-256 digits from the bottom: the lower S-1 digits in
// [-128, 127], the top digit (the remainder) in [-128, 128].  Every digit is
// an integer of magnitude <= 128, exact in bf16 (8 significant bits).
// Integer arithmetic on the bit pattern only, apart from the exact digit ->
// bf16 conversion.
//
// Epilogue.  The order-d sum (0-based, products a_k b_l with k + l = d) of
// one inner index is at most (d + 1) 2^14 in magnitude, so over an inner
// dimension K it is an exact integer in fp32 while K (d + 1) <= 1024: every
// far-field pass with K <= 204 stays exact at five slices; the mma.sync
// engine splits longer inner dimensions into exact 64-deep chunks, and on
// tcgen05 only the last order (relative weight 2^-32; in the near field,
// K = 256, orders 0..3 stay exact) can round.  Each order sum converts exactly to
// int32, and N = sum_d acc_d 256^{S-1-d} is an exact int64 (|N| < 2^57 for
// S <= 5).  The output N 2^{e_row + e_pair + e_vec - 16 - 8(S-1)} m_pair is
// then one rounding of the slice-product sum: the int64 -> FP64 conversion,
// the power of two applied to the exponent field, and one FP64 multiply only
// for a pair scale that is not a power of two.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "gemm.cuh"   // kSlicesS (slices stored per operand), kSliceBitsB (bits per slice)

namespace vpx {

constexpr int kSliceMaxPerLane = 8;   // elements per lane when a warp slices one vector: Kpad <= 256

// the slicing exponent e of a vector from its largest |bit pattern| (|x|
// compares as its bit pattern): max|x| < 2^(e-1), one above the frexp
// exponent, so that the top digit stays within [-128, 128]; 0 for an
// all-zero vector
__device__ inline int slice_expo_of_bits(uint64_t mb) {
    if (mb == 0) return 0;
    const int bex = (int)(mb >> 52);
    if (bex != 0) return bex - 1021;
    int e = 0;
    frexp(__longlong_as_double((long long)mb), &e);   // subnormal maximum
    return e + 1;
}

// the slicing exponent of a warp's elements, given each lane's max |bit pattern|
__device__ inline int slice_warp_expo(uint64_t mb) {
    for (int o = 16; o; o >>= 1) {
        const uint64_t t = (uint64_t)__shfl_xor_sync(0xffffffffu, (long long)mb, o);
        mb = t > mb ? t : mb;
    }
    return slice_expo_of_bits(mb);
}

__device__ inline uint64_t slice_abs_bits(double x) {
    return (uint64_t)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// N = round(x 2^{8S-e}) for S = kSlicesS
__device__ inline int64_t slice_fixed_point(double x, int e) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0) return 0;   // zero or subnormal: below the last slice for any normal max
    const uint64_t m = (b & 0xfffffffffffffull) | (1ull << 52);
    const int sh = 1075 - ex - kSlicesS * kSliceBitsB + e;   // x 2^{8S-e} = m 2^{-sh}, sh >= 6
    if (sh >= 64) return 0;
    const int64_t n = (int64_t)((m + (1ull << (sh - 1))) >> sh);
    return (b >> 63) ? -n : n;
}

// digits of N, most significant first, as bf16 bit patterns
__device__ inline void slice_digits(int64_t n, uint16_t (&d)[kSlicesS]) {
#pragma unroll
    for (int k = kSlicesS - 1; k > 0; --k) {
        const int64_t up = (n + 128) >> 8;
        d[k] = __bfloat16_as_ushort(__float2bfloat16_rn((float)(n - up * 256)));
        n = up;
    }
    d[0] = __bfloat16_as_ushort(__float2bfloat16_rn((float)n));
}

struct SliceScale {
    double mul;     // pair scale / 2^e (1 when the scale is a power of two, else in [1, 2))
    int e;          // its exponent, including the vector's exponent and 2^-14
    int pow2;       // 1: the scale is a power of two (mul = 1, no multiply)
};

__device__ inline SliceScale slice_pair_scale(double scale, int extra_e) {
    SliceScale s;
    int e = 0;
    const double m = frexp(scale, &e);   // scale = m 2^e, |m| in [0.5, 1)
    s.pow2 = m == 0.5;
    s.mul = s.pow2 ? 1.0 : 2.0 * m;
    s.e = e - 1 + extra_e;
    return s;
}

// The bit pattern of (double)a, a > 0, rounded to nearest with ties to even,
// from integer operations only: the leading one at bit ex = 63 - clz(a); for
// ex > 52 the ex - 52 bits below the 53 kept are rounded off, a carry out of
// the 53 bits stepping the exponent field.  (The FP64 pipe, which the
// conversion would use, issues about two operations per clock per SM here.)
__device__ inline uint64_t slice_u64_to_f64_bits(uint64_t a) {
    const int ex = 63 - __clzll((long long)a);
    if (ex <= 52) return ((uint64_t)(ex + 1023) << 52) + ((a << (52 - ex)) - (1ull << 52));
    const int sh = ex - 52;
    const uint64_t q = a >> sh, r = a & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    const uint64_t m = q + ((r > half || (r == half && (q & 1ull))) ? 1ull : 0ull);
    return ((uint64_t)(ex + 1023) << 52) + (m - (1ull << 52));
}

// n 2^e as a double: one rounding (the conversion, as (double)n), the scaling
// exact; integer operations unless the result leaves the normal range
__device__ inline double slice_i64_scaled(int64_t n, int e) {
    if (n == 0) return 0.0;
    const uint64_t sgn = n < 0 ? (1ull << 63) : 0ull;
    const uint64_t b = slice_u64_to_f64_bits(n < 0 ? (uint64_t)0 - (uint64_t)n : (uint64_t)n);
    const int ne = (int)(b >> 52) + e;
    if (ne <= 0 || ne >= 2047) return ldexp(__longlong_as_double((long long)(b | sgn)), e);
    return __longlong_as_double((long long)((b + ((uint64_t)(int64_t)e << 52)) | sgn));
}

// acc[0] is the most significant order
template <int S>
__device__ inline double slice_output(const float (&acc)[S], const SliceScale &ps, int row_e) {
    static_assert(S <= 5, "more slices than the int64 recombination holds");
    int64_t n = __float2int_rn(acc[0]);
#pragma unroll
    for (int d = 1; d < S; ++d) n = n * 256 + __float2int_rn(acc[d]);
    const double v = slice_i64_scaled(n, row_e + ps.e - kSliceBitsB * (S - 1));
    return ps.pow2 ? v : v * ps.mul;
}

}  // namespace vpx
