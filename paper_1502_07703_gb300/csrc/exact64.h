// Exact integer slicing of FP64 values and exact recombination of slice-product sums, for
// FP64-accurate dot products sum_n x_n y_n on the tensor cores (slices as BF16, products summed
// in FP32, where every partial sum is an integer small enough to be exact).
//
// Slicing (ex64_slices): with E the largest biased exponent over a row of values (so every
// |x| < 2^(E-1022)), a value x is the 63-bit fixed-point integer X = trunc(|x| 2^(1085-E)). X plus
// C = sum_{i=1..7} 64 * 2^(56-7i) is cut into eight balanced base-128 digits: a_0 = (X+C) >> 56
// in [0, 128] and a_i = ((X+C) >> (56-7i) mod 128) - 64 in [-64, 63] for i = 1..7, all carrying
// the sign of x. Then sum_i a_i 2^(56-7i) = X - (X mod 128), so x is represented to within
// 2^-56 of the row's scale 2^(E-1022). Zeros and subnormals slice to zero.
//
// Products: with b_j the slices of the other operand (largest exponent F), sum_n x_n y_n =
// 2^(E+F-2058) sum_s 2^(-7s) G_s with G_s = sum_{i+j=s} sum_n a_i b_j. Every a_i and b_j is an
// integer of at most 8 significant bits (exact in BF16), |a_i b_j| <= 16384 for i = j = 0,
// <= 8192 when one index is 0 and <= 4096 otherwise, so |G_s| <= K 4096 (s + 3) (s >= 1) and
// K 16384 (s = 0) over K terms: below 2^22 for K <= 102, hence exact in an FP32 accumulator,
// and G_s + 1.5 * 2^23 has G_s in its low mantissa bits. Keeping s = 0..7 drops levels 8..14,
// whose pairs have both indices >= 1: together below 7.1 K 2^-58 of the scale 2^(E+F-2044).
//
// Recombination (ex64_combine): V = sum_{s=0..7} G_s 2^(7(7-s)) is an integer below 2^79 in
// magnitude, formed exactly as a 128-bit integer from two 64-bit partial sums and rounded once
// to the nearest FP64 (ties to even), then scaled by 2^(E+F-2107), with integer operations only
// (FP64 arithmetic runs at a small fraction of the integer rate on this GPU). Results below the
// normal range flush to zero.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define EX64_HD __host__ __device__ __forceinline__
#else
#define EX64_HD static inline
#endif

#if defined(__cplusplus)
namespace pyrdg {
#endif

EX64_HD uint64_t ex64_bits(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  __builtin_memcpy(&b, &x, 8);
  return b;
#endif
}

EX64_HD double ex64_from_bits(uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double x;
  __builtin_memcpy(&x, &b, 8);
  return x;
#endif
}

EX64_HD int ex64_clz64(uint64_t v) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)v);
#else
  return v ? __builtin_clzll(v) : 64;
#endif
}

// Biased exponent of x (0 for zero and subnormals).
EX64_HD int ex64_exp(double x) { return (int)((ex64_bits(x) >> 52) & 0x7FF); }

// Digit offset C = sum_{i=1..7} 64 * 2^(56-7i).
#define EX64_BALANCE 0x81020408102000ull

// X = trunc(|x| 2^(1085-E)) = (m 2^10) >> (E - e) for the 53-bit significand m and biased
// exponent e <= E of x (0 for zeros and subnormals).
EX64_HD uint64_t ex64_fixed(uint64_t bits, int E) {
  const int e = (int)((bits >> 52) & 0x7FF);
  const uint64_t m = e ? ((bits & ((1ull << 52) - 1)) | (1ull << 52)) << 10 : 0;
  const int sh = E - e;
  return sh < 64 ? m >> sh : 0;
}

// The eight signed balanced slices of x against the row exponent E.
EX64_HD void ex64_slices(double x, int E, int32_t a[8]) {
  const uint64_t b = ex64_bits(x);
  const uint64_t Xb = ex64_fixed(b, E) + EX64_BALANCE;
  const int32_t sg = (b >> 63) ? -1 : 1;
  a[0] = sg * (int32_t)(Xb >> 56);
  for (int i = 1; i < 8; ++i) a[i] = sg * ((int32_t)((Xb >> (56 - 7 * i)) & 127u) - 64);
}

// sum_s G_s 2^(7(7-s)) 2^Z rounded to the nearest FP64 (ties to even), Z = E + F - 2107 for
// row and column exponents E and F; G_s exact integers (|G_s| < 2^24).
EX64_HD double ex64_combine(const int32_t G[8], int Z) {
  // V = P1 2^35 + P2, both partial sums exact in 64 bits
  const int64_t P1 = (int64_t)G[0] * 16384 + (int64_t)G[1] * 128 + (int64_t)G[2];
  const int64_t P2 = (int64_t)G[3] * 268435456 + (int64_t)G[4] * 2097152 + (int64_t)G[5] * 16384 +
                     (int64_t)G[6] * 128 + (int64_t)G[7];
  // 128-bit two's complement hi:lo
  const uint64_t lo1 = (uint64_t)P1 << 35, lo2 = (uint64_t)P2;
  uint64_t lo = lo1 + lo2;
  uint64_t hi = (uint64_t)(P1 >> 29) + (uint64_t)(P2 >> 63) + (lo < lo1 ? 1u : 0u);
  const int neg = (int64_t)hi < 0;
  if (neg) {  // magnitude
    lo = ~lo + 1;
    hi = ~hi + (lo == 0 ? 1u : 0u);
  }
  if (hi == 0 && lo == 0) return 0.0;
  const int msb = hi ? 127 - ex64_clz64(hi) : 63 - ex64_clz64(lo);
  uint64_t mant;
  int bexp = msb + Z + 1023;  // biased exponent of the result
  if (msb <= 52) {
    mant = lo << (52 - msb);  // exact
  } else {
    const int sh = msb - 52;  // 1 .. 26 (|V| < 2^79)
    mant = (lo >> sh) | (hi << (64 - sh));
    const uint64_t rem = lo & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (mant & 1))) ++mant;
    if (mant >> 53) {
      mant >>= 1;
      ++bexp;
    }
  }
  if (bexp <= 0) return 0.0;
  if (bexp >= 2047) return ex64_from_bits(((uint64_t)neg << 63) | (0x7FFull << 52));
  return ex64_from_bits(((uint64_t)neg << 63) | ((uint64_t)bexp << 52) | (mant & ((1ull << 52) - 1)));
}

// The same sum to FP64 through floor(V / 2^8), which fits in 63 bits when |G_0| < 2^21 (K <= 127
// terms) and |G_s| < 2^22: one 64-bit integer, rounded once to nearest (ties to even) and scaled
// by 2^(Z+8). The result is within 2^(Z+8) plus half an ulp of V 2^Z, below the truncation of
// the dropped levels for K >= 1 (2^(Z+8) = 2^-55 of the scale 2^(E+F-2044)). On the device the
// integer-to-FP64 conversion instruction normalises and rounds (the same round to nearest, ties
// to even, of the same integer) and the scale is added to its exponent field; the host spells
// the normalisation and rounding out, with the same results.
EX64_HD double ex64_combine_fast(const int32_t G[8], int Z) {
  const int64_t v = (int64_t)G[0] * (1ll << 41) + (int64_t)G[1] * (1ll << 34) + (int64_t)G[2] * (1ll << 27) +
                    (int64_t)G[3] * (1ll << 20) + (int64_t)G[4] * (1ll << 13) + (int64_t)G[5] * 64 +
                    (((int64_t)G[6] * 128 + G[7]) >> 8);
#if defined(__CUDA_ARCH__)
  if (v == 0) return 0.0;
  const uint64_t b = (uint64_t)__double_as_longlong(__ll2double_rn(v));
  const int bexp = (int)((b >> 52) & 0x7FF) + Z + 8;
  if (bexp <= 0) return 0.0;
  if (bexp >= 2047) return ex64_from_bits((b & (1ull << 63)) | (0x7FFull << 52));
  return ex64_from_bits(b + ((uint64_t)(int64_t)(Z + 8) << 52));
#else
  const uint64_t sgn = (uint64_t)(v >> 63);  // 0 or all ones
  uint64_t m = ((uint64_t)v ^ sgn) - sgn;    // |v|
  if (m == 0) return 0.0;
  const int lz = ex64_clz64(m);
  m <<= lz;                         // leading one at bit 63
  uint64_t mant = m >> 11;          // 53 bits, leading one at bit 52
  const uint64_t rest = m & 0x7FF;  // round bit 10 and sticky bits
  mant += (rest > 0x400 || (rest == 0x400 && (mant & 1))) ? 1 : 0;
  const int bexp = 63 - lz + Z + 8 + 1023;  // biased exponent of |v| 2^(Z+8)
  if (bexp <= 0) return 0.0;
  if (bexp >= 2047) return ex64_from_bits((sgn << 63) | (0x7FFull << 52));
  // the leading one adds 1 to the exponent field; a rounding carry to 2^53 adds one more
  return ex64_from_bits((sgn << 63) | (((uint64_t)(bexp - 1) << 52) + mant));
#endif
}

#if defined(__cplusplus)
}  // namespace pyrdg
#endif
