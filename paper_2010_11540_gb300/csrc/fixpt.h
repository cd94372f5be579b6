// Exact split of a grid coordinate xi = (x - xmin) / h into its cell index
// floor(xi), the CIC fixed-point weight rint(frac(xi) * 2^20) (ties to even)
// and, when asked, the fraction frac(xi) as a double -- all from the IEEE-754
// bits of xi with integer instructions (on GB300 every FP64 instruction,
// conversions included, takes one of two FP64 slots per SM clock, while
// integer instructions are plentiful).  The results are the ones the float64
// formulas floor / subtract / multiply / rint give: floor(xi) and xi - floor(xi)
// are exact in float64, and so is the scaling by 2^20 before the rounding.
// Plain C++ so that host tests can compile it.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define SC_HD __host__ __device__ __forceinline__
#else
#define SC_HD inline
#include <string.h>
#endif

namespace sc {

SC_HD uint64_t f64_bits(double v) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(v);
#else
  uint64_t b;
  memcpy(&b, &v, 8);
  return b;
#endif
}

SC_HD double bits_f64(uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double v;
  memcpy(&v, &b, 8);
  return v;
#endif
}

SC_HD int clz64(uint64_t v) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)v);
#else
  return __builtin_clzll(v);
#endif
}

// float -> double by moving bits (IEEE 754 binary32 -> binary64: sign kept,
// exponent rebiased by 1023 - 127, significand extended with zeros), so that
// widening a float32 field value takes integer instructions instead of a
// conversion on the FP64 pipe.  Equal to (double)f for zero, normal, infinite
// and NaN values; a subnormal float (below 2^-126) becomes zero of its sign.
SC_HD double f32_widen(float f) {
#if defined(__CUDA_ARCH__)
  const uint32_t u = (uint32_t)__float_as_uint(f);
#else
  uint32_t u;
  memcpy(&u, &f, 4);
#endif
  const uint32_t mag = u & 0x7fffffffu;
  uint32_t hi = (mag >> 3) + 0x38000000u, lo = mag << 29;
  if (mag < 0x00800000u) hi = lo = 0u;                                  // zero, subnormal
  if (mag >= 0x7f800000u) hi = 0x7ff00000u | ((mag >> 3) & 0x000fffffu);  // infinity, NaN
  return bits_f64(((uint64_t)(hi | (u & 0x80000000u)) << 32) | lo);
}

// 0 <= xi < limit (finite; -0.0 counts as 0): true, with i = floor(xi), the
// fixed-point weight a = rint((xi - i) * 2^20) in [0, 2^20], and, if f is not
// NULL, *f = xi - i.  Otherwise false (outputs unspecified).  limit <= 2^30.
SC_HD bool cic_split(double xi, int limit, int& i, int& a, double* f) {
  uint64_t b = f64_bits(xi);
  if (b == 0x8000000000000000ull) b = 0;  // -0.0
  const int e = (int)(b >> 52);           // biased exponent; the sign bit pushes negatives past 2047
  if (e >= 1023 + 30) return false;       // negative, >= 2^30, infinite or NaN
  if (e < 1023 - 60) {                    // |xi| < 2^-60 (zero, subnormal): weight rounds to 0
    i = 0;
    a = 0;
    if (f) *f = xi == 0.0 ? 0.0 : xi;
    return limit > 0;
  }
  const uint64_t m = (b & ((1ull << 52) - 1)) | (1ull << 52);  // xi = m * 2^-sh
  const int sh = 1075 - e;                                      // 23 .. 112 fraction bits
  uint64_t frac;
  if (sh <= 52) {
    i = (int)(m >> sh);
    frac = m & ((1ull << sh) - 1);
  } else {
    i = 0;
    frac = m;
  }
  if ((unsigned)i >= (unsigned)limit) return false;
  // a = frac * 2^(20 - sh), rounded to nearest, ties to even
  const int s = sh - 20;  // 3 .. 92
  if (s >= 64) {
    a = 0;
  } else {
    uint64_t q = frac >> s;
    const uint64_t r = frac & ((1ull << s) - 1), half = 1ull << (s - 1);
    if (r > half || (r == half && (q & 1ull))) ++q;
    a = (int)q;
  }
  if (f) {
    if (frac == 0) {
      *f = 0.0;
    } else {
      const int h = 63 - clz64(frac);  // leading bit of frac (h <= 52)
      const uint64_t mant = (frac << (52 - h)) & ((1ull << 52) - 1);
      *f = bits_f64(((uint64_t)(h - sh + 1023) << 52) | mant);
    }
  }
  return true;
}

// 0 <= z < limit (finite; -0.0 counts as 0): true with k = floor(z).
SC_HD bool floor_index(double z, int limit, int& k) {
  uint64_t b = f64_bits(z);
  if (b == 0x8000000000000000ull) b = 0;
  const int e = (int)(b >> 52);
  if (e >= 1023 + 30) return false;
  if (e < 1023) {
    k = 0;
  } else {
    const uint64_t m = (b & ((1ull << 52) - 1)) | (1ull << 52);
    k = (int)(m >> (1075 - e));
  }
  return (unsigned)k < (unsigned)limit;
}

}  // namespace sc
