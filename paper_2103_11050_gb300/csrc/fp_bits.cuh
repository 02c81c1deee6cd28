// Float64 helpers that run on the integer units instead of the float64 pipe.
//
// GB300 issues two float64 operations per clock per SM, and its float64 conversions and
// comparisons (F2F, DSETP, max) share that pipe with the arithmetic.  On the refinement and
// transport paths the conversions between float32 and float64 and the maxima of the stopping
// tests took about as many float64-pipe slots as the arithmetic itself.  These helpers repack
// IEEE-754 bit patterns with 32-bit integer operations:
//
//   f32_to_f64(f)     float32 -> float64, exact for normal numbers and zeros; a subnormal
//                     float32 gives a zero of its sign, an infinity or NaN gives NaN.
//   f64_to_f32_rn(x)  float64 -> float32 rounded to nearest, ties to even (the IEEE default),
//                     for |x| in the float32 normal range; |x| < 2^-126 gives a zero of its
//                     sign, |x| >= 2^128 (and rounding up past the largest float32) gives an
//                     infinity of its sign, NaN gives NaN.
//   f64_to_f32_rz(x)  the same with truncation (round toward zero), for a seed that only needs
//                     a relative error below 2^-23; same range rules.
//   nn_bits / nn_from_bits / nn_max
//                     for non-negative doubles (+0 included, -0 excluded) the unsigned order
//                     of the bit patterns is the numeric order, so a maximum, or a comparison
//                     with a threshold, is a 64-bit integer compare.  A NaN pattern lies above
//                     every finite one and so propagates through a maximum and fails every
//                     "<= threshold" test.
//
// The header also compiles as plain C++ (host only) so that the conversions can be checked
// exhaustively against the language's own casts without a GPU.
#pragma once

#include <cstdint>
#include <cstring>
#ifndef __CUDACC__
#define MPM_HD inline
#else
#define MPM_HD __host__ __device__ __forceinline__
#endif

namespace mpm {

MPM_HD uint64_t dbits(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  std::memcpy(&u, &x, 8);
  return u;
#endif
}

MPM_HD double dfrom(uint32_t hi, uint32_t lo) {
#if defined(__CUDA_ARCH__)
  return __hiloint2double((int)hi, (int)lo);
#else
  const uint64_t u = ((uint64_t)hi << 32) | lo;
  double x;
  std::memcpy(&x, &u, 8);
  return x;
#endif
}

MPM_HD uint32_t fbits(float f) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(f);
#else
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
#endif
}

MPM_HD float ffrom(uint32_t u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, 4);
  return f;
#endif
}

// float64 biased exponent e maps to float32 biased exponent e - 896 (1023 - 127).
constexpr uint32_t kRebias = 896u;

// f a normal float32: the exponent and top 20 mantissa bits form the high word, the low 3
// mantissa bits the top of the low word.
MPM_HD double f32_normal_to_f64(float f) {
  const uint32_t b = fbits(f);
  return dfrom((b & 0x80000000u) | (((b & 0x7fffffffu) >> 3) + (kRebias << 20)), b << 29);
}

MPM_HD double f32_to_f64(float f) {
  const uint32_t b = fbits(f);
  const uint32_t mag = b & 0x7fffffffu;
  if (mag < 0x00800000u) return dfrom(b & 0x80000000u, 0u);  // zero or subnormal
  if (mag >= 0x7f800000u) return dfrom(0x7ff80000u, 0u);     // infinity or NaN
  return f32_normal_to_f64(f);
}

// x (words hi, lo) in the float32 normal range: its truncation to float32.
MPM_HD float f64_normal_to_f32_rz(uint32_t hi, uint32_t lo) {
  return ffrom((hi & 0x80000000u) | (((hi & 0x7fffffffu) - (kRebias << 20)) << 3) | (lo >> 29));
}

// Shared range handling of the two narrowing conversions: true when x (words hi, lo) lies
// in the float32 normal range, with its sign bit in s and its exponent-and-top-mantissa word
// in mag; otherwise the result pattern is in special.
MPM_HD bool f64_narrow_range(uint32_t hi, uint32_t lo, uint32_t& s, uint32_t& mag, uint32_t& special) {
  s = hi & 0x80000000u;
  mag = hi & 0x7fffffffu;
  const uint32_t e = mag >> 20;
  if (e < kRebias + 1u) {  // below 2^-126 (zeros and subnormals included)
    special = s;
    return false;
  }
  if (e > kRebias + 254u) {  // 2^128 and above, infinities, NaN
    const bool nan = e == 0x7ffu && ((mag & 0xfffffu) | lo) != 0u;
    special = nan ? 0x7fc00000u : (s | 0x7f800000u);
    return false;
  }
  return true;
}

MPM_HD float f64_to_f32_rz(double x) {
  const uint64_t u = dbits(x);
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  uint32_t s, mag, special;
  if (!f64_narrow_range(hi, lo, s, mag, special)) return ffrom(special);
  return f64_normal_to_f32_rz(hi, lo);
}

MPM_HD float f64_to_f32_rn(double x) {
  const uint64_t u = dbits(x);
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  uint32_t s, mag, special;
  if (!f64_narrow_range(hi, lo, s, mag, special)) return ffrom(special);
  uint32_t f = ((mag - (kRebias << 20)) << 3) | (lo >> 29);  // truncated magnitude
  const uint32_t rest = lo & 0x1fffffffu;                      // the 29 dropped bits
  const uint32_t half = 0x10000000u;
  // round to nearest, ties to even; a carry out of the mantissa steps the exponent (and
  // past the largest finite value gives the infinity pattern 0x7f800000)
  f += (rest > half || (rest == half && (f & 1u))) ? 1u : 0u;
  return ffrom(s | f);
}

MPM_HD uint64_t nn_bits(double x) { return dbits(x); }

MPM_HD double nn_from_bits(uint64_t u) { return dfrom((uint32_t)(u >> 32), (uint32_t)u); }

MPM_HD double nn_max(double a, double b) {
  const uint64_t x = nn_bits(a), y = nn_bits(b);
  return nn_from_bits(x > y ? x : y);
}

}  // namespace mpm

#undef MPM_HD
