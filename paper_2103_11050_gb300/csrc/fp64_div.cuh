// Float64 reciprocal and division for a part whose float64 pipe is narrow (on GB300 the
// correctly rounded float64 division costs tens of float64 instructions).
//
//   Seed y0 = 1/x in float32 (hardware approximation of the reciprocal of x truncated to
//   float32; relative error e0 below 2^-22 + 2^-23).  A Newton-Raphson step for
//   f(y) = 1/y - x, y <- y + y (1 - x y), squares the relative error (e1 <= e0^2 + 2^-53,
//   about 2^-44).
//   rcp64(x): two steps (error below the float64 rounding of the iteration).
//   div64(a, b): one step, q = a y1, then one residual correction q <- q + y1 (a - b q)
//             (Markstein, IBM J. Res. Dev. 34(1), 1990): with r = a - b q from one fused
//             multiply-add, the corrected quotient is off by about |r / b| e1, i.e. 2^-88
//             |a / b|, before its final rounding, so q is within one ulp of a / b whenever
//             a / b is a finite normal number.
// The range test on the divisor, its truncation to float32 and the widening of the seed back
// to float64 are integer repackings of the bit patterns (fp_bits.cuh): on GB300 the float64
// conversions would occupy the narrow float64 pipe.  A divisor outside [2^-125, 2^125) in
// magnitude (where the float32 seed or its reciprocal would not be a normal number), zero,
// infinite or NaN takes the IEEE division instead.
#pragma once

#include "fp_bits.cuh"

namespace mpm {

__device__ __forceinline__ float rcp_approx_f32(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// x and 1/x both float32 normal numbers (2^-125 <= |x| < 2^125, from the biased exponent
// field: 898 <= e <= 1147); xf = x truncated to float32.
__device__ __forceinline__ bool f32_seed_ok(double x, float& xf) {
  const uint64_t u = dbits(x);
  const uint32_t hi = (uint32_t)(u >> 32);
  const uint32_t e = (hi >> 20) & 0x7ffu;
  if (e - 898u > 249u) return false;  // unsigned: also rejects e < 898
  xf = f64_normal_to_f32_rz(hi, (uint32_t)u);
  return true;
}

// seed and one Newton-Raphson step (relative error about 2^-44)
__device__ __forceinline__ double newton_rcp1(double x, float xf) {
  const double y = f32_normal_to_f64(rcp_approx_f32(xf));  // a normal float32: exact widening
  return fma(y, fma(-x, y, 1.0), y);
}

__device__ __forceinline__ double newton_rcp(double x, float xf) {
  const double y = newton_rcp1(x, xf);
  return fma(y, fma(-x, y, 1.0), y);
}

__device__ __forceinline__ double rcp64(double x) {
  float xf;
  if (!f32_seed_ok(x, xf)) return 1.0 / x;
  return newton_rcp(x, xf);
}

__device__ __forceinline__ double div64(double a, double b) {
  float bf;
  if (!f32_seed_ok(b, bf)) return a / b;
  const double y = newton_rcp1(b, bf);
  const double q = a * y;
  return fma(fma(-b, q, a), y, q);
}

}  // namespace mpm
