// Float64 reciprocal and division for a part whose float64 pipe is narrow (on GB300 the
// correctly rounded float64 division costs tens of float64 instructions).
//
//   rcp64(x): seed y0 = 1/x in float32 (hardware approximation of the reciprocal of x rounded
//             to float32, relative error < 2^-22), then two Newton-Raphson steps for f(y) =
//             1/y - x, y <- y + y (1 - x y), each squaring the relative error (2^-44, then
//             below the float64 rounding of the iteration itself).
//   div64(a, b): q = a rcp64(b), then one residual correction q <- q + rcp64(b) (a - b q)
//             (Markstein, IBM J. Res. Dev. 34(1), 1990), which leaves q within one ulp of
//             a / b whenever a / b is a finite normal number.
// A divisor outside [2^-125, 2^125] in magnitude (where the float32 seed or its reciprocal
// would not be a normal number), zero, infinite or NaN takes the IEEE division instead.
#pragma once

namespace mpm {

__device__ __forceinline__ float rcp_approx_f32(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// x and 1/x both float32 normal numbers: 2^-125 <= |x| <= 2^125.
__device__ __forceinline__ bool f32_seed_ok(double x, float& xf) {
  xf = __double2float_rn(x);
  const float ax = fabsf(xf);
  return ax >= 0x1p-125f && ax <= 0x1p125f;
}

__device__ __forceinline__ double newton_rcp(double x, float xf) {
  double y = (double)rcp_approx_f32(xf);
  y = fma(y, fma(-x, y, 1.0), y);
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
  const double y = newton_rcp(b, bf);
  const double q = a * y;
  return fma(fma(-b, q, a), y, q);
}

}  // namespace mpm
