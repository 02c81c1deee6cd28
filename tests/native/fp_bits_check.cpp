// Host check of the integer-unit float helpers (fp_bits.cuh, compiled here as plain C++)
// against the language's own conversions: every float32 bit pattern through f32_to_f64;
// seeded random, tie, carry and range-edge doubles through f64_to_f32_rn (against the cast,
// round to nearest even) and f64_to_f32_rz (the cast stepped one float32 toward zero where
// it rounded away from zero); the
// bit-pattern maximum of non-negative doubles against std::max.  Exits non-zero on the first
// mismatch, after printing it.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "fp_bits.cuh"

static uint64_t state = 0x243f6a8885a308d3ull;
static uint64_t next() {  // splitmix64
  uint64_t z = (state += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
static double from_bits(uint64_t u) {
  double x;
  std::memcpy(&x, &u, 8);
  return x;
}
static uint64_t bits64(double x) {
  uint64_t u;
  std::memcpy(&u, &x, 8);
  return u;
}
static uint32_t bits32(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}

// expected narrowing result under the helpers' range rules, with the cast for the normal range
static bool narrow_ok(double x, float got, bool rz) {
  const double ax = std::fabs(x);
  if (std::isnan(x)) return std::isnan(got);
  if (ax < 0x1p-126) return got == 0.0f && std::signbit(got) == std::signbit(x);
  if (ax >= 0x1p128) return std::isinf(got) && std::signbit(got) == std::signbit(x);
  float want = (float)x;  // round to nearest, ties to even (the default mode)
  if (rz && std::fabs((double)want) > ax) want = std::nextafterf(want, 0.0f);  // toward zero
  return bits32(got) == bits32(want);
}

static int check_narrow(double x) {
  const float rn = mpm::f64_to_f32_rn(x), rz = mpm::f64_to_f32_rz(x);
  if (!narrow_ok(x, rn, false)) {
    std::printf("f64_to_f32_rn mismatch: x=%a got=%a\n", x, (double)rn);
    return 1;
  }
  if (!narrow_ok(x, rz, true)) {
    std::printf("f64_to_f32_rz mismatch: x=%a got=%a\n", x, (double)rz);
    return 1;
  }
  return 0;
}

int main() {
  // widening: all 2^32 float32 patterns
  for (uint64_t k = 0; k < (1ull << 32); ++k) {
    const uint32_t b = (uint32_t)k;
    float f;
    std::memcpy(&f, &b, 4);
    const double got = mpm::f32_to_f64(f);
    const uint32_t mag = b & 0x7fffffffu;
    bool ok;
    if (mag >= 0x7f800000u) ok = std::isnan(got);
    else if (mag < 0x00800000u) ok = got == 0.0 && std::signbit(got) == std::signbit(f);
    else ok = bits64(got) == bits64((double)f);
    if (!ok) {
      std::printf("f32_to_f64 mismatch: pattern %08x got=%a\n", b, got);
      return 1;
    }
  }
  // narrowing: random doubles across (and beyond) the float32 range
  long long n = 0;
  for (int i = 0; i < 20000000; ++i, ++n) {
    const uint64_t r = next();
    const uint64_t e = 850 + (r >> 53) % 350;  // biased exponents 850..1199
    const double x = from_bits((r & 0x800fffffffffffffull) | (e << 52));
    if (check_narrow(x)) return 1;
  }
  // ties (the 29 dropped bits exactly half) with even and odd kept mantissas, carries into
  // the exponent, the largest float32 and its rounding to infinity, the normal-range edge
  for (int i = 0; i < 2000000; ++i, ++n) {
    const uint64_t r = next();
    const uint64_t e = 897 + (r >> 53) % 254;
    const uint64_t keep = (r >> 8) & 0x7fffffull;
    const uint64_t tail = (i % 4 == 0) ? 0x10000000ull : (i % 4 == 1) ? 0x0fffffffull : (i % 4 == 2) ? 0x10000001ull : 0;
    const double x = from_bits(((r & 1) << 63) | (e << 52) | (keep << 29) | tail);
    if (check_narrow(x)) return 1;
  }
  const double edges[] = {0.0, -0.0, 0x1p-126, -0x1p-126, 0x1.fffffffffffffp-127, 0x1p-127, 0x1.fffffep127,
                          0x1.fffffefffffffp127, 0x1.ffffffp127, 0x1p128, -0x1p128, 1.0, -1.0, 0x1.ffffffp0,
                          0x1.fffffffffffffp0, 3.0, 1.0 / 3.0, 1e300, -1e-300, INFINITY, -INFINITY, NAN};
  for (double x : edges) {
    ++n;
    if (check_narrow(x)) return 1;
  }
  // maximum of non-negative doubles on the bit patterns
  for (int i = 0; i < 5000000; ++i) {
    const double a = from_bits(next() & 0x7fefffffffffffffull), b = from_bits(next() & 0x7fefffffffffffffull);
    const double m = mpm::nn_max(a, b);
    if (bits64(m) != bits64(a > b ? a : b)) {
      std::printf("nn_max mismatch: %a %a -> %a\n", a, b, m);
      return 1;
    }
  }
  if (!std::isnan(mpm::nn_max(1.0, NAN)) || mpm::nn_max(0.0, 0x1p-1074) != 0x1p-1074) {
    std::printf("nn_max special case\n");
    return 1;
  }
  std::printf("ok: 2^32 widenings, %lld narrowings, 5000000 maxima\n", n);
  return 0;
}
